"""Discrete-velocity sets (Appendix A, Eqs. d2q9 and d3q19).

Test infrastructure (FP64 oracle).  The orderings are the ones the paper lists;
``opp`` is the opposite-direction table k -> kbar.  Pinned by the quadrature
identities in tests/test_oracle_kinetics.py (sum w = 1, sum w c = 0,
sum w c c = cs^2 I) and the opposite-table check c[opp[k]] = -c[k].
"""
from dataclasses import dataclass

import numpy as np

CS2 = 1.0 / 3.0  # squared lattice sound speed (Section 2.2.1)


@dataclass(frozen=True)
class Lattice:
    name: str
    d: int
    c: np.ndarray    # (Q, d) integer velocities, column alpha = component alpha
    w: np.ndarray    # (Q,) weights
    opp: np.ndarray  # (Q,) opposite direction

    @property
    def Q(self) -> int:
        return self.c.shape[0]


def _d2q9() -> Lattice:
    cx = [0, 1, 0, -1, 0, 1, -1, -1, 1]
    cy = [0, 0, 1, 0, -1, 1, 1, -1, -1]
    w = [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4
    opp = [0, 3, 4, 1, 2, 7, 8, 5, 6]
    return Lattice("D2Q9", 2, np.array([cx, cy], dtype=np.int64).T.copy(),
                   np.array(w, dtype=np.float64), np.array(opp, dtype=np.int64))


def _d3q19() -> Lattice:
    cx = [0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0]
    cy = [0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1]
    cz = [0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1]
    w = [1 / 3] + [1 / 18] * 6 + [1 / 36] * 12
    opp = [0, 2, 1, 4, 3, 6, 5, 8, 7, 10, 9, 12, 11, 14, 13, 16, 15, 18, 17]
    return Lattice("D3Q19", 3, np.array([cx, cy, cz], dtype=np.int64).T.copy(),
                   np.array(w, dtype=np.float64), np.array(opp, dtype=np.int64))


D2Q9 = _d2q9()
D3Q19 = _d3q19()


def lattice_for_dim(d: int) -> Lattice:
    if d == 2:
        return D2Q9
    if d == 3:
        return D3Q19
    raise ValueError("only d = 2 (D2Q9) and d = 3 (D3Q19) are defined")
