"""Host-side diagnostics of a march, from the statistics the device records (no device work).

* ``rho_observed`` - the measured contraction factor of an inner-residual history, the tail geometric
  mean of successive residual ratios (Eq. rho-observed): exp of the mean of log(R_j / R_{j-1}) over the
  last m_rho ratios, m_rho = min(m, l_f - 1), undefined (None) with fewer than three residuals.
* ``step_residuals`` - the flat residual history of a march call split into its physical steps.
* ``work_ratio`` - the fine-grid-equivalent work ratio S_work = n_ref / W (Eq. swork), n_ref =
  T_end / dt_ac with the acoustic step dt_ac = 1 lattice time unit, W = kinetic maps (one per inner
  sweep) + periodic spectral corrections (one per inner sweep that was not accepted), both weight one.
"""
import math
from typing import List, Optional, Sequence


def rho_observed(residuals: Sequence[float], m: int = 10) -> Optional[float]:
    """m = 10 for D2Q9 runs, 8 for D3Q19 (Section 4.1)."""
    R = [float(r) for r in residuals]
    lf = len(R)
    if lf < 3:
        return None
    m_rho = min(m, lf - 1)
    acc = 0.0
    for j in range(lf - m_rho, lf):
        acc += math.log(R[j] / R[j - 1])
    return math.exp(acc / m_rho)


def step_residuals(history: Sequence[float], step_iters: Sequence[int]) -> List[List[float]]:
    """Split the residual history of one march call (oldest first) by the accepted inner counts."""
    out, pos = [], 0
    for k in step_iters:
        out.append([float(r) for r in history[pos:pos + int(k)]])
        pos += int(k)
    if pos != len(history):
        raise ValueError("residual history and step counts disagree (history ring overwritten?)")
    return out


def work_ratio(t_end: float, inner_sweeps: int, steps: int, corrector: bool = True) -> float:
    """S_work for a run of `steps` accepted physical steps and `inner_sweeps` kinetic maps."""
    corrections = (inner_sweeps - steps) if corrector else 0
    return float(t_end) / float(inner_sweeps + corrections)
