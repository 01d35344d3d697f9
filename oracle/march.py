"""Dual-time BDF march: Algorithm 1 (MSC-LBM) and plain Picard, plus explicit LBM. FP64 oracle.

Test infrastructure.  Follows Sections 2.3 and 3.1 and Algorithm 1 in the
paper's order:

* physical step n -> n+1 uses BDF1 on the first step of the run, BDF2 after
  (Eq. bdf2);
* the trial populations start from the population-history extrapolation
  f^n, 2f^n - f^{n-1}, 3f^n - 3f^{n-1} + f^{n-2} (Section 3.1);
* inner iteration l = 1..K_max: f_T = T(f), r = f_T - f, R_l = RMS(r); accept
  when l >= n_min and R_l < eps (a NaN never passes); on acceptance
  f^{n+1} = f_T and m^{n+1} = R_{q,h}(f^{n+1}) with the unrotated histories,
  then the population and moment histories rotate; otherwise the next trial
  is f_T (Picard) or f_T + E delta m_sh (MSC, Eq. shadow-update);
* a step that exhausts K_max is recorded nonconvergent and the state stays at
  the last accepted step.

``replay`` forces the accepted inner count of each step (acceptance at
l == count regardless of R); it exists so that a second implementation can be
compared iteration for iteration without the acceptance test bifurcating on
rounding.

Pins (tests/test_oracle_march.py): Taylor-Green closed-form decay (Eq. tgv2d),
conservation of sum p_hat and sum u across steps, Picard and MSC reach the same
fixed point, the Picard tail contraction matches gamma_dt (Eq. slowrate), the
temporal self-convergence table (Table temporal-order), and the explicit LBM
against the same closed form.
"""
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from .kinetics import bdf_coefficients, feq, moments, reconstruct
from .lattice import Lattice
from .shadow import shadow_correction
from .sweep import explicit_step, residual, sweep


@dataclass
class MarchParams:
    dt: float                 # physical BDF step in lattice time units
    nu: float = 1.0 / 6.0     # viscosity used by the shadow solve (operating point: 1/6)
    eps: float = 1e-8         # acceptance tolerance on the raw population RMS residual
    kmax: int = 300           # maximum inner iterations per physical step
    nmin: int = 2             # minimum accepted inner count
    corrector: bool = True    # True: MSC-LBM; False: plain Picard dual-time stepping
    omega: Optional[tuple] = None  # None: operating point; (w+, w-): general TRT collision
    warm_order: int = 3       # accepted states used by the warm start: 3 is Section 3.1 (cubic);
                              # 1 (f^n) and 2 (2f^n - f^{n-1}) truncate it
    count_multiple: int = 1   # accept only at inner counts that are multiples of this (1: Algorithm 1;
                              # 2: sweeps in pairs, for reduced-precision storage)
    full_symbol: bool = False  # corrector: the full-symbol reference operator (Eq. full-symbol) instead of
                              # the shadow correction: f <- f + F^{-1}[(I - Z J)^{-1} F r]
    force: Optional[tuple] = None  # uniform body force F (d components); the paper has none.  Read as
                              # an addition to the momentum source, s_u = h_u - a u + F, which is the
                              # same as adding (0, F) to h in both the reconstruction and the source


@dataclass
class StepRecord:
    q: int
    iters: int
    residuals: List[float]
    converged: bool


@dataclass
class DualTimeState:
    lat: Lattice
    f_hist: list              # accepted populations, newest first: [f^n, f^{n-1}, f^{n-2}]
    m_n: np.ndarray
    m_nm1: np.ndarray
    steps_done: int = 0
    records: List[StepRecord] = field(default_factory=list)

    @property
    def f(self) -> np.ndarray:
        return self.f_hist[0]

    def fields(self):
        """(p_hat, u) of the last accepted state: the reconstructed m^n."""
        return self.m_n[0], self.m_n[1:]


def init_state(lat: Lattice, p_hat: np.ndarray, u: np.ndarray) -> DualTimeState:
    """f^0 = f_eq(p_hat_0, u_0), m^0 = P f^0, no pre-march relaxation (Section 4.1)."""
    f0 = feq(lat, np.asarray(p_hat, dtype=np.float64), np.asarray(u, dtype=np.float64))
    m0 = moments(lat, f0)
    return DualTimeState(lat, [f0], m0, m0.copy(), 0)


def warm_start(f_hist: list, order: int = 3) -> np.ndarray:
    """Population-history extrapolation used to start the inner solve (Section 3.1).

    Uses min(order, available) accepted states: f^n, then 2f^n - f^{n-1}, then
    3f^n - 3f^{n-1} + f^{n-2}.  The paper's rule is order 3; lower orders are offered for
    reduced-precision storage, where the cubic extrapolation amplifies rounding in slowly damped
    modes.  The warm start only sets the first iterate, never the accepted fixed point.
    """
    k = min(len(f_hist), order)
    if k == 1:
        return f_hist[0].copy()
    if k == 2:
        return 2.0 * f_hist[0] - f_hist[1]
    return 3.0 * f_hist[0] - 3.0 * f_hist[1] + f_hist[2]


def forced_history(lat: Lattice, h: np.ndarray, force) -> np.ndarray:
    """h + (0, F): the body force enters wherever the BDF history term does."""
    if force is None:
        return h
    h = h.copy()
    for al in range(lat.d):
        h[1 + al] += force[al]
    return h


def physical_step(st: DualTimeState, prm: MarchParams, replay_count: Optional[int] = None) -> StepRecord:
    """One physical step of Algorithm 1 (corrector on) or plain Picard (corrector off)."""
    lat = st.lat
    q = 1 if st.steps_done == 0 else 2
    a, h = bdf_coefficients(q, prm.dt, st.m_n, st.m_nm1)
    h = forced_history(lat, h, prm.force)
    f = warm_start(st.f_hist, prm.warm_order)
    res = []
    Minv = None
    if prm.full_symbol and prm.corrector:
        from .fullsymbol import correction_matrices, rest_jacobian
        Minv = correction_matrices(lat, rest_jacobian(lat, a, prm.omega or (1.0, 1.0)), f.shape[1:])
    for ell in range(1, prm.kmax + 1):
        f_T = sweep(lat, f, a, h, prm.omega)
        r, R = residual(f_T, f)
        res.append(R)
        if replay_count is not None:
            accept = ell == replay_count
        else:
            accept = ell >= prm.nmin and R < prm.eps and ell % prm.count_multiple == 0
        if accept:
            m_new = reconstruct(moments(lat, f_T), a, h)
            st.f_hist = [f_T] + st.f_hist[:2]
            st.m_nm1 = st.m_n
            st.m_n = m_new
            st.steps_done += 1
            rec = StepRecord(q, ell, res, True)
            st.records.append(rec)
            return rec
        if Minv is not None:
            from .fullsymbol import full_symbol_correction
            f = f + full_symbol_correction(lat, r, Minv)
        elif prm.corrector:
            _, df = shadow_correction(lat, r, a, prm.nu)
            f = f_T + df
        else:
            f = f_T
    rec = StepRecord(q, prm.kmax, res, False)
    st.records.append(rec)
    return rec


def march(st: DualTimeState, prm: MarchParams, n_steps: int, replay_counts=None) -> List[StepRecord]:
    """Run n_steps physical steps; stops at the first nonconvergent step."""
    out = []
    for i in range(n_steps):
        rc = None if replay_counts is None else int(replay_counts[i])
        rec = physical_step(st, prm, rc)
        out.append(rec)
        if not rec.converged:
            break
    return out


def explicit_march(lat: Lattice, f: np.ndarray, n_steps: int, omega=None) -> np.ndarray:
    """n_steps explicit LBM steps f <- S C(f) (same collision and streaming, no source)."""
    for _ in range(n_steps):
        f = explicit_step(lat, f, omega)
    return f


def rho_observed(residuals, m_rho: int) -> Optional[float]:
    """Tail geometric mean of residual ratios (Eq. rho-observed); None with < 3 residuals."""
    R = np.asarray(residuals, dtype=np.float64)
    lf = len(R)
    if lf < 3:
        return None
    m = min(m_rho, lf - 1)
    ratios = R[lf - m:] / R[lf - m - 1:lf - 1]
    return float(np.exp(np.mean(np.log(ratios))))
