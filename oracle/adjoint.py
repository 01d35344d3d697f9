"""Discrete adjoint of the periodic MSC-LBM march (D2Q9 / D3Q19, operating point), FP64.

Test infrastructure.  The accepted state of a physical step is the fixed point of the sweep,
f^{n+1} = T(f^{n+1}; h^n) (Eqs. fixed-point-problem, sweep), with h^n = h_q(m^n, m^{n-1}) + (0, F)
(Eq. bdf2 plus the body force) and m^{n+1} = R(f^{n+1}; h^n) (Eq. macro-reconstruct).  The warm
start only chooses the first iterate, so the converged march is the map
    (m^n, m^{n-1}, F) -> h^n -> f^{n+1}(h^n) -> m^{n+1},
and a loss of the final fields is differentiated by implicit differentiation of each fixed point:
    (I - dT/df)^T lambda = P^T mu / (1 + a/2),   mu = dL/dm^{n+1},
    dL/dh^n = (dT/dh)^T lambda + mu / (2 (1 + a/2)),
then back through h^n = c1 m^n - c2 m^{n-1} + (0, F) to the moment history and the force, and
through m^0 = P f_eq(p_hat_0, u_0) = (p_hat_0, u_0) (exact quadrature) to the initial fields.

At the operating point the collision depends on f only through m = R(f) (Eq.
collision-operating), so dT/df = S D_m P / (1 + a/2) and dT/dh = S (D_m / (2 (1 + a/2)) + G_s)
with D_m = dC/dm (s = h - a m carried along) and G_s = dC/ds at each site.  Here both per-site
Jacobians come from complex-step differentiation of this package's own collision (exact to
rounding for a polynomial), the sweep Jacobians are assembled as sparse matrices and every
transposed fixed-point system is solved directly (scipy sparse LU): no iteration, no
preconditioner.  Small lattices only.

Pins (tests/test_oracle_adjoint.py): the assembled dT/df against central differences of the
oracle sweep; the gradients with respect to u_0, p_hat_0 and F against central differences of the
oracle march's loss; the exact mean-momentum law <u>^n = <u>^0 + n dt F under a uniform force.
"""
from typing import List, Tuple

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .kinetics import collide_operating, moment_matrix
from .lattice import Lattice
from .march import MarchParams, forced_history, init_state, physical_step
from .kinetics import bdf_coefficients

_CSTEP = 1e-30


def collision_jacobians(lat: Lattice, m: np.ndarray, h: np.ndarray, a: float):
    """D_m[k, c] = dC_k/dm_c with s = h - a m, and G_s[k, c] = dC_k/ds_c, per site (complex step)."""
    F = lat.d + 1
    Dm = np.empty((lat.Q, F) + m.shape[1:])
    Gs = np.empty((lat.Q, F) + m.shape[1:])
    s = h - a * m
    for c in range(F):
        dm = np.zeros(m.shape, dtype=np.complex128)
        dm[c] = 1j * _CSTEP
        mc = m + dm
        Dm[:, c] = np.imag(collide_operating(lat, mc, h - a * mc)) / _CSTEP
        sc = s + dm
        Gs[:, c] = np.imag(collide_operating(lat, m + 0j, sc)) / _CSTEP
    return Dm, Gs


def _site_index(lat: Lattice, shape):
    n_sites = int(np.prod(shape))
    return np.arange(n_sites).reshape(shape)


def _streamed_index(lat: Lattice, shape, k: int):
    """Flat site index of x + c_k for every site x (periodic)."""
    idx = _site_index(lat, shape)
    d = lat.d
    axes = tuple(d - 1 - a for a in range(d))
    shifts = tuple(int(lat.c[k, a]) for a in range(d))
    # out(x + c_k) = in(x): the destination of site x is roll of the index array by -c_k
    return np.roll(idx, shift=tuple(-s for s in shifts), axis=axes)


def sweep_jacobians(lat: Lattice, m: np.ndarray, h: np.ndarray, a: float):
    """Sparse dT/df ((Q n) x (Q n)) and dT/dh ((Q n) x ((d+1) n)) at the state with moments m."""
    shape = m.shape[1:]
    n = int(np.prod(shape))
    F = lat.d + 1
    Dm, Gs = collision_jacobians(lat, m, h, a)
    P = moment_matrix(lat)
    inv = 1.0 / (1.0 + a / 2.0)
    src = _site_index(lat, shape).ravel()
    rows_f, cols_f, vals_f = [], [], []
    rows_h, cols_h, vals_h = [], [], []
    for k in range(lat.Q):
        dst = _streamed_index(lat, shape, k).ravel()  # T_k at x + c_k comes from C_k at x
        # d C_k(x) / d f_j(x) = sum_c D_m[k, c](x) P[c, j] / (1 + a/2)
        for j in range(lat.Q):
            v = sum(Dm[k, c].ravel() * P[c, j] for c in range(F)) * inv
            rows_f.append(k * n + dst)
            cols_f.append(j * n + src)
            vals_f.append(v)
        for c in range(F):
            v = Dm[k, c].ravel() * (0.5 * inv) + Gs[k, c].ravel()
            rows_h.append(k * n + dst)
            cols_h.append(c * n + src)
            vals_h.append(v)
    Jf = sp.csr_matrix((np.concatenate(vals_f), (np.concatenate(rows_f), np.concatenate(cols_f))),
                       shape=(lat.Q * n, lat.Q * n))
    Jh = sp.csr_matrix((np.concatenate(vals_h), (np.concatenate(rows_h), np.concatenate(cols_h))),
                       shape=(lat.Q * n, F * n))
    return Jf, Jh


def adjoint_step(lat: Lattice, m_new: np.ndarray, h: np.ndarray, a: float, mu: np.ndarray) -> np.ndarray:
    """dL/dh^n of one step given mu = dL/dm^{n+1} (exact sparse solves)."""
    shape = m_new.shape[1:]
    n = int(np.prod(shape))
    Jf, Jh = sweep_jacobians(lat, m_new, h, a)
    P = moment_matrix(lat)
    inv = 1.0 / (1.0 + a / 2.0)
    mu_f = mu.reshape(lat.d + 1, n)
    b = (P.T @ mu_f).ravel() * inv                       # P^T mu / (1 + a/2), population layout
    A = (sp.identity(lat.Q * n, format="csr") - Jf).T.tocsc()
    lam = spla.spsolve(A, b)
    nu_h = Jh.T @ lam + mu.ravel() * (0.5 * inv)
    return nu_h.reshape(mu.shape)


def forward_moments(lat: Lattice, p0, u0, prm: MarchParams, steps: int):
    """The march to convergence, recording m^0 .. m^S and each step's BDF order."""
    st = init_state(lat, p0, u0)
    ms = [st.m_n.copy()]
    qs = []
    for _ in range(steps):
        q = 1 if st.steps_done == 0 else 2
        rec = physical_step(st, prm)
        if not rec.converged:
            raise RuntimeError("forward step did not converge")
        qs.append(q)
        ms.append(st.m_n.copy())
    return st, ms, qs


def gradients(lat: Lattice, p0, u0, prm: MarchParams, steps: int, dL_dm_final: np.ndarray,
              ms: List[np.ndarray] = None, qs: List[int] = None) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """(dL/dp_hat_0, dL/du_0, dL/dF) of a loss whose gradient with respect to m^S is dL_dm_final."""
    if ms is None:
        _, ms, qs = forward_moments(lat, p0, u0, prm, steps)
    F = lat.d + 1
    abar = [np.zeros_like(ms[0]) for _ in range(steps + 1)]
    abar[steps] = np.array(dL_dm_final, dtype=np.float64).copy()
    dF = np.zeros(lat.d)
    for n in range(steps - 1, -1, -1):
        q = qs[n]
        m_prev = ms[n - 1] if n >= 1 else ms[0]
        a, h = bdf_coefficients(q, prm.dt, ms[n], m_prev)
        h = forced_history(lat, h, prm.force)
        nu_h = adjoint_step(lat, ms[n + 1], h, a, abar[n + 1])
        c1 = 1.0 / prm.dt if q == 1 else 4.0 / (2.0 * prm.dt)
        c2 = 0.0 if q == 1 else 1.0 / (2.0 * prm.dt)
        abar[n] += c1 * nu_h
        if n >= 1:
            abar[n - 1] -= c2 * nu_h
        dF += np.array([nu_h[1 + al].sum() for al in range(lat.d)])
    return abar[0][0], abar[0][1:F], dF


def misfit_loss(u: np.ndarray, u_target: np.ndarray) -> float:
    """L = 1/2 sum_x |u - u_target|^2 (the L2 misfit of the final velocity)."""
    return 0.5 * float(np.sum((u - u_target) ** 2))
