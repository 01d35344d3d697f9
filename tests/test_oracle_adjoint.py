"""Oracle pins: the body force and the discrete adjoint of the march (implicit differentiation of
each accepted fixed point), against central differences of the oracle's own forward march."""
import numpy as np
import pytest

from oracle import adjoint as AD
from oracle import kinetics as K
from oracle import march as M
from oracle import sweep as SW
from oracle.lattice import D2Q9, D3Q19
from workloads.fields import random_moments, random_phase, random_populations


@pytest.mark.parametrize("lat", [D2Q9, D3Q19], ids=["d2q9", "d3q19"])
def test_sweep_jacobian_matches_central_differences(lat):
    n = 6
    shape = (n,) * lat.d
    m0 = random_moments(lat.d, shape, seed=1, scale=0.05)
    f = K.feq(lat, m0[0], m0[1:]) + random_populations(lat.Q, shape, seed=2, scale=1e-3)
    h = random_moments(lat.d, shape, seed=3, scale=1e-3)
    a = 0.07
    m = K.reconstruct(K.moments(lat, f), a, h)
    Jf, Jh = AD.sweep_jacobians(lat, m, h, a)
    v = random_populations(lat.Q, shape, seed=4, scale=1.0)
    w = random_moments(lat.d, shape, seed=5, scale=1.0)
    d = 1e-6
    fd_f = (SW.sweep(lat, f + d * v, a, h) - SW.sweep(lat, f - d * v, a, h)) / (2 * d)
    fd_h = (SW.sweep(lat, f, a, h + d * w) - SW.sweep(lat, f, a, h - d * w)) / (2 * d)
    assert np.max(np.abs((Jf @ v.ravel()).reshape(f.shape) - fd_f)) < 1e-8 * np.max(np.abs(fd_f))
    assert np.max(np.abs((Jh @ w.ravel()).reshape(f.shape) - fd_h)) < 1e-8 * np.max(np.abs(fd_h))


def test_force_mean_momentum_law():
    # the mean mode of the BDF march integrates a uniform force exactly: <u>^n = <u>^0 + n dt F
    N, dt, S = 16, 10.0, 5
    p, u = random_phase(N, 2, 1.0, seed=2, kmax=4)
    F = (1e-6, -2e-6)
    st = M.init_state(D2Q9, p, u)
    recs = M.march(st, M.MarchParams(dt=dt, eps=1e-14, kmax=3000, force=F), S)
    assert all(r.converged for r in recs)
    mean_u = st.m_n[1:].mean(axis=(1, 2))
    assert np.allclose(mean_u, u.mean(axis=(1, 2)) + S * dt * np.array(F), rtol=1e-9, atol=1e-16)
    assert abs(st.m_n[0].mean()) < 1e-16  # mass (p_hat gauge) stays put


def _setup(N=12, S=3, dt=9.0):
    p0, u0 = random_phase(N, 2, 1.0, seed=3, kmax=3)
    pt, ut = random_phase(N, 2, 1.0, seed=2, kmax=3)
    U = 1.0 / 6.0 / N
    F_star = (0.5 * U / (S * dt), 0.25 * U / (S * dt))
    prm_t = M.MarchParams(dt=dt, eps=1e-15, kmax=5000, force=F_star)
    st_t = M.init_state(D2Q9, pt, ut)
    assert all(r.converged for r in M.march(st_t, prm_t, S))
    return p0, u0, st_t.m_n[1:].copy(), S, dt


def _loss(p0, u0, force, target, S, dt):
    st = M.init_state(D2Q9, p0, u0)
    recs = M.march(st, M.MarchParams(dt=dt, eps=1e-15, kmax=5000, force=force), S)
    assert all(r.converged for r in recs)
    return AD.misfit_loss(st.m_n[1:], target), st


def test_adjoint_gradients_match_central_differences():
    p0, u0, target, S, dt = _setup()
    force = (0.0, 0.0)
    L0, st = _loss(p0, u0, force, target, S, dt)
    dm = np.zeros_like(st.m_n)
    dm[1:] = st.m_n[1:] - target
    g_p, g_u, g_F = AD.gradients(D2Q9, p0, u0, M.MarchParams(dt=dt, eps=1e-15, kmax=5000, force=force), S, dm)
    rng = np.random.default_rng(7)
    # initial velocity along a random direction
    v = rng.standard_normal(u0.shape) * np.abs(u0).max()
    d = 1e-4
    fd = (_loss(p0, u0 + d * v, force, target, S, dt)[0] - _loss(p0, u0 - d * v, force, target, S, dt)[0]) / (2 * d)
    assert abs(np.sum(g_u * v) / fd - 1) < 1e-6
    # initial pressure (p_hat_0 itself is O(U^2): probe with O(U) perturbations so that the
    # difference quotient stands well above the forward tolerance)
    w = rng.standard_normal(p0.shape) * np.abs(u0).max()
    fd = (_loss(p0 + d * w, u0, force, target, S, dt)[0] - _loss(p0 - d * w, u0, force, target, S, dt)[0]) / (2 * d)
    assert abs(np.sum(g_p * w) / fd - 1) < 1e-6
    # body force, each component
    dF = 1e-9
    for al in range(2):
        e = np.zeros(2)
        e[al] = dF
        fd = (_loss(p0, u0, tuple(e), target, S, dt)[0] - _loss(p0, u0, tuple(-e), target, S, dt)[0]) / (2 * dF)
        assert abs(g_F[al] / fd - 1) < 1e-6


def test_adjoint_of_a_forced_march():
    # the gradient is also right away from F = 0 (the force enters every h^n)
    p0, u0, target, S, dt = _setup(N=8, S=2)
    force = (3e-6, -1e-6)
    L0, st = _loss(p0, u0, force, target, S, dt)
    dm = np.zeros_like(st.m_n)
    dm[1:] = st.m_n[1:] - target
    _, g_u, g_F = AD.gradients(D2Q9, p0, u0, M.MarchParams(dt=dt, eps=1e-15, kmax=5000, force=force), S, dm)
    dF = 1e-9
    e = np.array([dF, 0.0])
    fd = (_loss(p0, u0, tuple(np.array(force) + e), target, S, dt)[0]
          - _loss(p0, u0, tuple(np.array(force) - e), target, S, dt)[0]) / (2 * dF)
    assert abs(g_F[0] / fd - 1) < 1e-6
