"""Oracle pins: the full-symbol reference operator (Eq. full-symbol), TRT rates (Eq. trt), ghost
survival (Eq. eta) and the off-design collision."""
import numpy as np
import pytest

from oracle import fullsymbol as FS
from oracle import kinetics as K
from oracle import march as M
from oracle.lattice import D2Q9
from oracle.linear import gamma
from workloads.fields import tgv2d


def test_trt_rates_round_trip_and_operating_point():
    assert FS.trt_rates(1 / 6, 0.25) == pytest.approx((1.0, 1.0), abs=1e-15)
    for nu, lam in ((0.1, 0.25), (1 / 6, 0.05), (0.3, 3 / 16)):
        wp, wm = FS.trt_rates(nu, lam)
        tp, tm = 1 / wp, 1 / wm
        assert (tp - 0.5) / 3 == pytest.approx(nu, rel=1e-14)
        assert (tp - 0.5) * (tm - 0.5) == pytest.approx(lam, rel=1e-14)


def test_rest_jacobian_at_the_operating_point_is_gamma_E_P():
    # Eq. symbol: the local response at omega+- = 1 is gamma E P (forward difference, step 1e-7)
    a = 3 / (2 * 20.0)
    J = FS.rest_jacobian(D2Q9, a, (1.0, 1.0))
    ref = gamma(a) * K.lift_matrix(D2Q9) @ K.moment_matrix(D2Q9)
    assert np.max(np.abs(J - ref)) < 2e-7


@pytest.mark.parametrize("nu,lam", [(0.1, 0.25), (1 / 6, 0.05), (0.25, 0.4)])
def test_ghosts_relax_at_the_trt_rates_and_eta(nu, lam):
    wp, wm = FS.trt_rates(nu, lam)
    a = 0.05
    J = FS.rest_jacobian(D2Q9, a, (wp, wm))
    P = K.moment_matrix(D2Q9)
    # a basis of ghost vectors (P g = 0), split into even and odd parts under c -> -c
    _, _, vt = np.linalg.svd(P)
    G = vt[P.shape[0]:].T
    for g in G.T:
        ge = 0.5 * (g + g[D2Q9.opp])
        go = 0.5 * (g - g[D2Q9.opp])
        for v, lam_expected in ((ge, 1 - wp), (go, 1 - wm)):
            if np.linalg.norm(v) < 1e-12 or np.linalg.norm(P @ v) > 1e-12:
                continue
            assert np.allclose(J @ v, lam_expected * v, atol=3e-7)
    assert abs(1 - wp) == pytest.approx(FS.eta(nu), rel=1e-12)


def test_full_symbol_iteration_is_a_newton_step_in_the_linear_regime():
    # a 1e-9 perturbation of rest at an off-design point: one corrected iteration removes the
    # residual down to the forward-difference error of J (the map is linear to 1e-18 there)
    N = 16
    wp, wm = FS.trt_rates(0.08, 0.25)
    p, u = tgv2d(N, 1.0)
    amp = 1e-9 / np.abs(u).max()
    f = K.feq(D2Q9, 1.0 + amp * p, amp * u)
    st = M.init_state(D2Q9, amp * p, amp * u)
    st.f_hist = [f]
    st.m_n = K.moments(D2Q9, f)
    st.m_nm1 = st.m_n.copy()
    rec = M.physical_step(st, M.MarchParams(dt=20.0, eps=0.0, kmax=3, nmin=1, omega=(wp, wm), nu=0.08,
                                            full_symbol=True))
    R = rec.residuals
    assert R[1] / R[0] < 1e-5 and R[2] / R[0] < 1e-5


def test_full_symbol_converges_where_the_shadow_correction_fails():
    # off-design viscosity nu = 0.08 at Lambda = 1/4 (Section 4.6: the shadow correction diverges
    # by nu ~ 0.09, the full symbol keeps contracting)
    N, dt = 32, 20.0
    nu = 0.08
    wp, wm = FS.trt_rates(nu, 0.25)
    p, u = tgv2d(N, 1.0)
    st = M.init_state(D2Q9, p, u)
    base = dict(dt=dt, eps=1e-12, kmax=60, nmin=2, omega=(wp, wm), nu=nu)
    M.physical_step(st, M.MarchParams(**base, full_symbol=True))  # BDF1 starter
    st_sh = M.DualTimeState(D2Q9, list(st.f_hist), st.m_n.copy(), st.m_nm1.copy(), st.steps_done)
    full = M.physical_step(st, M.MarchParams(**base, full_symbol=True))
    shadow = M.physical_step(st_sh, M.MarchParams(**base))
    assert full.converged and full.iters < 20
    assert M.rho_observed(full.residuals, 10) < 0.2
    assert not shadow.converged or M.rho_observed(shadow.residuals, 10) > 0.9


@pytest.mark.parametrize("nu,lam", [(1 / 6, 0.25), (0.08, 0.25), (0.25, 0.05), (0.12, 2.0)])
def test_exact_rest_jacobian(nu, lam):
    # the complex-step derivative agrees with the paper's forward difference to the difference error
    # and, at the operating point, with gamma E P (Eq. symbol) to rounding
    wp, wm = FS.trt_rates(nu, lam)
    a = 3 / (2 * 20.0)
    Je = FS.rest_jacobian_exact(D2Q9, a, (wp, wm))
    Jf = FS.rest_jacobian(D2Q9, a, (wp, wm))
    assert np.max(np.abs(Je - Jf)) < 3e-7
    if nu == 1 / 6 and lam == 0.25:
        ref = gamma(a) * K.lift_matrix(D2Q9) @ K.moment_matrix(D2Q9)
        assert np.max(np.abs(Je - ref)) < 1e-15
    # conserved structure: the ghost space relaxes at 1 - omega+- exactly
    P = K.moment_matrix(D2Q9)
    _, _, vt = np.linalg.svd(P)
    for g in vt[P.shape[0]:]:
        for v, lam_e in ((0.5 * (g + g[D2Q9.opp]), 1 - wp), (0.5 * (g - g[D2Q9.opp]), 1 - wm)):
            if np.linalg.norm(v) > 1e-12 and np.linalg.norm(P @ v) < 1e-12:
                assert np.allclose(Je @ v, lam_e * v, atol=1e-14)
