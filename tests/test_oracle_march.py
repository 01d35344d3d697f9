"""Oracle pins: Algorithm 1, Picard dual-time stepping and the explicit LBM (Sections 3.1, 4)."""
import json
import os

import numpy as np
import pytest

from oracle import kinetics as K
from oracle import march as M
from oracle.lattice import D2Q9, D3Q19
from oracle.linear import gamma
from workloads.fields import random_phase, tgv2d, tgv3d
from workloads.metrics import rms_vector, velocity_error

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "temporal_order.json")


def test_tgv_decay_closed_form_msc_and_explicit():
    # Eq. tgv2d: u decays as exp(-2 nu k0^2 t).  N = 64, Re = 1, T_end = nint(0.05 N^2 / nu) = 1229,
    # S = 38 physical steps.  Both schemes must follow the closed form to lattice accuracy.
    N, Re, T_end, S = 64, 1.0, 1229, 38
    p, u = tgv2d(N, Re)
    _, u_ref = tgv2d(N, Re, t=T_end)
    st = M.init_state(D2Q9, p, u)
    recs = M.march(st, M.MarchParams(dt=T_end / S, eps=1e-10), S)
    assert all(r.converged for r in recs)
    e_msc = velocity_error(st.fields()[1], u_ref) / rms_vector(u_ref)
    f = M.explicit_march(D2Q9, M.init_state(D2Q9, p, u).f, T_end)
    e_ex = velocity_error(K.moments(D2Q9, f)[1:], u_ref) / rms_vector(u_ref)
    assert e_ex < 5e-3 and e_msc < 2e-2
    # the decay factor itself: a wrong viscosity (e.g. 1/3) would give exp(-7.9) instead of exp(-3.95)
    amp = np.sum(st.fields()[1] * u) / np.sum(u * u)
    assert abs(amp / np.exp(-2 * (1 / 6) * (2 * np.pi / N) ** 2 * T_end) - 1) < 2e-2


def test_conservation_across_steps():
    # with no force the domain sums of p_hat and u stay constant to O(eps) (BDF of a constant)
    N = 32
    p, u = random_phase(N, 2, 5.0, seed=5, kmax=4)
    st = M.init_state(D2Q9, p, u)
    s0 = st.m_n.reshape(3, -1).sum(axis=1)
    M.march(st, M.MarchParams(dt=16.0, eps=1e-12), 6)
    s1 = st.m_n.reshape(3, -1).sum(axis=1)
    assert np.max(np.abs(s1 - s0)) < 1e-12 * N * N


def test_picard_and_msc_share_the_fixed_point():
    # Section 3.1: both corrections vanish at r = 0, so the converged states agree within the
    # tolerance amplified by the slow rate (paper: 3.57e-11 abs at N = 128, Re = 100, dt = 38.9)
    N, dt = 32, 38.9
    p, u = random_phase(N, 2, 5.0, seed=6, kmax=4)  # Ma = 0.05 at N = 32
    out = {}
    for corr in (True, False):
        st = M.init_state(D2Q9, p, u)
        recs = M.march(st, M.MarchParams(dt=dt, eps=1e-13, kmax=5000, corrector=corr), 3)
        assert all(r.converged for r in recs)
        out[corr] = (st.fields()[1], sum(r.iters for r in recs))
    diff = velocity_error(out[True][0], out[False][0])
    assert diff < 1e-13 / (1 - gamma(3 / (2 * dt))) * 10
    assert out[True][1] < out[False][1] / 5  # the corrector cuts the inner work


def test_picard_tail_factor_matches_slow_rate():
    # Section 4.3: N = 128, dt = 38.9: gamma_dt = 0.9622; measured Picard tails 0.958-0.960
    N, dt = 128, 38.9
    p, u = tgv2d(N, 1.0)
    st = M.init_state(D2Q9, p, u)
    M.physical_step(st, M.MarchParams(dt=dt, eps=1e-12))  # BDF1 starter; the tail is taken on BDF2
    rec = M.physical_step(st, M.MarchParams(dt=dt, eps=1e-13, kmax=900, corrector=False))
    assert rec.q == 2 and rec.converged
    rho = M.rho_observed(rec.residuals, 10)
    assert 0.955 < rho <= gamma(3 / (2 * dt)) + 1e-4


def test_nonconvergent_step_leaves_state_at_last_accepted():
    p, u = tgv2d(16, 1.0)
    st = M.init_state(D2Q9, p, u)
    f0 = st.f.copy()
    recs = M.march(st, M.MarchParams(dt=8.0, eps=1e-30, kmax=3), 4)
    assert len(recs) == 1 and not recs[0].converged and recs[0].iters == 3
    assert st.steps_done == 0 and np.array_equal(st.f, f0)


def test_nan_never_passes_acceptance():
    p, u = tgv2d(16, 1.0)
    st = M.init_state(D2Q9, p, u)
    st.f_hist[0] = st.f_hist[0].copy()
    st.f_hist[0][3, 2, 2] = np.nan
    recs = M.march(st, M.MarchParams(dt=8.0, eps=1.0, kmax=4), 1)
    assert not recs[0].converged and st.steps_done == 0


def test_replay_reproduces_free_run():
    p, u = tgv2d(32, 1.0)
    st = M.init_state(D2Q9, p, u)
    recs = M.march(st, M.MarchParams(dt=20.0, eps=1e-9), 5)
    st2 = M.init_state(D2Q9, p, u)
    M.march(st2, M.MarchParams(dt=20.0, eps=1.0), 5, replay_counts=[r.iters for r in recs])
    assert np.array_equal(st.f, st2.f) and np.array_equal(st.m_n, st2.m_n)


def test_history_rotation_and_bdf_order():
    p, u = tgv2d(16, 1.0)
    st = M.init_state(D2Q9, p, u)
    m0 = st.m_n.copy()
    r1 = M.physical_step(st, M.MarchParams(dt=4.0, eps=1e-11))
    assert r1.q == 1 and np.array_equal(st.m_nm1, m0) and len(st.f_hist) == 2
    r2 = M.physical_step(st, M.MarchParams(dt=4.0, eps=1e-11))
    r3 = M.physical_step(st, M.MarchParams(dt=4.0, eps=1e-11))
    assert r2.q == 2 and r3.q == 2 and len(st.f_hist) == 3


def _self_convergence(lat, N, T_end, dts, nmin, init):
    p, u = init(N, 1.0)
    us, finals = [], []
    for dt in dts:
        S = int(round(T_end / dt))
        st = M.init_state(lat, p, u)
        recs = M.march(st, M.MarchParams(dt=T_end / S, eps=1e-12, kmax=20000, nmin=nmin), S)
        assert all(r.converged for r in recs)
        us.append(st.fields()[1].copy())
        finals.append(recs[-1].residuals[-1])
    d = lat.d
    # reading: the printed D_i averages over the d velocity components as well as the sites
    D = [velocity_error(us[i], us[i + 1]) / np.sqrt(d) for i in range(len(us) - 1)]
    return D, finals


def test_temporal_order_table_2d():
    g = json.load(open(GOLDEN))["d2"]
    D, _ = _self_convergence(D2Q9, g["N"], g["T_end"], g["dt"], 2, tgv2d)
    assert abs(D[0] / g["D"][0] - 1) < 2e-4
    assert abs(D[1] / g["D"][1] - 1) < 2e-4
    assert abs(D[2] / g["D"][2] - 1) < 2e-3   # the dt = 25 run ends on a borderline inner count
    p = [np.log2(D[i] / D[i + 1]) for i in range(2)]
    assert np.allclose(p, g["p"], atol=2e-3)


@pytest.mark.slow
def test_temporal_order_table_3d():
    g = json.load(open(GOLDEN))["d3"]
    D, finals = _self_convergence(D3Q19, g["N"], g["T_end"], g["dt"], 1, tgv3d)
    assert np.allclose(D, g["D"], rtol=1e-4, atol=0)
    p = [np.log2(D[i] / D[i + 1]) for i in range(2)]
    assert np.allclose(p, g["p"], atol=1e-3)
    # the final raw residuals span the printed range exactly (to the printed digits)
    lo, hi = g["final_residual_range"]
    assert abs(min(finals) / lo - 1) < 2e-3 and abs(max(finals) / hi - 1) < 2e-3


def test_warm_start_orders():
    f0, f1, f2 = (np.full((2, 2), v) for v in (3.0, 2.0, 0.5))
    assert np.all(M.warm_start([f0, f1, f2], 3) == 3 * 3.0 - 3 * 2.0 + 0.5)
    assert np.all(M.warm_start([f0, f1, f2], 2) == 2 * 3.0 - 2.0)
    assert np.all(M.warm_start([f0, f1, f2], 1) == 3.0)
    assert np.all(M.warm_start([f0], 3) == 3.0) and np.all(M.warm_start([f0, f1], 3) == 4.0)
    # the cubic rule is exact for quadratic-in-time data, the linear one for linear data
    t = np.array([3.0, 2.0, 1.0])
    quad = [np.full(1, tt ** 2) for tt in t]
    assert np.allclose(M.warm_start(quad, 3), 16.0)
    lin = [np.full(1, 2 * tt + 1) for tt in t]
    assert np.allclose(M.warm_start(lin, 2), 9.0)


def _staggered_amplitudes(warm_order, count, steps=8):
    # u_x perturbed by 1e-9 (-1)^x: the k = (pi, 0) staggered mode, sweep eigenvalue -1 and outside
    # the shadow mask; the inner count is forced (replay) so only the warm start and its parity act
    N = 32
    p, u = random_phase(N, 2, 1.0, seed=3, kmax=4)
    stag = (-1.0) ** np.arange(N)[None, :] * np.ones((N, 1))
    st = M.init_state(D2Q9, p, u + 1e-9 * np.stack([stag, 0 * stag]))
    prm = M.MarchParams(dt=40.0, eps=1.0, warm_order=warm_order)
    amps = []
    for _ in range(steps):
        M.physical_step(st, prm, replay_count=count)
        amps.append(abs(np.fft.fft2(st.m_n[1])[0, N // 2]) / N ** 2)
    return np.array(amps)


def test_staggered_mode_under_warm_start_and_count_parity():
    # per step the staggered mode is multiplied by c = (-gamma)^l after the warm start; with the
    # linear extrapolation e' = c (2e - e_prev) an odd count (c ~ -1) grows it by ~1 + sqrt(2),
    # the cubic one by more, while an even count (c ~ +1) or no extrapolation keeps it bounded
    lin_odd = _staggered_amplitudes(2, 3)
    assert np.all(lin_odd[3:] / lin_odd[2:-1] > 2.0)
    cub_odd = _staggered_amplitudes(3, 3)
    assert cub_odd[-1] / cub_odd[-2] > 3.0
    for wo, cnt in ((2, 2), (2, 4), (1, 3)):
        a = _staggered_amplitudes(wo, cnt)
        assert a.max() < 1.1e-9, (wo, cnt)


def test_count_multiple_accepts_even_counts_at_the_same_fixed_point():
    N = 32
    p, u = random_phase(N, 2, 1.0, seed=8, kmax=4)
    out = {}
    for cm in (1, 2):
        st = M.init_state(D2Q9, p, u)
        recs = M.march(st, M.MarchParams(dt=30.0, eps=1e-11, warm_order=2, count_multiple=cm), 6)
        assert all(r.converged for r in recs)
        out[cm] = (st.fields()[1].copy(), [r.iters for r in recs])
    assert all(k % 2 == 0 for k in out[2][1])
    assert any(k % 2 == 1 for k in out[1][1])  # the case exercises the rule
    # both accept at R < eps: the states agree to the tolerance amplified by the slow rate
    assert velocity_error(out[1][0], out[2][0]) < 1e-11 / (1 - gamma(3 / 60.0)) * 10
