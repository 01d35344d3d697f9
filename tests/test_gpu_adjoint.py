"""GPU discrete adjoint (msc_adjoint_step, checkpointed reverse pass, torch.autograd.Function)
against the FP64 oracle adjoint and against central differences of the GPU march."""
import numpy as np
import pytest
import torch

from oracle import adjoint as AD
from oracle import kinetics as OK
from oracle import march as OM
from oracle.lattice import D2Q9
from workloads.fields import random_phase
from tests.gpu_helpers import dev, host, rel_l2

pytestmark = pytest.mark.gpu
NU = 1.0 / 6.0


def _lat(n, precision="fp64"):
    from paper_2609_39474_b300.lattice import MscLattice
    return MscLattice(2, n, precision)


@pytest.mark.parametrize("q", [1, 2])
def test_adjoint_step_matches_oracle(q):
    # one step's transposed solve and its passage to m^n, m^{n-1} and F, on the oracle's own
    # forward moments (FP64)
    N, dt = 16, 9.0
    F = (2e-6, -1e-6)
    p0, u0 = random_phase(N, 2, 1.0, seed=3, kmax=3)
    st, ms, qs = AD.forward_moments(D2Q9, p0, u0, OM.MarchParams(dt=dt, eps=1e-15, kmax=5000, force=F), 3)
    n = 0 if q == 1 else 2
    # a smooth seed, like a misfit of smooth fields (a rough one excites the staggered modes outside
    # the mask, which contract only at gamma per iteration in the transposed solve as in the forward)
    mp, mv = random_phase(N, 2, 50.0, seed=9, kmax=3)
    mu = np.concatenate([mp[None], mv]) / np.abs(mv).max()
    a, h = OK.bdf_coefficients(q, dt, ms[n], ms[n - 1] if n else ms[0])
    h = OM.forced_history(D2Q9, h, F)
    nu = AD.adjoint_step(D2Q9, ms[n + 1], h, a, mu)
    c1 = 1 / dt if q == 1 else 2 / dt
    c2 = 0.0 if q == 1 else 1 / (2 * dt)
    L = _lat(N)
    L.set_params(dt=dt, eps=1e-10, force=F)
    ab_cur = torch.zeros((3, N, N), dtype=torch.float64, device="cuda")
    ab_prev = torch.zeros_like(ab_cur)
    dF = torch.zeros(3, dtype=torch.float64, device="cuda")
    r = L.adjoint_step(q, dev(ms[n + 1]), dev(ms[n]), dev(ms[n - 1]) if q == 2 else None, dev(mu), ab_cur,
                       ab_prev if q == 2 else None, dF, eps=1e-13, kmax=500)
    assert r["residual"] < 1e-13 and r["iters"] < 200  # ~119 with the exact transpose on the CPU
    assert rel_l2(host(ab_cur), c1 * nu) < 1e-11
    if q == 2:
        assert rel_l2(host(ab_prev), -c2 * nu) < 1e-11
    assert np.allclose(host(dF)[:2], [nu[1].sum(), nu[2].sum()], rtol=1e-10, atol=1e-14)


def _problem(N, S, dt, seed_target=2, seed_init=3):
    p0, u0 = random_phase(N, 2, 1.0, seed=seed_init, kmax=min(8, N // 4))
    pt, ut = random_phase(N, 2, 1.0, seed=seed_target, kmax=min(8, N // 4))
    U = NU / N
    F_star = (0.5 * U / (S * dt), 0.25 * U / (S * dt))
    return p0, u0, pt, ut, F_star


def test_full_gradient_matches_oracle_fp64():
    from paper_2609_39474_b300.adjoint import MarchRunner
    N, S, dt = 16, 5, 9.0
    p0, u0, pt, ut, F_star = _problem(N, S, dt)
    st_t, _, _ = AD.forward_moments(D2Q9, pt, ut, OM.MarchParams(dt=dt, eps=1e-15, kmax=5000, force=F_star), S)
    target = st_t.m_n[1:]
    prm = OM.MarchParams(dt=dt, eps=1e-15, kmax=5000)
    st, ms, qs = AD.forward_moments(D2Q9, p0, u0, prm, S)
    dm = np.zeros_like(st.m_n)
    dm[1:] = st.m_n[1:] - target
    g_p, g_u, g_F = AD.gradients(D2Q9, p0, u0, prm, S, dm, ms, qs)
    R = MarchRunner(_lat(N), dt=dt, steps=S, eps=1e-14, checkpoint_every=2, eps_adjoint=1e-13, kmax=5000)
    uS = R.forward(dev(p0), dev(u0), (0.0, 0.0))
    assert rel_l2(host(uS), st.m_n[1:]) < 1e-10
    gp, gu, gF = R.backward(uS - dev(target))
    assert rel_l2(host(gu), g_u) < 1e-8
    assert rel_l2(host(gp), g_p) < 1e-8
    assert rel_l2(host(gF), g_F) < 1e-8


def _runner(N, S, dt, precision, K, eps=1e-7):
    from paper_2609_39474_b300.adjoint import MarchRunner
    # FP32 working arrays put the reduced adjoint residual's rounding floor near 1e-7
    return MarchRunner(_lat(N, precision), dt=dt, steps=S, eps=eps, checkpoint_every=K,
                       eps_adjoint=1e-5 if precision == "fp32" else 1e-10)


def test_checkpoint_interval_gives_identical_gradients():
    N, S, dt = 64, 12, 24.0
    p0, u0, pt, ut, F_star = _problem(N, S, dt)
    out = []
    for K in (1, 4, 12):
        R = _runner(N, S, dt, "fp32", K, eps=1e-6 * NU / N)
        uS = R.forward(dev(p0), dev(u0))
        out.append((uS, R.backward(uS - dev(ut))))
    for uS, g in out[1:]:
        assert torch.equal(uS, out[0][0])
        for a, b in zip(g, out[0][1]):
            assert torch.equal(a, b)


def test_fp32_gradients_against_central_differences():
    # config-5 style at N = 64: L = 1/2 |u^S - u*|^2, u* from a seeded target run under a force
    N, S, dt = 64, 16, 30.0
    p0, u0, pt, ut, F_star = _problem(N, S, dt)
    eps = 1e-6 * NU / N
    Rt = _runner(N, S, dt, "fp32", 8, eps)
    target = Rt.forward(dev(pt), dev(ut), F_star)
    R = _runner(N, S, dt, "fp32", 8, eps)

    def loss(u0_, F_):
        uS = R.forward(dev(p0), u0_, F_)
        return 0.5 * float(((uS - target) ** 2).sum())

    uS = R.forward(dev(p0), dev(u0), (0.0, 0.0))
    _, gu, gF = R.backward(uS - target)
    rng = np.random.default_rng(5)
    v = dev(rng.standard_normal(u0.shape) * np.abs(u0).max())
    d = 1e-2
    fd = (loss(dev(u0) + d * v, (0.0, 0.0)) - loss(dev(u0) - d * v, (0.0, 0.0))) / (2 * d)
    assert abs(float((gu * v).sum()) / fd - 1) < 2e-3
    dF = 0.2 * abs(F_star[0])
    for al in range(2):
        e = [0.0, 0.0]
        e[al] = dF
        fd = (loss(dev(u0), tuple(e)) - loss(dev(u0), tuple(-x for x in e))) / (2 * dF)
        assert abs(float(gF[al]) / fd - 1) < 2e-3


def test_autograd_function():
    from paper_2609_39474_b300.adjoint import MscMarch
    N, S, dt = 32, 6, 16.0
    p0, u0, pt, ut, _ = _problem(N, S, dt)
    R = _runner(N, S, dt, "fp64", 4, eps=1e-12)
    u0_t = dev(u0).requires_grad_(True)
    F_t = torch.zeros(2, dtype=torch.float64, requires_grad=True)
    uS = MscMarch.apply(u0_t, F_t, R, dev(p0))
    loss = 0.5 * ((uS - dev(ut)) ** 2).sum()
    loss.backward()
    _, gu, gF = R.backward(uS.detach() - dev(ut))
    assert torch.equal(u0_t.grad, gu)
    assert torch.allclose(F_t.grad, gF.cpu())
    assert F_t.grad.abs().sum() > 0 and u0_t.grad.abs().sum() > 0


def _step_inputs(N=16, dt=9.0):
    p0, u0 = random_phase(N, 2, 1.0, seed=3, kmax=3)
    st, ms, qs = AD.forward_moments(D2Q9, p0, u0, OM.MarchParams(dt=dt, eps=1e-15, kmax=5000), 3)
    mp, mv = random_phase(N, 2, 50.0, seed=9, kmax=3)
    mu = np.concatenate([mp[None], mv]) / np.abs(mv).max()
    return [dev(m) for m in ms], dev(mu)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_adjoint_steps_equal_single_steps_across_chunks(precision):
    # 70 steps (two runs of the 64-step chunk) through one call are bit-identical to 70 single calls
    # and to the host-driven run of the same kernels
    N, dt = 16, 9.0
    ms, mu = _step_inputs(N, dt)
    outs = []
    for mode in ("single", "graph", "stepwise"):
        L = _lat(N, precision)
        L.set_params(dt=dt, eps=1e-10)
        ab_cur = torch.zeros_like(mu)
        ab_prev = torch.zeros_like(mu)
        dF = torch.zeros(3, dtype=torch.float64, device="cuda")
        steps = [(2 if i % 3 else 1, ms[3], ms[2], ms[1], mu, ab_cur, ab_prev) for i in range(70)]
        eps = 1e-12 if precision == "fp64" else 1e-5
        if mode == "single":
            rs = [L.adjoint_step(q, a, b, c if q == 2 else None, d, e, f if q == 2 else None, dF, eps=eps, kmax=500)
                  for q, a, b, c, d, e, f in steps]
        else:
            rs = L.adjoint_steps(steps, dF, eps=eps, kmax=500, stepwise=mode == "stepwise")
        outs.append((ab_cur, ab_prev, dF, [r["iters"] for r in rs]))
    for o in outs[1:]:
        for x, y in zip(outs[0][:3], o[:3]):
            assert torch.equal(x, y)
        assert outs[0][3] == o[3]
    assert min(outs[0][3]) > 0


def test_adjoint_steps_stop_after_a_failed_step():
    # kmax = 0 cannot reach eps: the first step reports MSC_ERR_NONCONVERGED, the later ones are not
    # run (MSC_ERR_STATE) and every accumulator stays untouched
    from paper_2609_39474_b300 import _lib
    N, dt = 16, 9.0
    ms, mu = _step_inputs(N, dt)
    L = _lat(N)
    L.set_params(dt=dt, eps=1e-10)
    ab_cur = torch.zeros_like(mu)
    ab_prev = torch.zeros_like(mu)
    dF = torch.zeros(3, dtype=torch.float64, device="cuda")
    arr = (_lib.AdjointIO * 3)()
    for i in range(3):
        arr[i] = _lib.AdjointIO(2, ms[3].data_ptr(), ms[2].data_ptr(), ms[1].data_ptr(), mu.data_ptr(),
                                ab_cur.data_ptr(), ab_prev.data_ptr())
    out = (_lib.AdjointStats * 3)()
    rc = _lib.lib.msc_adjoint_steps(L._ctx, 3, arr, dF.data_ptr(), 1e-12, 0, out)
    assert rc == 2  # MSC_ERR_NONCONVERGED
    assert [s.status for s in out] == [2, 6, 6] and [s.iters for s in out] == [0, 0, 0]
    assert out[0].residual > 1e-12
    assert not ab_cur.any() and not ab_prev.any() and not dF.any()
    # the context stays usable: the same steps then converge
    rs = L.adjoint_steps([(2, ms[3], ms[2], ms[1], mu, ab_cur, ab_prev)], dF, eps=1e-12, kmax=500)
    assert rs[0]["status"] == 0 and ab_cur.abs().sum() > 0


def test_warm_start_reaches_the_same_fixed_point():
    # a repeated step started from its predecessor's solution (warm) needs no correction and accumulates
    # what a cold start accumulates, within the solve's tolerance
    N, dt = 16, 9.0
    ms, mu = _step_inputs(N, dt)
    res = {}
    for warm in (False, True):
        L = _lat(N)
        L.set_params(dt=dt, eps=1e-10)
        ab_cur = torch.zeros_like(mu)
        ab_prev = torch.zeros_like(mu)
        dF = torch.zeros(3, dtype=torch.float64, device="cuda")
        steps = [(2, ms[3], ms[2], ms[1], mu, ab_cur, ab_prev, warm and i > 0) for i in range(4)]
        rs = L.adjoint_steps(steps, dF, eps=1e-12, kmax=500)
        res[warm] = (ab_cur, ab_prev, dF, [r["iters"] for r in rs])
    cold, hot = res[False], res[True]
    assert hot[3][0] == cold[3][0] and max(hot[3][1:]) <= 1 and min(cold[3][1:]) > 5
    for x, y in zip(cold[:3], hot[:3]):
        assert rel_l2(host(y), host(x)) < 1e-10


def test_recorded_moments_give_the_checkpointed_gradients():
    # keeping every step's moments (no replay) changes nothing: same march, same adjoint steps
    N, S, dt = 64, 12, 24.0
    p0, u0, pt, ut, F_star = _problem(N, S, dt)
    out = []
    for record in (False, True):
        from paper_2609_39474_b300.adjoint import MarchRunner
        R = MarchRunner(_lat(N, "fp32"), dt=dt, steps=S, eps=1e-6 * NU / N, checkpoint_every=4, eps_adjoint=1e-5,
                        record_moments=record)
        uS = R.forward(dev(p0), dev(u0), F_star)
        out.append((uS, R.backward(uS - dev(ut)), list(R.adjoint_iters)))
    assert torch.equal(out[0][0], out[1][0]) and out[0][2] == out[1][2]
    for a, b in zip(out[0][1], out[1][1]):
        assert torch.equal(a, b)
