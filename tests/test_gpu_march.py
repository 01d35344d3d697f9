"""GPU parity of the device-resident march (Algorithm 1, Picard, explicit LBM) against the FP64
oracle, through the C ABI.  Parity runs in replay mode: the oracle's accepted inner counts are
forced on the GPU so that a residual within rounding of eps cannot change the iteration path."""
import numpy as np
import pytest
import torch

from oracle import kinetics as OK
from oracle import march as OM
from oracle.lattice import lattice_for_dim
from workloads.fields import random_phase, tgv2d, tgv3d
from workloads.metrics import nint
from tests.gpu_helpers import host, rel_l2

pytestmark = pytest.mark.gpu


def _lattice(dim, n, precision, **kw):
    from paper_2609_39474_b300.lattice import MscLattice
    return MscLattice(dim, n, precision, **kw)


def _replay_run(dim, n, precision, p, u, prm: OM.MarchParams, counts, corrector=True):
    L = _lattice(dim, n, precision)
    L.set_params(dt=prm.dt, eps=prm.eps, nu=prm.nu, kmax=prm.kmax, nmin=prm.nmin, corrector=corrector,
                 replay=True, warm_order=prm.warm_order, count_multiple=prm.count_multiple)
    L.set_replay_counts(counts)
    L.init_fields(p, u)
    L.march(len(counts))
    return L


def _config1():
    # D2Q9 N = 64, FP64, Taylor-Green at Re = 1, T_end = nint(0.05 N^2 / nu) = 1229, S = 38 steps
    N, T_end = 64, nint(0.05 * 64 ** 2 * 6)
    S = nint(T_end / 32)
    prm = OM.MarchParams(dt=T_end / S, eps=1e-10)
    p, u = tgv2d(N, 1.0)
    return N, S, prm, p, u


def test_config1_tgv_fp64_replay_parity_short_horizon():
    # Continuous replay: identical inner counts, so GPU and oracle differ only by rounding.  Over
    # the first 20 steps that difference stays at rounding level (sub-tolerance components are
    # amplified only later in the run, see the step-by-step test below).
    N, S, prm, p, u = _config1()
    st = OM.init_state(lattice_for_dim(2), p, u)
    recs = OM.march(st, prm, 20)
    counts = [r.iters for r in recs]
    L = _replay_run(2, N, "fp64", p, u, prm, counts)
    s = L.stats()
    assert s["status"] == 0 and s["steps_done"] == 20 and s["inner_total"] == sum(counts)
    ph, uu = L.fields(on_device=False)
    assert rel_l2(uu.numpy(), st.m_n[1:]) < 1e-12
    assert rel_l2(ph.numpy(), st.m_n[0]) < 1e-10
    assert rel_l2(L.populations(), st.f) < 1e-12
    R = L.residual_history()
    Ro = np.concatenate([r.residuals for r in recs])
    assert len(R) == len(Ro) and rel_l2(R, Ro) < 1e-9
    assert list(L.step_iters()) == counts


def test_config1_tgv_fp64_stepwise_parity_full_run():
    # Every one of the 38 physical steps from the oracle's own previous state: 1e-12 in u per step.
    N, S, prm, p, u = _config1()
    from tests.gpu_helpers import state_blob
    st = OM.init_state(lattice_for_dim(2), p, u)
    L = _lattice(2, N, "fp64")
    L.set_params(dt=prm.dt, eps=prm.eps, replay=True)
    worst = 0.0
    for k in range(S):
        blob = state_blob(2, N, "fp64", st)
        rec = OM.physical_step(st, prm)
        L.load_state(blob)
        L.set_replay_counts([rec.iters])
        L.march(1)
        s = L.stats()
        assert s["status"] == 0 and s["last_q"] == (1 if k == 0 else 2)
        worst = max(worst, rel_l2(host(L.fields()[1]), st.m_n[1:]))
    assert worst < 1e-12


def test_config1_free_run_agrees_to_tolerance_level():
    # Over the whole run, rounding differences below eps are amplified across steps (in the oracle
    # as well: a 1e-15 perturbation of its own input grows to ~2e-5); the free-running GPU march must
    # agree with the oracle to that eps level and meet the same closed-form accuracy.
    N, S, prm, p, u = _config1()
    st = OM.init_state(lattice_for_dim(2), p, u)
    OM.march(st, prm, S)
    L = _lattice(2, N, "fp64")
    L.set_params(dt=prm.dt, eps=prm.eps)
    L.init_fields(p, u)
    L.march(S)
    assert L.stats()["status"] == 0
    ug = host(L.fields()[1])
    assert rel_l2(ug, st.m_n[1:]) < 1e-3
    _, u_ref = tgv2d(N, 1.0, t=nint(0.05 * 64 ** 2 * 6))
    e_gpu = np.sqrt(np.mean(np.sum((ug - u_ref) ** 2, axis=0)))
    e_or = np.sqrt(np.mean(np.sum((st.m_n[1:] - u_ref) ** 2, axis=0)))
    assert abs(e_gpu / e_or - 1) < 1e-2


def test_free_running_march_follows_the_oracle():
    N = 64
    p, u = random_phase(N, 2, 1.0, seed=11, kmax=8)
    prm = OM.MarchParams(dt=40.0, eps=1e-9)
    st = OM.init_state(lattice_for_dim(2), p, u)
    recs = OM.march(st, prm, 12)
    L = _lattice(2, N, "fp64")
    L.set_params(dt=prm.dt, eps=prm.eps)
    L.init_fields(p, u)
    L.march(12)
    s = L.stats()
    assert s["status"] == 0 and s["steps_done"] == 12
    it = L.step_iters()
    assert np.mean(it == np.array([r.iters for r in recs])) >= 0.9
    assert rel_l2(host(L.fields()[1]), st.m_n[1:]) < 1e-7  # within the tolerance-level path noise


def test_picard_replay_parity_fp64():
    N = 32
    p, u = tgv2d(N, 1.0)
    prm = OM.MarchParams(dt=16.0, eps=1e-11, corrector=False, kmax=2000)
    st = OM.init_state(lattice_for_dim(2), p, u)
    recs = OM.march(st, prm, 4)
    L = _replay_run(2, N, "fp64", p, u, prm, [r.iters for r in recs], corrector=False)
    assert rel_l2(host(L.fields()[1]), st.m_n[1:]) < 1e-12


def test_3d_tgv_fp64_replay_parity():
    N = 16
    p, u = tgv3d(N, 1.0)
    prm = OM.MarchParams(dt=4.0, eps=1e-10, nmin=1)
    st = OM.init_state(lattice_for_dim(3), p, u)
    recs = OM.march(st, prm, 5)
    L = _replay_run(3, N, "fp64", p, u, prm, [r.iters for r in recs])
    assert L.stats()["status"] == 0
    assert rel_l2(host(L.fields()[1]), st.m_n[1:]) < 1e-12


@pytest.mark.parametrize("dim,N,steps", [(2, 64, 10), (3, 16, 4)])
def test_fp32_storage_against_fp64_oracle(dim, N, steps):
    # FP32 deviation storage with FP64 history and solve: gate 1e-5 relative L2 in u
    p, u = random_phase(N, dim, 1.0, seed=12, kmax=8 if dim == 2 else 4)
    # the FP32 path's default warm start is the linear one (warm_order 2); the oracle uses the same
    prm = OM.MarchParams(dt=32.0, eps=1e-9, nmin=2 if dim == 2 else 1, warm_order=2,
                         count_multiple=2 if dim == 2 else 1)
    st = OM.init_state(lattice_for_dim(dim), p, u)
    recs = OM.march(st, prm, steps)
    L = _replay_run(dim, N, "fp32", p, u, prm, [r.iters for r in recs])
    assert L.stats()["status"] == 0
    assert rel_l2(host(L.fields()[1]), st.m_n[1:]) < 1e-5


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_explicit_march_matches_oracle(precision):
    N, steps = 32, 37  # odd count exercises the unpaired last step
    p, u = tgv2d(N, 10.0)
    L = _lattice(2, N, precision)
    L.init_fields(p, u)
    L.explicit_march(steps)
    f = OM.explicit_march(lattice_for_dim(2), OM.init_state(lattice_for_dim(2), p, u).f, steps)
    tol = 1e-12 if precision == "fp64" else 1e-5
    assert rel_l2(L.populations(), f) < tol
    m = OK.moments(lattice_for_dim(2), f)
    assert rel_l2(host(L.fields()[1]), m[1:]) < tol


def test_explicit_march_3d():
    N, steps = 16, 6
    p, u = tgv3d(N, 10.0)
    L = _lattice(3, N, "fp64")
    L.init_fields(p, u)
    L.explicit_march(steps)
    f = OM.explicit_march(lattice_for_dim(3), OM.init_state(lattice_for_dim(3), p, u).f, steps)
    assert rel_l2(L.populations(), f) < 1e-12


def test_nonconvergent_step_reports_and_keeps_state():
    p, u = tgv2d(32, 1.0)
    L = _lattice(2, 32, "fp64")
    L.set_params(dt=8.0, eps=1e-30, kmax=3)
    L.init_fields(p, u)
    f0 = L.populations()
    L.march(4)
    s = L.stats()
    assert s["status"] == 2 and s["steps_done"] == 0 and s["inner_total"] == 3
    assert np.array_equal(L.populations(), f0)


def test_nonfinite_residual_stops_the_march():
    p, u = tgv2d(32, 1.0)
    u = u.copy()
    u[0, 3, 3] = np.nan
    L = _lattice(2, 32, "fp64")
    L.set_params(dt=8.0, eps=1e-8)
    L.init_fields(p, u)
    L.march(2)
    s = L.stats()
    assert s["status"] == 3 and s["steps_done"] == 0


def test_save_load_roundtrip_continues_identically():
    p, u = tgv2d(32, 1.0)
    prm = dict(dt=16.0, eps=1e-10)
    A = _lattice(2, 32, "fp64")
    A.set_params(**prm)
    A.init_fields(p, u)
    A.march(3)
    blob = A.save_state()
    A.march(2)
    B = _lattice(2, 32, "fp64")
    B.set_params(**prm)
    B.load_state(blob)
    B.march(2)
    assert np.array_equal(A.populations(), B.populations())
    assert B.stats()["steps_done"] == 5


def test_march_continues_across_calls():
    p, u = tgv2d(32, 1.0)
    prm = OM.MarchParams(dt=16.0, eps=1e-10)
    st = OM.init_state(lattice_for_dim(2), p, u)
    recs = OM.march(st, prm, 6)
    counts = [r.iters for r in recs]
    L = _lattice(2, 32, "fp64")
    L.set_params(dt=16.0, eps=1e-10, replay=True)
    L.init_fields(p, u)
    L.set_replay_counts(counts[:2])
    L.march(2)
    L.set_replay_counts(counts[2:])
    L.march(4)
    assert L.stats()["steps_done"] == 6
    assert rel_l2(host(L.fields()[1]), st.m_n[1:]) < 1e-12


def test_full_size_march_conserves_and_converges():
    # D2Q9 N = 1024 FP32, the benchmark configuration: a few steps, properties that hold at any size
    N = 1024
    p, u = random_phase(N, 2, 1.0, seed=1)
    L = _lattice(2, N, "fp32")
    L.set_params(dt=128.0, eps=1e-9)
    L.init_fields(p, u)
    m0 = [float(x.sum()) for x in (L.fields()[0], *L.fields()[1])]
    L.march(4)
    s = L.stats()
    assert s["status"] == 0 and s["steps_done"] == 4
    it = L.step_iters()
    assert np.all(it >= 2) and np.all(it <= 12)
    ph, uu = L.fields()
    m1 = [float(ph.sum()), float(uu[0].sum()), float(uu[1].sum())]
    scale = float(torch.abs(uu).max()) * N * N
    assert max(abs(a - b) for a, b in zip(m0, m1)) < 1e-6 * scale


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_benchmark_configuration_matches_oracle(precision):
    # The benchmark's workload itself: D2Q9 N = 1024, the random-phase field of seed 1 at Re = 1, the
    # headline candidate's step dt = T_end / 16 (T_end = nint(0.15 N^2)) and eps = 1e-6, through the
    # BDF1 starter and one BDF2 step, with each precision's default warm start and pairing; the GPU
    # replays the oracle's inner counts.  Gates: 1e-5 relative L2 in u with FP32 storage, 1e-12 with
    # FP64.  At this step a_1 = 1/dt ~ 1e-4 and the Schur solve (Eq. schur) divides the long waves of
    # the residual moments by a + nu |k|^2, so a coherent relative bias of one unit roundoff in the
    # collision's moments would move u by ~u_r / a (~6e-4 in binary32); the sweep therefore keeps the
    # rounded 1/(1 + a/2) and the rounded lattice weights from biasing them.
    N = 1024
    p, u = random_phase(N, 2, 1.0, seed=1)
    fp32 = precision == "fp32"
    prm = OM.MarchParams(dt=nint(0.15 * N * N) / 16, eps=1e-6, nmin=2, warm_order=2 if fp32 else 3,
                         count_multiple=2 if fp32 else 1)
    st = OM.init_state(lattice_for_dim(2), p, u)
    recs = OM.march(st, prm, 2)
    assert all(r.converged for r in recs)
    L = _replay_run(2, N, precision, p, u, prm, [r.iters for r in recs])
    assert L.stats()["status"] == 0 and L.stats()["steps_done"] == 2
    _, uu = L.fields()
    # the gate is on u (p_hat of this field is the quadratic Poisson pressure, O(U^2))
    assert rel_l2(host(uu), st.m_n[1:]) < (1e-5 if fp32 else 1e-12)


@pytest.mark.parametrize("dim,N,precision,nmin,corrector,eps", [
    (2, 64, "fp64", None, True, 1e-9), (2, 128, "fp32", None, True, 1e-9), (3, 16, "fp64", None, True, 1e-9),
    # the graph runs the first n_min - 1 iterations of a step as straight-line nodes: three of them,
    # in 2D and 3D, and with the corrector off (their correction passes then return at once)
    (2, 64, "fp64", 4, True, 1e-9), (3, 16, "fp32", 4, True, 1e-9), (2, 32, "fp64", 3, False, 1e-6)])
def test_stepwise_march_equals_graph_march(dim, N, precision, nmin, corrector, eps):
    # the host-driven march launches the same kernels: identical bits to the graph march
    p, u = random_phase(N, dim, 1.0, seed=21, kmax=4)
    out = []
    for stepwise in (False, True):
        L = _lattice(dim, N, precision)
        L.set_params(dt=24.0 if corrector else 4.0, eps=eps, nmin=nmin, corrector=corrector, kmax=2000)
        L.init_fields(p, u)
        (L.march_stepwise if stepwise else L.march)(5)
        out.append((L.populations(), L.step_iters().tolist(), L.stats()))
    assert out[0][2]["status"] == out[1][2]["status"] == 0
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1] and out[0][2]["steps_done"] == out[1][2]["steps_done"] == 5
    if nmin:
        assert min(out[0][1]) >= nmin


def test_fp32_long_run_stays_at_a_few_iterations():
    # D2Q9 N = 256, Re = 1, 64 steps of dt = 153.6: with FP32 storage the cubic warm start grows the
    # rounding in the staggered modes (k = (pi, 0), (0, pi): P Z E has eigenvalue -1 there, outside the
    # mask) until the inner solve stalls; the linear warm start with inner sweeps in pairs (the FP32
    # D2Q9 defaults) keeps 2-4 iterations
    N, S = 256, 64
    p, u = random_phase(N, 2, 1.0, seed=1)
    L = _lattice(2, N, "fp32")
    L.set_params(dt=9830.0 / S, eps=1e-8)
    L.init_fields(p, u)
    L.march(S)
    s = L.stats()
    assert s["status"] == 0 and s["steps_done"] == S
    assert np.max(L.step_iters()) <= 4


@pytest.mark.parametrize("order", [1, 2])
def test_warm_order_parity_fp64(order):
    # truncated warm starts against the oracle with the same rule (replay mode)
    p, u = tgv2d(32, 1.0)
    prm = OM.MarchParams(dt=16.0, eps=1e-10, warm_order=order)
    st = OM.init_state(lattice_for_dim(2), p, u)
    recs = OM.march(st, prm, 5)
    L = _replay_run(2, 32, "fp64", p, u, prm, [r.iters for r in recs])
    assert rel_l2(host(L.fields()[1]), st.m_n[1:]) < 1e-12


def test_count_multiple_free_run_fp64():
    # sweeps in pairs: the free-running GPU march takes the oracle's (even) inner counts
    N = 32
    p, u = random_phase(N, 2, 1.0, seed=8, kmax=4)
    prm = OM.MarchParams(dt=30.0, eps=1e-11, warm_order=2, count_multiple=2)
    st = OM.init_state(lattice_for_dim(2), p, u)
    recs = OM.march(st, prm, 6)
    L = _lattice(2, N, "fp64")
    L.set_params(dt=prm.dt, eps=prm.eps, warm_order=2, count_multiple=2)
    L.init_fields(p, u)
    L.march(6)
    it = L.step_iters().tolist()
    assert all(k % 2 == 0 for k in it) and L.stats()["status"] == 0
    assert np.mean(np.array(it) == np.array([r.iters for r in recs])) >= 0.8
    assert rel_l2(host(L.fields()[1]), st.m_n[1:]) < 1e-8


def _fp32_horizon_parity(N, S, steps, eps, nmin=2):
    # Table protocol T_end = nint(0.15 N^2), dt = T_end / S, the FP32 D2Q9 defaults (linear warm start,
    # inner sweeps in pairs) on both sides; the GPU replays the oracle's accepted inner counts
    p, u = random_phase(N, 2, 1.0, seed=1)
    prm = OM.MarchParams(dt=nint(0.15 * N * N) / S, eps=eps, nmin=nmin, warm_order=2, count_multiple=2)
    st = OM.init_state(lattice_for_dim(2), p, u)
    recs = OM.march(st, prm, steps)
    assert all(r.converged for r in recs)
    L = _replay_run(2, N, "fp32", p, u, prm, [r.iters for r in recs])
    s = L.stats()
    assert s["status"] == 0 and s["steps_done"] == steps
    err = rel_l2(host(L.fields()[1]), st.m_n[1:])
    print(f"FP32 storage vs FP64 oracle, D2Q9 N={N}, dt=T_end/{S}, n_min={nmin}, {steps} steps: "
          f"rel L2(u) = {err:.2e} (gate 1e-5)")
    return err


def test_fp32_full_horizon_n256_matches_oracle():
    # The N = 256 workload over its whole horizon at the timed candidate: S = 192 physical steps to
    # T_end = 9830 (eps = 1e-6, n_min = 2), 1e-5 relative L2 in u against the FP64 oracle
    assert _fp32_horizon_parity(256, 192, 192, 1e-6) < 1e-5


def test_fp32_n1024_many_steps_match_oracle():
    # The N = 1024 benchmark workload at the timed candidate, dt = T_end / 352 with n_min = 4 (four
    # sweeps per step, eps = 1e-8), over the BDF1 starter and 17 BDF2 steps: 1e-5 relative L2 in u
    # against the FP64 oracle
    assert _fp32_horizon_parity(1024, 352, 18, 1e-8, nmin=4) < 1e-5


def test_fp32_n1024_two_sweep_candidate_matches_oracle():
    # the two-sweep candidate of the same workload (dt = T_end / 512, eps = 1e-10, n_min = 2)
    assert _fp32_horizon_parity(1024, 512, 18, 1e-10) < 1e-5
