"""GPU parity of the batched D2Q9 march (msc_batch_*): every instance of a batch must compute what
the FP64 oracle computes for it (replay mode, 1e-12 in FP64), what a single-context march computes
(bitwise, same iteration path), and keep its own step count, parameters and failure status."""
import numpy as np
import pytest
import torch

from oracle import march as OM
from oracle.lattice import lattice_for_dim
from workloads.fields import random_phase
from tests.gpu_helpers import host, rel_l2

pytestmark = pytest.mark.gpu

NU = 1.0 / 6.0


def _lat(n, precision, **kw):
    from paper_2609_39474_b300.lattice import MscLattice
    return MscLattice(2, n, precision, **kw)


def _batch(lats):
    from paper_2609_39474_b300.lattice import MscBatch
    return MscBatch(lats)


# uneven sizes, Reynolds numbers and step sizes; the tolerance scales with the amplitude U = Re nu / n
# (relative 1e-8 for FP64 storage, 1e-5 for FP32, whose rounding floor is ~1e-7 U)
CASES = [  # n, Re, dt
    (64, 1.0, 40.0),
    (16, 0.1, 6.0),
    (32, 10.0, 12.0),
    (64, 1e-3, 60.0),
    (32, 1.0, 25.0),
]


def _eps(n, Re, precision):
    return (1e-8 if precision == "fp64" else 1e-5) * Re * NU / n


def _fields(i, n, Re):
    return random_phase(n, 2, Re, seed=1000 + i, kmax=min(8, n // 4))


def test_batch_fp64_replay_matches_oracle():
    steps = [5, 7, 4, 3, 6]
    ors, lats = [], []
    for i, ((n, Re, dt), S) in enumerate(zip(CASES, steps)):
        p, u = _fields(i, n, Re)
        eps = _eps(n, Re, "fp64")
        prm = OM.MarchParams(dt=dt, eps=eps)
        st = OM.init_state(lattice_for_dim(2), p, u)
        recs = OM.march(st, prm, S)
        assert all(r.converged for r in recs)
        counts = [r.iters for r in recs]
        L = _lat(n, "fp64")
        L.set_params(dt=dt, eps=eps, replay=True)
        L.set_replay_counts(counts)
        L.init_fields(p, u)
        ors.append((st, recs, counts))
        lats.append(L)
    B = _batch(lats)
    B.march(steps)
    for (st, recs, counts), L, S in zip(ors, lats, steps):
        s = L.stats()
        assert s["status"] == 0 and s["steps_done"] == S and s["inner_total"] == sum(counts)
        assert list(L.step_iters()) == counts
        ph, uu = L.fields(on_device=False)
        assert rel_l2(uu.numpy(), st.m_n[1:]) < 1e-12
        assert rel_l2(L.populations(), st.f) < 1e-12
        Ro = np.concatenate([r.residuals for r in recs])
        assert rel_l2(L.residual_history(), Ro) < 1e-9


def _singles_and_batch(precision, steps, replay_from_single=True, tune=None):
    """Free-running single marches, then the same instances batched (replay of the single counts)."""
    singles, counts, lats = [], [], []
    for i, ((n, Re, dt), S) in enumerate(zip(CASES, steps)):
        p, u = _fields(i, n, Re)
        eps = _eps(n, Re, precision)
        A = _lat(n, precision)
        A.set_params(dt=dt, eps=eps)
        A.init_fields(p, u)
        A.march(S)
        assert A.stats()["status"] == 0
        singles.append(A)
        counts.append(list(A.step_iters()))
        L = _lat(n, precision)
        L.set_params(dt=dt, eps=eps, replay=replay_from_single)
        if replay_from_single:
            L.set_replay_counts(counts[-1])
        L.init_fields(p, u)
        lats.append(L)
    B = _batch(lats)
    if tune is not None:
        tune(B)
    B.march(steps)
    return singles, counts, lats, B


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_replay_is_bitwise_the_single_march(precision):
    steps = [4, 6, 3, 5, 2]
    singles, counts, lats, _ = _singles_and_batch(precision, steps)
    for A, L, c in zip(singles, lats, counts):
        assert list(L.step_iters()) == c
        assert np.array_equal(A.populations(), L.populations())
        assert torch.equal(A.fields()[1], L.fields()[1])


def test_batch_free_run_follows_single_marches_fp32():
    steps = [6, 6, 6, 6, 6]
    singles, counts, lats, _ = _singles_and_batch("fp32", steps, replay_from_single=False)
    agree = 0
    for A, L, c in zip(singles, lats, counts):
        s = L.stats()
        assert s["status"] == 0 and s["steps_done"] == 6
        agree += int(list(L.step_iters()) == c)
        assert rel_l2(host(L.fields()[1]), host(A.fields()[1])) < 1e-5
    assert agree >= 4  # the residual norm is summed in another order: a borderline step may differ


def test_batch_autotune_keeps_results_bitwise():
    steps = [3, 4, 2, 3, 4]
    tuned = {}

    def tune(B):
        tuned.update(B.autotune(reps=2))

    singles, counts, lats, B = _singles_and_batch("fp32", steps, tune=tune)
    assert tuned["n"] == [64, 32, 16]
    for k, n in enumerate(tuned["n"]):
        assert tuned["sweep_rows"][k] in (4, 8, 16, 32, 64) and tuned["sweep_rows"][k] <= n
        pts = 4 if n <= 256 else 16  # points per thread: radix-4 transforms at n <= 256
        assert tuned["fft_rows"][k] * n // pts <= 256 and tuned["col_lines"][k] >= 1
    assert tuned["sweep_us"] > 0 and tuned["rowfft_us"] > 0 and tuned["colsolve_us"] > 0
    assert B.tuning["sweep_rows"] == tuned["sweep_rows"]
    for A, L, c in zip(singles, lats, counts):
        assert list(L.step_iters()) == c
        assert np.array_equal(A.populations(), L.populations())


def test_batch_set_tuning_validates():
    from paper_2609_39474_b300._lib import MscError
    lats = []
    for n, Re, dt in CASES[:2]:
        L = _lat(n, "fp32")
        lats.append(L)
    B = _batch(lats)
    t = B.tuning
    bad = dict(t, sweep_rows=[3] + t["sweep_rows"][1:])
    with pytest.raises(MscError):
        B.set_tuning(bad)
    bad = dict(t, fft_rows=[t["n"][0]] + t["fft_rows"][1:])  # P > n/2
    with pytest.raises(MscError):
        B.set_tuning(bad)
    good = dict(t, sweep_rows=[8, 8], fft_rows=[2, 2], col_lines=[2, 4], sweep_ctas_per_sm=2)
    B.set_tuning(good)
    assert B.tuning["col_lines"] == [2, 4] and B.tuning["sweep_ctas_per_sm"] == 2


def test_batch_uneven_counts_zero_steps_and_a_failing_instance():
    # instance 1 takes no step; instance 2 cannot converge (K_max = 2, eps unreachable) and stops
    # at its first step with the state of the last accepted step; the others are unaffected
    steps = [4, 0, 3, 5]
    cases = [CASES[0], CASES[1], CASES[2], CASES[4]]
    singles, lats = [], []
    for i, ((n, Re, dt), S) in enumerate(zip(cases, steps)):
        p, u = _fields(i, n, Re)
        eps = _eps(n, Re, "fp64")
        L = _lat(n, "fp64")
        if i == 2:
            L.set_params(dt=dt, eps=1e-300, kmax=2)
        else:
            L.set_params(dt=dt, eps=eps)
        L.init_fields(p, u)
        lats.append(L)
        A = _lat(n, "fp64")
        if i == 2:
            A.set_params(dt=dt, eps=1e-300, kmax=2)
        else:
            A.set_params(dt=dt, eps=eps)
        A.init_fields(p, u)
        if S:
            A.march(S)
        singles.append(A)
    f_before = [L.populations() for L in lats]
    B = _batch(lats)
    B.march(steps)
    for i, (A, L) in enumerate(zip(singles, lats)):
        s = L.stats()
        if i == 1:
            assert s["steps_done"] == 0 and np.array_equal(L.populations(), f_before[1])
        elif i == 2:
            assert s["status"] == 2 and s["steps_done"] == 0  # MSC_ERR_NONCONVERGED
            assert np.array_equal(L.populations(), f_before[2])
        else:
            assert s["status"] == 0 and s["steps_done"] == steps[i]
            assert list(L.step_iters()) == list(A.step_iters())
            assert np.array_equal(L.populations(), A.populations())
    # a second call continues every instance from where it stopped
    B.march([1, 2, 0, 1])
    assert lats[0].stats()["steps_done"] == 5 and lats[1].stats()["steps_done"] == 2
    assert lats[3].stats()["steps_done"] == 6


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_explicit_march_is_bitwise_the_single(precision):
    counts = [13, 8, 0, 5, 16]
    singles, lats = [], []
    for i, (n, Re, dt) in enumerate(CASES):
        p, u = _fields(i, n, Re)
        A = _lat(n, precision)
        A.init_fields(p, u)
        if counts[i]:
            A.explicit_march(counts[i])
        singles.append(A)
        L = _lat(n, precision)
        L.init_fields(p, u)
        lats.append(L)
    B = _batch(lats)
    B.explicit_march(counts)
    for A, L in zip(singles, lats):
        assert np.array_equal(A.populations(), L.populations())
        assert torch.equal(A.fields()[1], L.fields()[1])


def test_batch_reynolds_sweep_fp32_against_the_fp64_oracle():
    # the parameter sweep of the batched workload at small n: Re log-spaced over 1e-4 .. 10 (the
    # Mach number U sqrt(3) stays small at these n), two sizes, FP32 storage in replay of the
    # oracle's counts (same warm-start order on both sides)
    Res = np.logspace(-4, 1, 4)
    ors, lats, steps = [], [], []
    for i, (n, Re) in enumerate([(n, Re) for n in (64, 32) for Re in Res]):
        p, u = _fields(i, n, Re)
        U = Re * NU / n
        T_end = round(0.15 * n * n)
        S = 16
        # the FP32 D2Q9 defaults: linear warm start, inner sweeps in pairs
        prm = OM.MarchParams(dt=T_end / S, eps=1e-6 * U, warm_order=2, count_multiple=2)
        st = OM.init_state(lattice_for_dim(2), p, u)
        recs = OM.march(st, prm, S)
        assert all(r.converged for r in recs)
        counts = [r.iters for r in recs]
        L = _lat(n, "fp32")
        L.set_params(dt=prm.dt, eps=prm.eps, replay=True, warm_order=2, count_multiple=2)
        L.set_replay_counts(counts)
        L.init_fields(p, u)
        ors.append(st)
        lats.append(L)
        steps.append(S)
    B = _batch(lats)
    B.autotune(reps=1)
    B.march(steps)
    for st, L in zip(ors, lats):
        assert L.stats()["status"] == 0
        assert rel_l2(host(L.fields()[1]), st.m_n[1:]) < 1e-5
