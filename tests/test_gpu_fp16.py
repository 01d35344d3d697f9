"""FP16 population storage (populations in binary16 as f / sigma, FP32 working fields and
arithmetic, FP64 history and solve) against the FP64 oracle: single stages to within one unit in
the last place of the storage format, marches to a stated relative error."""
import numpy as np
import pytest
import torch

from oracle import kinetics as OK
from oracle import march as OM
from oracle import sweep as OSW
from oracle.lattice import lattice_for_dim
from workloads.fields import random_moments, random_phase, random_populations
from tests.gpu_helpers import dev, host, rel_l2

pytestmark = pytest.mark.gpu


def _lib():
    from paper_2609_39474_b300 import lattice as PL
    return PL


def _ulps16(g, o):
    """|g - o| in units of the binary16 spacing at o; below 2^-8 in magnitude the FP32 arithmetic
    (error ~1e-7 of the O(1) terms that cancel there) is the floor, so the unit is 2^-19 there."""
    sp = np.maximum(np.spacing(np.abs(o).astype(np.float16)).astype(np.float64), 2.0 ** -19)
    return np.abs(g - o) / sp


@pytest.mark.parametrize("lift", [False, True], ids=["nolift", "lift"])
@pytest.mark.parametrize("n", [8, 64, 256, 1024])
def test_fp16_sweep_within_one_ulp_of_the_oracle(n, lift):
    PL = _lib()
    lat = lattice_for_dim(2)
    # |f| ~ 0.1 .. 1 (the scaled range msc_init_fields produces) keeps every value a normal binary16
    f = 0.5 + random_populations(9, (n, n), seed=1, scale=0.2)
    h = random_moments(2, (n, n), seed=2, scale=1e-2)
    dm = random_moments(2, (n, n), seed=3, scale=1e-2) if lift else None
    f_s = dev(f, torch.float16)
    h_s = dev(h, torch.float32)
    dm_s = dev(dm, torch.float32) if lift else None
    a = 0.05
    f_out, pr, ss = PL.sweep(2, n, "fp16", a, f_s, h_s, dm_s)
    torch.cuda.synchronize()
    trial = host(f_s) + (OK.linear_lift(lat, host(dm_s)) if lift else 0.0)
    f_T = OSW.sweep(lat, trial, a, host(h_s))
    r, _ = OSW.residual(f_T, trial)
    # outputs: the oracle's value rounded to binary16, up to FP32 arithmetic flipping a rounding
    assert np.max(_ulps16(host(f_out), f_T)) <= 1.0
    # P r and sum r^2 come from the unrounded FP32 collision
    assert rel_l2(host(pr), OK.moments(lat, r)) < 1e-5
    assert abs(float(ss.item()) / float(np.sum(r * r)) - 1) < 1e-5


def test_fp16_equilibrium_within_one_ulp():
    PL = _lib()
    lat = lattice_for_dim(2)
    n = 32
    m = random_moments(2, (n, n), seed=5, scale=1e-1)
    m[0] += 1.0  # keep f_eq in the normal binary16 range
    f = host(PL.equilibrium(2, n, "fp16", dev(m[0]), dev(m[1:])))
    assert np.max(_ulps16(f, OK.feq(lat, m[0], m[1:]))) <= 1.0


def test_fp16_shadow_solve_is_the_fp32_solve():
    # FP16 storage keeps FP32 working fields: the stage solve is the FP32 one
    PL = _lib()
    n = 64
    pr = dev(random_moments(2, (n, n), seed=6, scale=1e-6), torch.float32)
    a = 3.0 / 64.0
    assert torch.equal(PL.shadow_solve(2, n, "fp16", a, 1 / 6, pr), PL.shadow_solve(2, n, "fp32", a, 1 / 6, pr))


def _replay(n, steps, dt, seed, Re=1.0):
    p, u = random_phase(n, 2, Re, seed=seed, kmax=min(8, n // 4))
    U = Re / 6.0 / n
    prm = OM.MarchParams(dt=dt, eps=1e-4 * U, warm_order=2, count_multiple=2)
    st = OM.init_state(lattice_for_dim(2), p, u)
    recs = OM.march(st, prm, steps)
    assert all(r.converged for r in recs)
    PL = _lib()
    L = PL.MscLattice(2, n, "fp16")
    L.set_params(dt=dt, eps=prm.eps, replay=True, warm_order=2, count_multiple=2)
    L.set_replay_counts([r.iters for r in recs])
    L.init_fields(p, u)
    L.march(steps)
    return L, st


# the error against the FP64 oracle (replay of its inner counts), stated per case: binary16 rounds
# every stored population to 2^-11 relative; the march keeps the error in u below that
FP16_GATES = {(64, 10, 32.0): 5e-4, (256, 8, 128.0): 5e-4}  # measured 1.9e-4, 2.3e-4


@pytest.mark.parametrize("n,steps,dt", list(FP16_GATES))
def test_fp16_march_against_fp64_oracle(n, steps, dt):
    L, st = _replay(n, steps, dt, seed=12)
    assert L.stats()["status"] == 0
    err = rel_l2(host(L.fields()[1]), st.m_n[1:])
    print(f"FP16 storage N={n} steps={steps} dt={dt}: relative L2 error in u vs FP64 oracle = {err:.3e}")
    assert err < FP16_GATES[(n, steps, dt)]


def test_fp16_scale_and_state_round_trip():
    # sigma is the power of two above max |f^0|; a saved state (sigma in the header) resumes exactly
    PL = _lib()
    n = 64
    p, u = random_phase(n, 2, 1.0, seed=3, kmax=8)
    A = PL.MscLattice(2, n, "fp16")
    A.set_params(dt=24.0, eps=1e-5)  # ~4e-3 of U: above the binary16 rounding floor (~1e-4 U)
    A.init_fields(p, u)
    f0 = A.populations()
    fmax = np.max(np.abs(OK.feq(lattice_for_dim(2), p, u)))
    sig = 2.0 ** np.ceil(np.log2(fmax))
    if sig == fmax:
        sig *= 2
    stored = f0 / sig
    assert np.max(np.abs(stored)) < 1.0 and np.max(np.abs(stored)) > 0.5
    assert np.array_equal(stored.astype(np.float16).astype(np.float64), stored)  # exactly representable
    A.march(3)
    assert A.stats()["status"] == 0 and A.stats()["steps_done"] == 3
    blob = A.save_state()
    B = PL.MscLattice(2, n, "fp16")
    B.set_params(dt=24.0, eps=1e-5)
    B.load_state(blob)
    assert np.array_equal(A.populations(), B.populations())
    A.march(2)
    B.march(2)
    assert A.stats()["steps_done"] == B.stats()["steps_done"] == 5
    assert np.array_equal(A.populations(), B.populations())
    assert torch.equal(A.fields()[1], B.fields()[1])


def test_fp16_full_size_march_runs_at_a_few_iterations():
    # D2Q9 N = 1024 with FP16 storage, the benchmark field and step: converges like FP32
    PL = _lib()
    n = 1024
    p, u = random_phase(n, 2, 1.0, seed=1)
    L = PL.MscLattice(2, n, "fp16")
    L.set_params(dt=round(0.15 * n * n) / 16, eps=1e-6)
    L.init_fields(p, u)
    L.march(8)
    s = L.stats()
    assert s["status"] == 0 and s["steps_done"] == 8
    assert np.all(L.step_iters() <= 6)


@pytest.mark.parametrize("nu,lam", [(0.12, 0.25), (1 / 6, 0.05), (0.25, 1.0)])
def test_fp16_trt_sweep_within_one_ulp_of_the_oracle(nu, lam):
    # the general TRT collision (Eq. collision) with binary16 storage: the same one-ulp bar
    from oracle import fullsymbol as FS
    PL = _lib()
    lat = lattice_for_dim(2)
    n = 64
    wp, wm = FS.trt_rates(nu, lam)
    f = 0.5 + random_populations(9, (n, n), seed=4, scale=0.2)
    h = random_moments(2, (n, n), seed=5, scale=1e-2)
    dm = random_moments(2, (n, n), seed=6, scale=1e-2)
    f_s, h_s, dm_s = dev(f, torch.float16), dev(h, torch.float32), dev(dm, torch.float32)
    a = 0.05
    f_out, pr, ss = PL.sweep_trt(n, "fp16", a, wp, wm, f_s, h_s, dm_s)
    torch.cuda.synchronize()
    trial = host(f_s) + OK.linear_lift(lat, host(dm_s))
    f_T = OSW.sweep(lat, trial, a, host(h_s), omega=(wp, wm))
    r, _ = OSW.residual(f_T, trial)
    assert np.max(_ulps16(host(f_out), f_T)) <= 1.0
    assert rel_l2(host(pr), OK.moments(lat, r)) < 1e-5
    assert abs(float(ss.item()) / float(np.sum(r * r)) - 1) < 1e-5


def test_fp16_adjoint_gradients_track_fp32():
    # the discrete adjoint on a binary16-storage march (FP32 fields, FP64 history and solve): its
    # gradients follow the FP32-storage ones to the storage format's relative precision
    from paper_2609_39474_b300.adjoint import MarchRunner
    N, S, dt = 64, 8, 24.0
    nu = 1.0 / 6.0
    p0, u0 = random_phase(N, 2, 1.0, seed=3, kmax=8)
    pt, ut = random_phase(N, 2, 1.0, seed=2, kmax=8)
    grads = {}
    for prec in ("fp32", "fp16"):
        # eps above the binary16 rounding floor (~1e-4 U), the same for both storages
        R = MarchRunner(_lib().MscLattice(2, N, prec), dt=dt, steps=S, eps=2e-4 * nu / N, checkpoint_every=4,
                        eps_adjoint=1e-5)
        uS = R.forward(dev(p0), dev(u0))
        grads[prec] = R.backward(uS - dev(ut))
    for a, b in zip(grads["fp16"][1:], grads["fp32"][1:]):
        assert rel_l2(host(a), host(b)) < 5e-3
