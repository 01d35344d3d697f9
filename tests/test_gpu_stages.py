"""GPU parity of the single stages (sweep, shadow solve, equilibrium, explicit step) against the
FP64 oracle on the same seeded inputs, through the C ABI."""
import numpy as np
import pytest
import torch

from oracle import kinetics as OK
from oracle import shadow as OS
from oracle import sweep as OSW
from oracle.lattice import lattice_for_dim
from workloads.fields import random_moments, random_populations
from tests.gpu_helpers import dev, host, rel_l2

pytestmark = pytest.mark.gpu

# (dim, n): n = 8 wraps the 32-column warp strip onto itself, 64 leaves a ragged last strip,
# 256 spans many strips and row blocks, 1024 is the full 2D benchmark size; 3D likewise up to 128.
SWEEP_CASES = [(2, 8), (2, 16), (2, 64), (2, 256), (3, 8), (3, 16), (3, 32)]
TOL = {"fp64": dict(f=1e-14, pr=1e-13, ss=1e-12), "fp32": dict(f=1e-6, pr=1e-5, ss=1e-5)}


def _lib():
    from paper_2609_39474_b300 import lattice as PL
    return PL


def _sweep_case(dim, n, precision, lift, seed=0, a=0.05):
    PL = _lib()
    lat = lattice_for_dim(dim)
    shape = (n,) * dim
    f = random_populations(lat.Q, shape, seed=seed, scale=1e-3)
    h = random_moments(dim, shape, seed=seed + 1, scale=1e-4)
    dm = random_moments(dim, shape, seed=seed + 2, scale=1e-4) if lift else None
    T = PL.storage_dtype(precision)
    # both sides start from the same (storage-rounded) inputs
    f_s = dev(f, T)
    h_s = dev(h, T)
    dm_s = dev(dm, T) if lift else None
    f_out, pr, ss = PL.sweep(dim, n, precision, a, f_s, h_s, dm_s)
    torch.cuda.synchronize()
    f_in = host(f_s)
    trial = f_in + (OK.linear_lift(lat, host(dm_s)) if lift else 0.0)
    f_T = OSW.sweep(lat, trial, a, host(h_s))
    r, R = OSW.residual(f_T, trial)
    return host(f_out), host(pr), float(ss.item()), f_T, OK.moments(lat, r), float(np.sum(r * r))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("lift", [False, True], ids=["nolift", "lift"])
@pytest.mark.parametrize("dim,n", SWEEP_CASES)
def test_sweep_matches_oracle(dim, n, precision, lift):
    g_f, g_pr, g_ss, o_f, o_pr, o_ss = _sweep_case(dim, n, precision, lift)
    tol = TOL[precision]
    assert rel_l2(g_f, o_f) < tol["f"]
    assert rel_l2(g_pr, o_pr) < tol["pr"]
    assert abs(g_ss / o_ss - 1) < tol["ss"]


@pytest.mark.parametrize("dim,n", [(2, 1024), (3, 128)])
def test_sweep_full_size_fp32(dim, n):
    # the benchmark sizes (D2Q9 N = 1024, D3Q19 N = 128) in the benchmark's launch configuration
    g_f, g_pr, g_ss, o_f, o_pr, o_ss = _sweep_case(dim, n, "fp32", True, seed=7)
    assert rel_l2(g_f, o_f) < TOL["fp32"]["f"]
    assert rel_l2(g_pr, o_pr) < TOL["fp32"]["pr"]
    assert abs(g_ss / o_ss - 1) < TOL["fp32"]["ss"]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("dim,n", [(2, 8), (2, 16), (2, 64), (2, 256), (3, 8), (3, 16), (3, 32)])
def test_shadow_solve_matches_oracle(dim, n, precision):
    PL = _lib()
    shape = (n,) * dim
    pr = random_moments(dim, shape, seed=3, scale=1e-6)
    a, nu = 3.0 / (2 * 32.0), 1.0 / 6.0
    T = PL.storage_dtype(precision)
    pr_s = dev(pr, T)
    dm = host(PL.shadow_solve(dim, n, precision, a, nu, pr_s))
    ref = OS.shadow_dm(host(pr_s), a, nu)
    assert rel_l2(dm, ref) < (1e-13 if precision == "fp64" else 2e-6)


def test_shadow_solve_full_size_fp32():
    PL = _lib()
    n = 1024
    pr = random_moments(2, (n, n), seed=4, scale=1e-6)
    a = 3.0 / (2 * 64.0)
    pr_s = dev(pr, torch.float32)
    dm = host(PL.shadow_solve(2, n, "fp32", a, 1 / 6, pr_s))
    ref = OS.shadow_dm(host(pr_s), a, 1 / 6)
    assert rel_l2(dm, ref) < 2e-6


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("dim,n", [(2, 256), (2, 1024), (3, 32)])
def test_shadow_solve_unaligned_arrays_match_aligned(dim, n, precision):
    # the row passes move 16-byte vectors of P r and dm when both arrays are 16-byte aligned and
    # single elements otherwise: arrays one element off alignment give the same bits (and both
    # match the oracle)
    import ctypes
    from paper_2609_39474_b300 import _lib as LB
    PL = _lib()
    shape = (n,) * dim
    pr = random_moments(dim, shape, seed=9, scale=1e-6)
    a, nu = 3.0 / (2 * 48.0), 1.0 / 6.0
    T = PL.storage_dtype(precision)
    pr_s = dev(pr, T)
    dm0 = PL.shadow_solve(dim, n, precision, a, nu, pr_s)
    k = pr_s.numel()
    pb = torch.zeros(k + 1, dtype=T, device=pr_s.device)
    pb[1:] = pr_s.reshape(-1)
    db = torch.zeros(k + 1, dtype=T, device=pr_s.device)
    assert pb[1:].data_ptr() % 16 != 0 and db[1:].data_ptr() % 16 != 0
    sc = PL.StageScratch(dim, n, precision, pr_s.device)
    rc = LB.lib.msc_shadow_solve(dim, n, PL.precision_code(precision), a, nu, ctypes.c_void_p(pb[1:].data_ptr()),
                                 ctypes.c_void_p(db[1:].data_ptr()), ctypes.c_void_p(sc.buf.data_ptr()), sc.nbytes,
                                 None)
    assert rc == 0
    torch.cuda.synchronize()
    assert torch.equal(db[1:].reshape(dm0.shape), dm0)
    assert rel_l2(host(dm0), OS.shadow_dm(host(pr_s), a, nu)) < (1e-13 if precision == "fp64" else 2e-6)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("dim,n", [(2, 16), (3, 8)])
def test_equilibrium_matches_oracle(dim, n, precision):
    PL = _lib()
    lat = lattice_for_dim(dim)
    m = random_moments(dim, (n,) * dim, seed=5, scale=1e-2)
    f = host(PL.equilibrium(dim, n, precision, dev(m[0]), dev(m[1:])))
    ref = OK.feq(lat, m[0], m[1:])
    assert rel_l2(f, ref) < (1e-15 if precision == "fp64" else 1e-7)


@pytest.mark.parametrize("dim,n", [(2, 64), (3, 16)])
def test_sweep_with_zero_source_is_explicit_step(dim, n):
    PL = _lib()
    lat = lattice_for_dim(dim)
    f = random_populations(lat.Q, (n,) * dim, seed=6, scale=1e-3)
    zero = torch.zeros((dim + 1,) + (n,) * dim, dtype=torch.float64, device="cuda")
    f_out, _, _ = PL.sweep(dim, n, "fp64", 0.0, dev(f), zero)
    assert rel_l2(host(f_out), OSW.explicit_step(lat, f)) < 1e-14


def test_stage_argument_checks():
    PL = _lib()
    from paper_2609_39474_b300 import _lib as L
    f = torch.zeros((9, 16, 16), dtype=torch.float64, device="cuda")
    with pytest.raises(L.MscError):
        PL.sweep(2, 16, "fp64", -1.0, f, torch.zeros((3, 16, 16), dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        PL.sweep(2, 16, "fp32", 0.1, f, torch.zeros((3, 16, 16), dtype=torch.float64, device="cuda"))


def test_integer_pipe_conversions_match_the_hardware():
    # the step kernels' binary32 <-> binary64 conversions (widening, round-to-nearest-even
    # narrowing) against CUDA's conversions on 16 M random patterns each, ties included
    import ctypes
    from paper_2609_39474_b300 import _lib as L
    bad = ctypes.c_int(-1)
    assert L.lib.msc_selftest_conversions(64, 1024, 12345, ctypes.byref(bad)) == 0
    assert bad.value == 0


def _periodic_window(t, starts, size):
    """Rows starts[i] - 1 .. starts[i] + size of each grid axis of the device tensor t (C, *grid), with
    periodic wrap, as a host array: a window whose interior sweeps exactly like the full grid."""
    n = t.shape[1]
    idx = [torch.as_tensor(np.arange(s - 1, s + size + 1) % n, device=t.device) for s in starts]
    w = t
    for ax, ix in enumerate(idx):
        w = torch.index_select(w, 1 + ax, ix)
    return host(w)


@pytest.mark.parametrize("dim,n,precision", [(2, 4096, "fp32"), (2, 2048, "fp64"), (3, 256, "fp32"),
                                             (3, 128, "fp64")])
def test_sweep_at_the_largest_sizes_sampled(dim, n, precision):
    # the largest lattices each precision supports (D2Q9 N = 4096 is also the size of the benchmark's
    # roofline loop): the oracle sweeps small periodic windows around sampled sites (the wrap-around
    # corners, strip and tile boundaries, the ragged last strip) whose interiors are exact, and the
    # reported sum r^2 equals the norm of the GPU outputs' own residual
    PL = _lib()
    lat = lattice_for_dim(dim)
    shape = (n,) * dim
    T = PL.storage_dtype(precision)
    a = 0.05
    f_s = dev(random_populations(lat.Q, shape, seed=11, scale=1e-3), T)
    h_s = dev(random_moments(dim, shape, seed=12, scale=1e-4), T)
    dm_s = dev(random_moments(dim, shape, seed=13, scale=1e-4), T)
    f_out, pr, ss = PL.sweep(dim, n, precision, a, f_s, h_s, dm_s)
    torch.cuda.synchronize()
    size = 8 if dim == 2 else 4
    last = n - size
    picks = [0, last, 29, 30 * (n // 30) - 3, n // 2 - 1] if dim == 2 else [0, last, 28, 5, n // 2 - 2]
    corners = [(picks[i], picks[(i + 1) % len(picks)], picks[(i + 2) % len(picks)]) for i in range(len(picks))]
    tol = TOL[precision]
    for c in corners:
        starts = c[:dim]
        f_w = _periodic_window(f_s, starts, size)
        trial = f_w + OK.linear_lift(lat, _periodic_window(dm_s, starts, size))
        f_T = OSW.sweep(lat, trial, a, _periodic_window(h_s, starts, size))
        inner = (slice(None),) + (slice(1, -1),) * dim
        r = (f_T - trial)[inner]
        assert rel_l2(_periodic_window(f_out, starts, size)[inner], f_T[inner]) < tol["f"]
        assert rel_l2(_periodic_window(pr, starts, size)[inner], OK.moments(lat, r)) < tol["pr"]
    # sum r^2 against the outputs' residual, r = f_out - (f + E dm), formed in FP64 on the device
    w = torch.as_tensor(lat.w, dtype=torch.float64, device="cuda")
    c = torch.as_tensor(lat.c, dtype=torch.float64, device="cuda")
    ssq = 0.0
    for k in range(lat.Q):
        lift = w[k] * (dm_s[0].double() + 3.0 * sum(c[k, al] * dm_s[1 + al].double() for al in range(dim)))
        ssq += float(((f_out[k].double() - f_s[k].double() - lift) ** 2).sum())
    assert abs(float(ss.item()) / ssq - 1) < tol["ss"]


@pytest.mark.parametrize("dim,n,precision", [(2, 4096, "fp32"), (2, 2048, "fp64"), (3, 256, "fp32"),
                                             (3, 128, "fp64")])
def test_shadow_solve_at_the_largest_sizes_single_modes(dim, n, precision):
    # The shadow solve is linear and diagonal in k (Eqs. shadow-update, schur): a cosine mode in
    # moment field q comes back as Re(H(k)^{-1} e_q e^{ik.x}) inside the mask (|j_alpha| <= N/4,
    # the edge included) and as zero outside it; checked on the whole field at the largest lattices
    PL = _lib()
    a, nu = 3.0 / (2 * 64.0), 1.0 / 6.0
    T = PL.storage_dtype(precision)
    q4 = n // 4
    if dim == 2:
        modes = [((3, -5), 0), ((q4, q4), 1), ((-q4, 7), 2), ((0, 0), 0), ((q4 + 1, 2), 1), ((1, -q4 - 3), 2)]
    else:
        modes = [((1, 2, -3), 0), ((q4, 0, -q4), 3), ((0, q4, 5), 1), ((0, 0, 0), 2), ((q4 + 1, 0, 0), 1),
                 ((2, 1, q4 + 2), 3)]
    grids = np.meshgrid(*([np.arange(n, dtype=np.int64)] * dim), indexing="ij")  # (z,) y, x
    tol = 1e-12 if precision == "fp64" else 5e-6  # binary32 transforms of 2 x 12 radix-2 levels
    for j, q in modes:
        # phase 2 pi (j . x) / N with the integer part reduced exactly; j[alpha] pairs with grid axis d-1-alpha
        iph = sum(j[al] * grids[dim - 1 - al] for al in range(dim)) % n
        ph = iph.astype(np.float64) * (2 * np.pi / n)
        pr = torch.zeros((dim + 1,) + (n,) * dim, dtype=T, device="cuda")
        pr[q] = torch.as_tensor(np.cos(ph), device="cuda").to(T)
        dm = PL.shadow_solve(dim, n, precision, a, nu, pr)
        torch.cuda.synchronize()
        dm = host(dm)
        inside = all(abs(v) <= q4 for v in j)
        if not inside:
            assert np.max(np.abs(dm)) < tol / a
            continue
        e = np.zeros(dim + 1)
        e[q] = 1.0
        kvec = [2 * np.pi * j[al] / n for al in range(dim)]
        dp, du = OS.schur_solve(np.complex128(e[0]), e[1:].astype(np.complex128), kvec, a, nu)
        sol = [dp] + [du[al] for al in range(dim)]
        z = np.exp(1j * ph)
        ref = np.stack([np.real(sol[c] * z) for c in range(dim + 1)])
        del z
        assert rel_l2(dm, ref) < tol


def _pair(h64):
    """Binary32 pair (hi, lo) of an FP64 field: hi = RN(h), lo = RN(h - hi); hi + lo is exact in FP64."""
    hi = h64.astype(np.float32)
    lo = (h64 - hi.astype(np.float64)).astype(np.float32)
    return hi, lo


@pytest.mark.parametrize("n,lift", [(8, True), (64, False), (256, True), (1024, True)])
def test_sweep_hpair_matches_oracle(n, lift):
    # the FP32 march's sweep (history term as a binary32 pair) against the oracle fed h = hi + lo
    PL = _lib()
    lat = lattice_for_dim(2)
    f = random_populations(9, (n, n), seed=31, scale=1e-3).astype(np.float32)
    h64 = random_moments(2, (n, n), seed=32, scale=1e-4)
    dm = random_moments(2, (n, n), seed=33, scale=1e-4).astype(np.float32) if lift else None
    hi, lo = _pair(h64)
    a = 0.05
    f_out, pr, ss = PL.sweep_hpair(n, "fp32", a, dev(f, torch.float32), dev(np.stack([hi, lo]), torch.float32),
                                   dev(dm, torch.float32) if lift else None)
    trial = f.astype(np.float64) + (OK.linear_lift(lat, dm.astype(np.float64)) if lift else 0.0)
    f_T = OSW.sweep(lat, trial, a, hi.astype(np.float64) + lo.astype(np.float64))
    r, _ = OSW.residual(f_T, trial)
    assert rel_l2(host(f_out), f_T) < TOL["fp32"]["f"]
    assert rel_l2(host(pr), OK.moments(lat, r)) < TOL["fp32"]["pr"]
    assert abs(float(ss.item()) / float(np.sum(r * r)) - 1) < TOL["fp32"]["ss"]
    # caller-given outputs (the bench's timed loop): the same values, written in place
    out = (torch.full_like(f_out, float("nan")), torch.full_like(pr, float("nan")), torch.zeros_like(ss))
    res = PL.sweep_hpair(n, "fp32", a, dev(f, torch.float32), dev(np.stack([hi, lo]), torch.float32),
                         dev(dm, torch.float32) if lift else None, out=out)
    assert all(x is y for x, y in zip(res, out))
    assert torch.equal(out[0], f_out) and torch.equal(out[1], pr) and torch.equal(out[2], ss)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("n,lift", [(8, True), (16, False), (32, True), (64, True)])
def test_sweep_d3q19_halo_free_matches_oracle(n, lift, precision):
    # the march's D3Q19 sweep (moments of the input given, outputs pulled from the neighbours' collision
    # inputs) against the oracle's sweep, and its P f_out against the oracle's moments of f_T
    PL = _lib()
    lat = lattice_for_dim(3)
    T = PL.storage_dtype(precision)
    f = random_populations(19, (n, n, n), seed=41, scale=1e-3)
    h = random_moments(3, (n, n, n), seed=42, scale=1e-4)
    dm = random_moments(3, (n, n, n), seed=43, scale=1e-4) if lift else None
    f_s = dev(f, T)
    if precision == "fp32":  # the FP32 march's history pair; the oracle sees h = hi + lo exactly
        hi, lo = _pair(h)
        h_s = dev(np.stack([hi, lo]), T)
        h_o = hi.astype(np.float64) + lo.astype(np.float64)
    else:
        h_s = dev(h, T)
        h_o = h
    dm_s = dev(dm, T) if lift else None
    pf_s = dev(OK.moments(lat, host(f_s)), T)
    a = 0.05
    f_out, pf_out, pr, ss = PL.sweep_d3q19_pf(n, precision, a, f_s, pf_s, h_s, dm_s)
    out = tuple(torch.empty_like(t) for t in (f_out, pf_out, pr, ss))
    PL.sweep_d3q19_pf(n, precision, a, f_s, pf_s, h_s, dm_s, out=out)
    assert all(torch.equal(x, y) for x, y in zip(out, (f_out, pf_out, pr, ss)))
    trial = host(f_s) + (OK.linear_lift(lat, host(dm_s)) if lift else 0.0)
    f_T = OSW.sweep(lat, trial, a, h_o)
    r, _ = OSW.residual(f_T, trial)
    tol = TOL[precision]
    assert rel_l2(host(f_out), f_T) < tol["f"]
    assert rel_l2(host(pr), OK.moments(lat, r)) < tol["pr"]
    assert rel_l2(host(pf_out), OK.moments(lat, f_T)) < tol["pr"]
    assert abs(float(ss.item()) / float(np.sum(r * r)) - 1) < tol["ss"]
