"""GPU full-symbol reference correction (Eq. full-symbol) against the FP64 oracle (dense per-wavevector
inverse of I - Z(k) J with the exact rest Jacobian), and the corrected off-design iteration."""
import numpy as np
import pytest
import torch

from oracle import fullsymbol as FS
from oracle import sweep as OSW
from oracle.lattice import D2Q9
from workloads.fields import random_moments, random_populations
from tests.gpu_helpers import dev, host, rel_l2

pytestmark = pytest.mark.gpu
A_BDF2 = 3 / (2 * 20.0)
RATES = [(0.08, 0.25), (0.25, 0.05), (1 / 6, 0.25), (0.12, 2.0)]


def _PL():
    from paper_2609_39474_b300 import lattice as PL
    return PL


def _oracle_df(n, a, wp, wm, r):
    Minv = FS.correction_matrices(D2Q9, FS.rest_jacobian_exact(D2Q9, a, (wp, wm)), (n, n))
    return FS.full_symbol_correction(D2Q9, r, Minv)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("n", [8, 16, 64])
@pytest.mark.parametrize("nu,lam", RATES)
def test_correction_matches_oracle(n, precision, nu, lam):
    PL = _PL()
    wp, wm = FS.trt_rates(nu, lam)
    T = PL.storage_dtype(precision)
    f = dev(random_populations(9, (n, n), seed=1, scale=1e-3), T)
    ft = dev(host(f) + random_populations(9, (n, n), seed=2, scale=1e-5), T)
    out = PL.full_symbol_correct(n, precision, A_BDF2, wp, wm, f, ft)
    torch.cuda.synchronize()
    fh = host(f)
    df_ref = _oracle_df(n, A_BDF2, wp, wm, host(ft) - fh)
    # FP32: the correction is read back as out - f, so f's rounding (1e-3 x 6e-8) is 1e-5 of df
    assert rel_l2(host(out) - fh, df_ref) < (1e-11 if precision == "fp64" else 3e-5)


def test_correction_in_place_and_at_the_largest_size():
    # f_out may alias f; n = 1024 (the bound) runs the large column variant: checked against the
    # oracle on sampled wavevectors through linearity (one Fourier mode in, that mode's column out)
    PL = _PL()
    wp, wm = FS.trt_rates(0.08, 0.25)
    n = 1024
    f = dev(random_populations(9, (n, n), seed=3, scale=1e-3))
    x = np.arange(n)
    for jx, jy, q in ((0, 0, 0), (3, 5, 4), (512, 7, 6), (100, 1000, 8)):
        r = np.zeros((9, n, n))
        r[q] = np.cos(2 * np.pi * (jx * x[None, :] + jy * x[:, None]) / n)
        ft = f + dev(r)
        g = f.clone()
        PL.full_symbol_correct(n, "fp64", A_BDF2, wp, wm, g, ft, out=g)
        torch.cuda.synchronize()
        df = host(g) - host(f)
        # oracle: M(k) for +-k applied to the single mode (real input: the two conjugate modes)
        J = FS.rest_jacobian_exact(D2Q9, A_BDF2, (wp, wm))
        ref = np.zeros((9, n, n))
        for sgn in (1, -1):
            k = 2 * np.pi * np.array([sgn * jx, sgn * jy]) / n
            Z = np.exp(-1j * (D2Q9.c[:, 0] * k[0] + D2Q9.c[:, 1] * k[1]))
            col = np.linalg.solve(np.eye(9) - Z[:, None] * J, np.eye(9)[:, q])
            ref += np.real(col[:, None, None] * 0.5 * np.exp(1j * (k[0] * x[None, :] + k[1] * x[:, None]))[None])
        assert rel_l2(df, ref) < 1e-11


@pytest.mark.parametrize("nu,lam", [(0.08, 0.25), (0.25, 0.05)])
def test_corrected_iteration_matches_oracle(nu, lam):
    # f <- f + full-symbol correction of (T(f) - f) with the GPU TRT sweep, against the same iteration
    # in the oracle; near rest it contracts like a Newton iteration (the shadow correction diverges at
    # nu = 0.08, Section 4.6)
    PL = _PL()
    n, K = 32, 6
    wp, wm = FS.trt_rates(nu, lam)
    f0 = random_populations(9, (n, n), seed=4, scale=1e-3)
    h = random_moments(2, (n, n), seed=5, scale=1e-4)
    f, hd = dev(f0), dev(h)
    R_gpu = []
    for _ in range(K):
        ft, _, ss = PL.sweep_trt(n, "fp64", A_BDF2, wp, wm, f, hd)
        R_gpu.append(float(ss.item()) ** 0.5)
        f = PL.full_symbol_correct(n, "fp64", A_BDF2, wp, wm, f, ft)
    torch.cuda.synchronize()
    Minv = FS.correction_matrices(D2Q9, FS.rest_jacobian_exact(D2Q9, A_BDF2, (wp, wm)), (n, n))
    fo = f0.copy()
    R_ora = []
    for _ in range(K):
        ft = OSW.sweep(D2Q9, fo, A_BDF2, h, omega=(wp, wm))
        r, _ = OSW.residual(ft, fo)
        R_ora.append(float(np.sqrt(np.sum(r * r))))
        fo = fo + FS.full_symbol_correction(D2Q9, r, Minv)
    for rg, ro in zip(R_gpu, R_ora):
        if ro > 1e-8 * R_ora[0]:
            assert abs(rg / ro - 1) < 1e-6
    assert R_gpu[2] / R_gpu[0] < 1e-4
    assert rel_l2(host(f), fo) < 1e-11
