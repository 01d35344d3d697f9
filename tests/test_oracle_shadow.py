"""Oracle pins: DFT convention, mask, Schur solve and lift (Section 3.2)."""
import itertools

import numpy as np
import pytest

from oracle import kinetics as K
from oracle import shadow as SH
from oracle.lattice import D2Q9, D3Q19
from oracle.linear import gamma
from oracle.sweep import residual, sweep
from workloads.fields import random_moments, random_populations


def brute_dft(g, sign):
    """O(N^{2d}) sum over every site and every mode (full spectrum, numpy FFT index layout)."""
    shape = g.shape
    out = np.zeros(shape, dtype=np.complex128)
    for kidx in itertools.product(*(range(n) for n in shape)):
        acc = 0.0 + 0.0j
        for xidx in itertools.product(*(range(n) for n in shape)):
            ph = sum(2 * np.pi * kidx[a] * xidx[a] / shape[a] for a in range(len(shape)))
            acc += g[xidx] * np.exp(sign * 1j * ph)
        out[kidx] = acc
    return out


def masked_view(full):
    """Pick the masked signed indices -N/4..N/4 out of a full numpy-layout spectrum."""
    idx = [np.mod(SH.masked_indices(n), n) for n in full.shape]
    return full[np.ix_(*idx)]


@pytest.mark.parametrize("shape", [(4, 4), (8, 4), (8, 8), (4, 4, 8)])
def test_masked_dft_matches_brute_force(shape):
    g = np.random.default_rng(1).standard_normal(shape)
    got = SH.dft_forward_masked(g)
    ref = masked_view(brute_dft(g, -1))
    assert np.allclose(got, ref, atol=1e-12)


@pytest.mark.parametrize("shape", [(16, 16), (32, 8), (8, 16, 16)])
def test_masked_dft_matches_library_fft(shape):
    g = np.random.default_rng(2).standard_normal(shape)
    got = SH.dft_forward_masked(g)
    assert np.allclose(got, masked_view(np.fft.fftn(g)), atol=1e-11)


@pytest.mark.parametrize("shape", [(16, 16), (8, 8, 8)])
def test_masked_inverse_reproduces_band_limited_field(shape):
    rng = np.random.default_rng(3)
    full = np.fft.fftn(rng.standard_normal(shape))
    keep = np.zeros(shape, dtype=bool)
    keep[np.ix_(*[np.mod(SH.masked_indices(n), n) for n in shape])] = True
    g = np.real(np.fft.ifftn(np.where(keep, full, 0)))  # real, band-limited to the mask
    back = SH.dft_inverse_masked(SH.dft_forward_masked(g), shape)
    assert np.max(np.abs(back.imag)) < 1e-13
    assert np.allclose(back.real, g, atol=1e-13)
    # the inverse convention carries 1/N_Omega: a constant spectrum value c at k=0 gives c/N_Omega
    spec = np.zeros(tuple(len(SH.masked_indices(n)) for n in shape), dtype=np.complex128)
    spec[tuple(len(SH.masked_indices(n)) // 2 for n in shape)] = 7.0
    assert np.allclose(SH.dft_inverse_masked(spec, shape).real, 7.0 / np.prod(shape))


def test_mask_keeps_the_boundary_and_drops_beyond():
    J = SH.masked_indices(16)
    k = SH.wavenumber(J, 16)
    assert J[0] == -4 and J[-1] == 4 and len(J) == 9
    assert np.isclose(np.max(np.abs(k)), np.pi / 2)  # |k| = pi/2 is retained (Eq. shadow-mask)


@pytest.mark.parametrize("d", [2, 3])
def test_schur_matches_dense_solve(d):
    rng = np.random.default_rng(4)
    a, nu = 0.07, 1.0 / 6.0
    for _ in range(20):
        kv = rng.uniform(-np.pi / 2, np.pi / 2, size=d)
        r = rng.standard_normal(d + 1) + 1j * rng.standard_normal(d + 1)
        dp, du = SH.schur_solve(np.array(r[0]), r[1:].reshape(d, 1), [np.array([kv[i]]) for i in range(d)], a, nu)
        ref = np.linalg.solve(SH.shadow_matrix(kv, a, nu), r)
        assert np.allclose(np.concatenate([np.atleast_1d(dp), du.ravel()]), ref, rtol=1e-12, atol=0)


@pytest.mark.parametrize("lat", [D2Q9, D3Q19], ids=lambda l: l.name)
def test_zero_residual_gives_zero_correction(lat):
    shape = (8,) * lat.d
    dm, df = SH.shadow_correction(lat, np.zeros((lat.Q,) + shape), 0.1, 1.0 / 6.0)
    assert np.all(dm == 0.0) and np.all(df == 0.0)


@pytest.mark.parametrize("lat", [D2Q9, D3Q19], ids=lambda l: l.name)
def test_one_corrected_iteration_scales_mean_error_by_minus_half_one_minus_gamma(lat):
    # k = 0: H(0) = a I, while the sweep moves the mean by (gamma - 1) (M - M*); one MSC
    # iteration therefore multiplies the mean-moment error by gamma + (gamma - 1)/a = -(1 - gamma)/2.
    shape = (8,) * lat.d
    a = 0.09
    h = random_moments(lat.d, shape, seed=5, scale=1e-3)
    f = random_populations(lat.Q, shape, seed=6, scale=1e-2)
    mean = lambda g: K.moments(lat, g).reshape(lat.d + 1, -1).mean(axis=1)
    Mstar = h.reshape(lat.d + 1, -1).mean(axis=1) / a
    f_T = sweep(lat, f, a, h)
    r, _ = residual(f_T, f)
    _, df = SH.shadow_correction(lat, r, a, 1.0 / 6.0)
    err0 = mean(f) - Mstar
    err1 = mean(f_T + df) - Mstar
    assert np.allclose(err1, -(1 - gamma(a)) / 2 * err0, rtol=1e-9, atol=0)
