"""Seeded input generators: shapes, spectra, divergence, pressure consistency."""
import numpy as np
import pytest

from workloads.fields import poisson_pressure, random_phase, tgv2d, tgv3d, velocity_scale
from workloads.metrics import nint, rel_l2, rms_vector


def spectral_div(u):
    d = u.shape[0]
    N = u.shape[1]
    k1 = 2 * np.pi * np.fft.fftfreq(N)
    K = np.meshgrid(*(k1,) * d, indexing="ij")
    return np.real(np.fft.ifftn(sum(1j * K[d - 1 - a] * np.fft.fftn(u[a]) for a in range(d))))


def test_tgv_pressure_is_the_poisson_pressure():
    # Eq. tgv2d-pressure-init is the incompressible pressure of the Taylor-Green velocity
    p, u = tgv2d(64, 1.0)
    assert rel_l2(poisson_pressure(u), p) < 1e-12
    assert abs(np.mean(p)) < 1e-18  # zero-mean gauge


@pytest.mark.parametrize("d,N,kmax", [(2, 64, 8), (2, 256, 8), (3, 32, 6)])
def test_random_phase_field(d, N, kmax):
    Re = 1.0
    p, u = random_phase(N, d, Re, seed=1, kmax=kmax)
    assert u.shape == (d,) + (N,) * d and p.shape == (N,) * d
    assert np.isclose(np.sqrt(np.sum(u * u, axis=0)).max(), velocity_scale(N, Re))
    assert np.max(np.abs(spectral_div(u))) < 1e-12 * velocity_scale(N, Re)
    assert abs(np.mean(u)) < 1e-15 and abs(np.mean(p)) < 1e-15
    # band limit: no energy outside 1 <= |j| <= kmax
    spec = np.sum(np.abs(np.fft.fftn(u, axes=tuple(range(1, d + 1)))) ** 2, axis=0)
    j1 = np.fft.fftfreq(N) * N
    J = np.sqrt(sum(g ** 2 for g in np.meshgrid(*(j1,) * d, indexing="ij")))
    assert spec[(J < 1) | (J > kmax)].sum() < 1e-20 * spec.sum()
    # same seed -> same field; different seed -> different field
    assert np.array_equal(random_phase(N, d, Re, seed=1, kmax=kmax)[1], u)
    assert rel_l2(random_phase(N, d, Re, seed=2, kmax=kmax)[1], u) > 0.5


def test_shell_spectrum_slope_2d():
    # shell energy ~ k^-2 (streamfunction amplitude ~ |j|^-5/2)
    N = 128
    _, u = random_phase(N, 2, 1.0, seed=3)
    spec = np.sum(np.abs(np.fft.fft2(u, axes=(1, 2))) ** 2, axis=0)
    j1 = np.fft.fftfreq(N) * N
    jy, jx = np.meshgrid(j1, j1, indexing="ij")
    J = np.sqrt(jx ** 2 + jy ** 2)
    shells = np.array([spec[(J >= s - 0.5) & (J < s + 0.5)].sum() for s in range(2, 8)])
    slope = np.polyfit(np.log(np.arange(2, 8)), np.log(shells), 1)[0]
    assert -2.6 < slope < -1.4


def test_tgv3d_and_helpers():
    p, u = tgv3d(16, 1.0)
    assert np.all(p == 0) and np.all(u[2] == 0)
    assert np.isclose(rms_vector(u), velocity_scale(16, 1.0) / 2 ** 1.5 * np.sqrt(2), rtol=1e-12)
    assert nint(1228.8) == 1229 and nint(2.5) == 3 and nint(0.15 * 256 ** 2) == 9830
