"""Oracle pins: the linearised symbol of a sweep and of one corrected iteration (Section 2.4)."""
import numpy as np
import pytest

from oracle import kinetics as K
from oracle import linear as L
from oracle.lattice import D2Q9, D3Q19
from oracle.shadow import shadow_correction
from oracle.sweep import residual, sweep


@pytest.mark.parametrize("lat", [D2Q9, D3Q19], ids=lambda l: l.name)
def test_zero_mode_scale(lat):
    # Eq. zero-mode-scale: P [I - T'(0)] E = (1 - gamma_q) I = a/(1 + a/2) I
    a = 0.13
    T0 = L.sweep_symbol(lat, np.zeros(lat.d), a)
    M = K.moment_matrix(lat) @ (np.eye(lat.Q) - T0) @ K.lift_matrix(lat)
    assert np.allclose(M, a / (1 + a / 2) * np.eye(lat.d + 1), atol=1e-15)
    assert np.isclose(1 - L.gamma(a), a / (1 + a / 2))


def test_slow_rate_value_quoted_in_the_paper():
    # Section 4.3: N = 128, dt = 38.9 gives a Picard tail factor gamma_dt = 0.9622 (Eq. slowrate)
    assert abs(L.gamma(3.0 / (2 * 38.9)) - 0.9622) < 5e-5


def _single_mode(lat, shape, jvec, v, amp):
    """amp * Re(v e^{ik.x}) on the grid; jvec = integer wavevector (x first)."""
    d = lat.d
    grids = np.meshgrid(*(np.arange(n) for n in shape), indexing="ij")
    phase = sum(2 * np.pi * jvec[a] * grids[d - 1 - a] / shape[d - 1 - a] for a in range(d))
    return amp * np.real(v[(slice(None),) + (None,) * d] * np.exp(1j * phase)[None])


@pytest.mark.parametrize("lat,shape,jvec", [(D2Q9, (16, 16), (2, -1)), (D2Q9, (16, 16), (4, 3)),
                                            (D3Q19, (16, 8, 16), (1, -1, 2))],
                         ids=["d2-inner", "d2-mask-edge", "d3"])
@pytest.mark.parametrize("corrected", [False, True], ids=["picard", "msc"])
def test_symbol_predicts_one_nonlinear_iteration(lat, shape, jvec, corrected):
    # About rest with h = 0 a 1e-8 single mode along an eigenvector of the symbol must come
    # back multiplied by the eigenvalue after one oracle iteration (Eqs. symbol, shadow-update).
    d = lat.d
    a, nu = 3.0 / (2 * 20.0), 1.0 / 6.0
    kvec = np.array([2 * np.pi * jvec[i] / shape[d - 1 - i] for i in range(d)])
    G = L.corrected_symbol(lat, kvec, a, nu) if corrected else L.sweep_symbol(lat, kvec, a)
    lam, V = np.linalg.eig(G)
    i = int(np.argmax(np.abs(lam)))
    amp = 1e-8
    f0 = _single_mode(lat, shape, jvec, V[:, i], amp)
    h = np.zeros((d + 1,) + shape)
    f_T = sweep(lat, f0, a, h)
    f1 = f_T
    if corrected:
        r, _ = residual(f_T, f0)
        f1 = f_T + shadow_correction(lat, r, a, nu)[1]
    expect = _single_mode(lat, shape, jvec, lam[i] * V[:, i], amp)
    assert np.linalg.norm(f1 - expect) / np.linalg.norm(expect) < 1e-6
    # a corrected iteration contracts a long-wave mode far more than Picard does (near the
    # mask edge the shadow closure no longer helps: the mask is a design choice, Eq. shadow-mask)
    if corrected and max(abs(j) for j in jvec) <= 2:
        rho_p = L.spectral_radius(L.sweep_symbol(lat, kvec, a))
        assert abs(lam[i]) < 0.7 * rho_p
