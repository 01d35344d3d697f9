"""Oracle pins: the linearised symbol of a sweep and of one corrected iteration (Section 2.4)."""
import numpy as np
import pytest

from oracle import fullsymbol as FS
from oracle import kinetics as K
from oracle import linear as L
from oracle import march as M
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


# ---- off the collision operating point (Section 4.6) ----

def _mode_fields(N, jvec, amp):
    """A small single Fourier mode in p_hat and u on an N x N grid (x fastest), zero base state."""
    x = np.arange(N)
    ph = 2 * np.pi * (jvec[0] * x[None, :] + jvec[1] * x[:, None]) / N
    p = amp * np.cos(ph)
    u = np.stack([0.3 * amp * np.sin(ph), -0.7 * amp * np.cos(ph + 0.4)])
    return p, u


@pytest.mark.parametrize("lat", [D2Q9, D3Q19], ids=lambda l: l.name)
def test_off_design_symbols_reduce_to_the_operating_point(lat):
    # at omega+ = omega- = 1 the general TRT collision is the operating-point one (Eq. collision vs
    # Eq. collision-operating), so Z J = gamma Z E P and the corrected symbols coincide
    a, nu = 0.07, 1.0 / 6.0
    for jvec in ([1, -2, 3], [4, 4, 4], [0, 3, -1]):
        k = 2 * np.pi * np.array(jvec[:lat.d]) / 16
        T_off = L.trt_sweep_symbol(lat, k, a, (1.0, 1.0))
        assert np.max(np.abs(T_off - L.sweep_symbol(lat, k, a))) < 1e-14
        G_off = L.trt_corrected_symbol(lat, k, a, nu, (1.0, 1.0))
        assert np.max(np.abs(G_off - L.corrected_symbol(lat, k, a, nu))) < 1e-13


@pytest.mark.parametrize("nu,lam,jvec,diverges", [(0.1, 0.25, (4, 4), True), (0.1, 0.25, (2, 1), True),
                                                  (0.12, 0.25, (4, -4), True), (0.14, 0.25, (4, 0), False),
                                                  (0.2, 0.25, (4, 4), False), (1 / 6, 2.0, (2, 1), False),
                                                  (1 / 6, 1 / 64, (1, -2), False), (0.25, 0.05, (2, 1), False)])
def test_off_design_symbol_predicts_the_march_contraction(nu, lam, jvec, diverges):
    # The linear Fourier analysis of Section 4.6: a 1e-12 single mode marched by the nonlinear oracle
    # (one BDF1 step, general TRT sweep, shadow correction, no acceptance) shrinks or grows by the
    # spectral radius of G(k) per inner iteration, at wavevectors that converge (rho < 1) and that
    # diverge below the threshold viscosity (rho > 1); the cases have the largest eigenvalue at least
    # 1/0.8 times the next distinct one, so that ten ratios settle on it
    N, dt = 16, 20.0
    omega = FS.trt_rates(nu, lam)
    k = 2 * np.pi * np.array(jvec) / N
    rho = L.spectral_radius(L.trt_corrected_symbol(D2Q9, k, 1.0 / dt, nu, omega))
    # amplitude 1e-12 and 60 iterations: a growing mode stays below 1e-3, a shrinking one (rho >= 0.6)
    # above both rounding and the second harmonic that the quadratic terms make (amplitude^2)
    p, u = _mode_fields(N, jvec, 1e-12)
    st = M.init_state(D2Q9, p, u)
    rec = M.physical_step(st, M.MarchParams(dt=dt, nu=nu, eps=0.0, kmax=60, omega=omega))
    assert not rec.converged and len(rec.residuals) == 60
    assert abs(M.rho_observed(rec.residuals, 10) / rho - 1) < 1e-4
    assert (rho > 1) == diverges


@pytest.mark.parametrize("a", [3 / (2 * 38.4), 0.625], ids=["a-small", "a-large"])
def test_off_design_envelope(a):
    # Section 4.6: along the Lambda axis at nu = 1/6 the shadow correction loses contraction but does
    # not diverge; along the nu axis at Lambda = 1/4 its worst masked mode grows as nu falls and
    # passes 1 (divergence), at the mask corner |k_x| = |k_y| = pi/2
    N = 16
    r0, _ = L.masked_spectral_radius(D2Q9, N, a, 1.0 / 6.0, (1.0, 1.0))
    r_lam = [L.masked_spectral_radius(D2Q9, N, a, 1.0 / 6.0, FS.trt_rates(1.0 / 6.0, lam))[0]
             for lam in (1 / 64, 0.05, 0.5, 2.0, 4.0)]
    assert r0 < 0.8 and all(r < 1.0 for r in r_lam) and max(r_lam) > r0 + 0.15
    prev = r0
    for nu in (0.14, 0.12, 0.10, 0.09, 0.07):
        r, arg = L.masked_spectral_radius(D2Q9, N, a, nu, FS.trt_rates(nu, 0.25))
        assert r > prev
        prev = r
    assert prev > 1.0 and tuple(abs(j) for j in arg) == (N // 4, N // 4)
    # the ghost survival at the paper's threshold viscosity (Eq. eta: eta(0.09) ~ 0.30)
    assert abs(FS.eta(0.09) - 0.30) < 0.005
