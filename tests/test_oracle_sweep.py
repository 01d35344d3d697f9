"""Oracle pins: streaming, the sweep T and the raw residual (Eqs. sweep, residual)."""
import numpy as np
import pytest

from oracle import kinetics as K
from oracle.lattice import D2Q9, D3Q19
from oracle.linear import gamma
from oracle.sweep import explicit_step, residual, stream, sweep
from workloads.fields import random_moments, random_populations

LATS = [D2Q9, D3Q19]
SHAPES = {2: (8, 4), 3: (4, 8, 4)}


@pytest.mark.parametrize("lat", LATS, ids=lambda l: l.name)
def test_push_streaming_moves_to_x_plus_c(lat):
    # (S g)_k(x + c_k) = g_k(x): a one-hot population at site x0 lands at x0 + c_k (periodic)
    shape = SHAPES[lat.d]
    x0 = tuple(n - 1 for n in shape)  # a corner, so every direction wraps in some axis
    g = np.zeros((lat.Q,) + shape)
    for k in range(lat.Q):
        g[(k,) + x0] = 1.0 + k
    out = stream(lat, g)
    for k in range(lat.Q):
        # grid axis ax holds coordinate alpha = d-1-ax
        dest = tuple((x0[ax] + lat.c[k, lat.d - 1 - ax]) % shape[ax] for ax in range(lat.d))
        assert out[(k,) + dest] == 1.0 + k
        assert np.count_nonzero(out[k]) == 1


@pytest.mark.parametrize("lat", LATS, ids=lambda l: l.name)
def test_sweep_global_balance(lat):
    # sum_x P T(f) = sum_x (P f + s): streaming conserves sums, P f_eq = m, P Phi = s, m = Pf + s/2
    shape = SHAPES[lat.d]
    f = random_populations(lat.Q, shape, seed=11, scale=1e-2)
    h = random_moments(lat.d, shape, seed=12, scale=1e-3)
    a = 0.31
    f_T = sweep(lat, f, a, h)
    Pf = K.moments(lat, f)
    m = K.reconstruct(Pf, a, h)
    s = K.source_moments(a, h, m)
    lhs = K.moments(lat, f_T).reshape(lat.d + 1, -1).sum(axis=1)
    rhs = (Pf + s).reshape(lat.d + 1, -1).sum(axis=1)
    assert np.allclose(lhs, rhs, rtol=0, atol=1e-15)


@pytest.mark.parametrize("lat", LATS, ids=lambda l: l.name)
def test_mean_moment_map_is_affine_with_slope_gamma(lat):
    # For any nonlinear field the domain-mean moments map as M -> gamma_q M + mean(h)/(1 + a/2)
    # (Eqs. local-linear-response, zero-mode-scale): so Picard contracts the mean error by gamma_q.
    shape = SHAPES[lat.d]
    h = random_moments(lat.d, shape, seed=13, scale=1e-3)
    a = 0.05
    f = random_populations(lat.Q, shape, seed=14, scale=1e-2)
    mean = lambda g: K.moments(lat, g).reshape(lat.d + 1, -1).mean(axis=1)
    M0 = mean(f)
    M1 = mean(sweep(lat, f, a, h))
    hbar = h.reshape(lat.d + 1, -1).mean(axis=1)
    assert np.allclose(M1, gamma(a) * M0 + hbar / (1 + a / 2), rtol=0, atol=1e-16)
    # and the fixed point of that map is mean(h)/a (zero mean source)
    Mstar = hbar / a
    fstar = f + K.linear_lift(lat, (Mstar - M0)[(slice(None),) + (None,) * lat.d] * np.ones(shape))
    assert np.allclose(mean(sweep(lat, fstar, a, h)), Mstar, rtol=1e-12, atol=0)


@pytest.mark.parametrize("lat", LATS, ids=lambda l: l.name)
def test_ghost_error_removed_in_one_sweep(lat):
    # Section 2.4.1: with P df = 0 the perturbation vanishes after collision at omega = 1
    shape = SHAPES[lat.d]
    h = random_moments(lat.d, shape, seed=15, scale=1e-3)
    f = random_populations(lat.Q, shape, seed=16, scale=1e-2)
    g = random_populations(lat.Q, shape, seed=17, scale=1e-3)
    E, P = K.lift_matrix(lat), K.moment_matrix(lat)
    ghost = g - np.tensordot(E @ P, g, axes=([1], [0]))  # (I - EP) g has zero moments
    assert np.allclose(K.moments(lat, ghost), 0.0, atol=1e-17)
    a = 0.4
    assert np.allclose(sweep(lat, f + ghost, a, h), sweep(lat, f, a, h), atol=1e-17)
    # ...but the general TRT collision off the operating point keeps part of it
    assert np.max(np.abs(sweep(lat, f + ghost, a, h, omega=(0.7, 1.4)) -
                         sweep(lat, f, a, h, omega=(0.7, 1.4)))) > 1e-5


@pytest.mark.parametrize("lat", LATS, ids=lambda l: l.name)
def test_residual_rms_definition(lat):
    shape = SHAPES[lat.d]
    f = random_populations(lat.Q, shape, seed=18)
    g = random_populations(lat.Q, shape, seed=19)
    r, R = residual(g, f)
    n = lat.Q * int(np.prod(shape))
    assert np.isclose(R, np.sqrt(sum(float(v) ** 2 for v in (g - f).ravel()) / n), rtol=1e-14)


@pytest.mark.parametrize("lat", LATS, ids=lambda l: l.name)
def test_explicit_step_conserves_mass_and_momentum(lat):
    shape = SHAPES[lat.d]
    f = random_populations(lat.Q, shape, seed=20, scale=1e-2)
    f2 = explicit_step(lat, f)
    s = lambda g: K.moments(lat, g).reshape(lat.d + 1, -1).sum(axis=1)
    assert np.allclose(s(f2), s(f), rtol=0, atol=1e-15)
    # and it is f_eq of the moments, streamed
    Pf = K.moments(lat, f)
    assert np.allclose(f2, stream(lat, K.feq(lat, Pf[0], Pf[1:])), atol=1e-18)
