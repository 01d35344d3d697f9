"""Oracle pins: lattice tables and the sitewise kinetic pieces (Section 2.2)."""
import numpy as np
import pytest

from oracle import kinetics as K
from oracle.lattice import CS2, D2Q9, D3Q19
from workloads.fields import random_moments, random_populations

LATS = [D2Q9, D3Q19]
SHAPES = {2: (6, 5), 3: (3, 4, 5)}


@pytest.mark.parametrize("lat", LATS, ids=lambda l: l.name)
def test_lattice_quadrature(lat):
    # sum w = 1, sum w c = 0, sum w c_a c_b = cs^2 delta_ab, opposite table reverses c
    assert np.isclose(lat.w.sum(), 1.0, atol=1e-15)
    assert np.allclose(lat.w @ lat.c, 0.0, atol=1e-15)
    cc = np.einsum("k,ka,kb->ab", lat.w, lat.c, lat.c)
    assert np.allclose(cc, CS2 * np.eye(lat.d), atol=1e-15)
    assert np.array_equal(lat.c[lat.opp], -lat.c)
    assert lat.Q == {2: 9, 3: 19}[lat.d]


@pytest.mark.parametrize("lat", LATS, ids=lambda l: l.name)
def test_feq_carries_the_hydrodynamic_moments(lat):
    # Eq. feq: sum_k f_eq = p_hat and sum_k c_k f_eq = u, for any (p_hat, u)
    m = random_moments(lat.d, SHAPES[lat.d], seed=1, scale=0.05)
    fe = K.feq(lat, m[0], m[1:])
    assert np.allclose(K.moments(lat, fe), m, rtol=0, atol=1e-15)


@pytest.mark.parametrize("lat", LATS, ids=lambda l: l.name)
def test_source_distribution_moments(lat):
    # Eq. source-moments-check: sum Phi = s0, sum c Phi = s_u
    m = random_moments(lat.d, SHAPES[lat.d], seed=2, scale=0.05)
    s = random_moments(lat.d, SHAPES[lat.d], seed=3, scale=0.01)
    phi = K.source_distribution(lat, m, s)
    assert np.allclose(K.moments(lat, phi), s, rtol=0, atol=1e-16)


@pytest.mark.parametrize("lat", LATS, ids=lambda l: l.name)
def test_lift_is_right_inverse_of_moments(lat):
    # Eq. linear-lift: P E = I, and the lift function equals E applied sitewise
    E = K.lift_matrix(lat)
    P = K.moment_matrix(lat)
    assert np.allclose(P @ E, np.eye(lat.d + 1), atol=1e-15)
    dm = random_moments(lat.d, SHAPES[lat.d], seed=4)
    df = K.linear_lift(lat, dm)
    assert np.allclose(np.tensordot(E, dm, axes=([1], [0])), df, atol=1e-18)
    # E is the derivative of f_eq at rest: f_eq(eps dm) / eps -> E dm
    e = 1e-7
    fe = K.feq(lat, e * dm[0], e * dm[1:]) / e
    assert np.allclose(fe, df, atol=1e-9)


def test_bdf_coefficients():
    m_n, m_nm1 = np.array([1.0]), np.array([0.5])
    a1, h1 = K.bdf_coefficients(1, 4.0, m_n, m_nm1)
    a2, h2 = K.bdf_coefficients(2, 4.0, m_n, m_nm1)
    assert a1 == 0.25 and h1[0] == 0.25
    assert a2 == 3.0 / 8.0 and h2[0] == (4.0 - 0.5) / 8.0
    # BDF2 is exact for a linear-in-time field: m(t) = t, D m^{n+1} = 1
    dt = 0.7
    a, h = K.bdf_coefficients(2, dt, np.array([2 * dt]), np.array([dt]))
    assert np.isclose(a * 3 * dt - h[0], 1.0)


@pytest.mark.parametrize("lat", LATS, ids=lambda l: l.name)
def test_reconstruction_solves_half_source_relation(lat):
    # Eq. macro-reconstruct: m = Pf + s/2 with s = h - a m
    f = random_populations(lat.Q, SHAPES[lat.d], seed=5)
    h = random_moments(lat.d, SHAPES[lat.d], seed=6, scale=1e-4)
    a = 0.37
    Pf = K.moments(lat, f)
    m = K.reconstruct(Pf, a, h)
    s = K.source_moments(a, h, m)
    assert np.allclose(m, Pf + s / 2, atol=1e-17)


@pytest.mark.parametrize("lat", LATS, ids=lambda l: l.name)
def test_trt_at_unit_rates_is_operating_point_form(lat):
    # Eq. collision with omega+ = omega- = 1 reduces to Eq. collision-operating for any f
    f = random_populations(lat.Q, SHAPES[lat.d], seed=7, scale=1e-2)
    h = random_moments(lat.d, SHAPES[lat.d], seed=8, scale=1e-3)
    a = 0.2
    m = K.reconstruct(K.moments(lat, f), a, h)
    s = K.source_moments(a, h, m)
    c_trt = K.collide_trt(lat, f, m, s, 1.0, 1.0)
    c_op = K.collide_operating(lat, m, s)
    # the paper's bound for this comparison after one step is 2e-14 (Section 4.1)
    assert np.max(np.abs(c_trt - c_op)) < 2e-14


@pytest.mark.parametrize("lat", LATS, ids=lambda l: l.name)
def test_unit_rate_collision_without_source_returns_equilibrium(lat):
    # one omega = 1 collision with no source maps f to f_eq of its own moments,
    # whatever the nonequilibrium content of f
    f = random_populations(lat.Q, SHAPES[lat.d], seed=9, scale=1e-2)
    zero = np.zeros((lat.d + 1,) + SHAPES[lat.d])
    m = K.reconstruct(K.moments(lat, f), 0.0, zero)
    c = K.collide_trt(lat, f, m, K.source_moments(0.0, zero, m), 1.0, 1.0)
    Pf = K.moments(lat, f)
    assert np.allclose(c, K.feq(lat, Pf[0], Pf[1:]), atol=1e-17)
    # the collision conserves the moments when there is no source
    assert np.allclose(K.moments(lat, c), Pf, atol=1e-17)
    # off the operating point the nonequilibrium part survives (Eq. eta): TRT differs from f_eq
    c2 = K.collide_trt(lat, f, m, K.source_moments(0.0, zero, m), 0.8, 1.3)
    assert np.max(np.abs(c2 - c)) > 1e-4
