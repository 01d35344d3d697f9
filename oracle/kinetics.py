"""Sitewise kinetic pieces of the sweep (Section 2.2), FP64 oracle.

Test infrastructure.  Array conventions: populations ``f`` have shape
(Q, *grid); hydrodynamic fields ``m`` have shape (d+1, *grid) with m[0] = p_hat
and m[1:] = u (x, y[, z]); the grid is (Ny, Nx) in 2D and (Nz, Ny, Nx) in 3D,
x fastest.

Pins (tests/test_oracle_kinetics.py): quadrature identities of f_eq (Eq. feq),
source moments of Phi (Eq. source-moments-check), P E = I (Eq. linear-lift),
the half-source reconstruction solves m = Pf + s/2 (Eq. macro-reconstruct),
general TRT at omega+ = omega- = 1 equals the operating-point form
(Eq. collision vs Eq. collision-operating) for arbitrary f, and with no source
one collision returns f_eq of the incoming moments.
"""
import numpy as np

from .lattice import CS2, Lattice


def cdot(lat: Lattice, v: np.ndarray) -> np.ndarray:
    """c_k . v for every direction: (d, *grid) -> (Q, *grid)."""
    return np.stack([sum(lat.c[k, a] * v[a] for a in range(lat.d)) for k in range(lat.Q)])


def moments(lat: Lattice, f: np.ndarray) -> np.ndarray:
    """P f = (sum_k f_k, sum_k c_k f_k)   (Eq. moments)."""
    out = [f.sum(axis=0)]
    for a in range(lat.d):
        out.append(sum(lat.c[k, a] * f[k] for k in range(lat.Q)))
    return np.stack(out)


def feq(lat: Lattice, p_hat: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Incompressible He-Luo equilibrium (Eq. feq)."""
    cu = cdot(lat, u)
    uu = sum(u[a] * u[a] for a in range(lat.d))
    return np.stack([lat.w[k] * (p_hat + cu[k] / CS2 + cu[k] ** 2 / (2 * CS2 ** 2) - uu / (2 * CS2))
                     for k in range(lat.Q)])


def bdf_coefficients(q: int, dt: float, m_n: np.ndarray, m_nm1: np.ndarray):
    """(a_q, h_q) of Eq. bdf2: BDF1 (q = 1) or BDF2 (q = 2)."""
    if q == 1:
        return 1.0 / dt, m_n / dt
    if q == 2:
        return 3.0 / (2.0 * dt), (4.0 * m_n - m_nm1) / (2.0 * dt)
    raise ValueError("q must be 1 or 2")


def reconstruct(Pf: np.ndarray, a: float, h: np.ndarray) -> np.ndarray:
    """Half-source reconstruction m = (P f + h/2) / (1 + a/2)   (Eq. macro-reconstruct)."""
    return (Pf + h / 2.0) / (1.0 + a / 2.0)


def source_moments(a: float, h: np.ndarray, m: np.ndarray) -> np.ndarray:
    """s = h - a m   (Eq. source-moments)."""
    return h - a * m


def source_distribution(lat: Lattice, m: np.ndarray, s: np.ndarray) -> np.ndarray:
    """Phi_k = w s0 + w[(c - u)/cs^2 + (c.u) c / cs^4] . s_u   (Eq. source-distribution)."""
    u = m[1:]
    su = s[1:]
    cu = cdot(lat, u)
    csu = cdot(lat, su)
    usu = sum(u[a] * su[a] for a in range(lat.d))
    return np.stack([lat.w[k] * (s[0] + (csu[k] - usu) / CS2 + cu[k] * csu[k] / CS2 ** 2)
                     for k in range(lat.Q)])


def even_odd(lat: Lattice, g: np.ndarray):
    """TRT split g^+- = (g_k +- g_kbar)/2   (Eq. trt)."""
    gb = g[lat.opp]
    return 0.5 * (g + gb), 0.5 * (g - gb)


def collide_trt(lat: Lattice, f: np.ndarray, m: np.ndarray, s: np.ndarray,
                omega_p: float, omega_m: float) -> np.ndarray:
    """General TRT collision with the BDF source (Eq. collision)."""
    fe = feq(lat, m[0], m[1:])
    phi = source_distribution(lat, m, s)
    fp, fm = even_odd(lat, f)
    ep, em = even_odd(lat, fe)
    pp, pm = even_odd(lat, phi)
    return (f - omega_p * (fp - ep) - omega_m * (fm - em)
            + (1.0 - omega_p / 2.0) * pp + (1.0 - omega_m / 2.0) * pm)


def collide_operating(lat: Lattice, m: np.ndarray, s: np.ndarray) -> np.ndarray:
    """Operating-point collision C = f_eq(m) + Phi(m, s)/2   (Eq. collision-operating)."""
    return feq(lat, m[0], m[1:]) + 0.5 * source_distribution(lat, m, s)


def linear_lift(lat: Lattice, dm: np.ndarray) -> np.ndarray:
    """Equilibrium lift delta f_k = w_k (dp + c_k . du / cs^2)   (Eqs. linear-lift, lift)."""
    cdu = cdot(lat, dm[1:])
    return np.stack([lat.w[k] * (dm[0] + cdu[k] / CS2) for k in range(lat.Q)])


def lift_matrix(lat: Lattice) -> np.ndarray:
    """E in R^{Q x (d+1)}: E_k0 = w_k, E_ka = w_k c_ka / cs^2   (Eq. linear-lift)."""
    E = np.zeros((lat.Q, lat.d + 1))
    E[:, 0] = lat.w
    for a in range(lat.d):
        E[:, 1 + a] = lat.w * lat.c[:, a] / CS2
    return E


def moment_matrix(lat: Lattice) -> np.ndarray:
    """P in R^{(d+1) x Q}: P_0k = 1, P_ak = c_ka   (Eq. moments)."""
    P = np.zeros((lat.d + 1, lat.Q))
    P[0, :] = 1.0
    for a in range(lat.d):
        P[1 + a, :] = lat.c[:, a]
    return P
