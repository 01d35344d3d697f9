"""Seeded initial macroscopic fields and unit-test inputs.

Arrays are indexed [y, x] in 2D and [z, y, x] in 3D (x fastest); velocity
fields have a leading component axis (u_x, u_y[, u_z]).  Lattice units: unit
spacing, N sites per direction, nu = 1/6 at the operating point, U = Re nu / N
(Section 4.1).  p_hat is the pressure-like variable p'/cs^2 with rho_0 = 1 not
added (zero-mean gauge, Eq. tgv2d-pressure-init).
"""
import numpy as np

CS2 = 1.0 / 3.0


def velocity_scale(N: int, Re: float, nu: float = 1.0 / 6.0) -> float:
    """U = Re nu / N (Section 4.1)."""
    return Re * nu / N


def tgv2d(N: int, Re: float, nu: float = 1.0 / 6.0, t: float = 0.0, rho0: float = 1.0):
    """2D Taylor-Green field at time t (Eq. tgv2d) with p_hat = p'/cs^2 (Eq. tgv2d-pressure-init)."""
    U = velocity_scale(N, Re, nu)
    k0 = 2.0 * np.pi / N
    y, x = np.meshgrid(np.arange(N, dtype=np.float64), np.arange(N, dtype=np.float64), indexing="ij")
    decay = np.exp(-2.0 * nu * k0 * k0 * t)
    ux = -U * np.cos(k0 * x) * np.sin(k0 * y) * decay
    uy = U * np.sin(k0 * x) * np.cos(k0 * y) * decay
    p = -rho0 * U * U / 4.0 * (np.cos(2 * k0 * x) + np.cos(2 * k0 * y)) * np.exp(-4.0 * nu * k0 * k0 * t)
    return p / CS2, np.stack([ux, uy])


def tgv3d(N: int, Re: float, nu: float = 1.0 / 6.0):
    """3D Taylor-Green initial field (Eq. tgv3d-ic), zero initial pressure."""
    U = velocity_scale(N, Re, nu)
    k0 = 2.0 * np.pi / N
    z, y, x = np.meshgrid(*(np.arange(N, dtype=np.float64),) * 3, indexing="ij")
    ux = U * np.sin(k0 * x) * np.cos(k0 * y) * np.cos(k0 * z)
    uy = -U * np.cos(k0 * x) * np.sin(k0 * y) * np.cos(k0 * z)
    uz = np.zeros_like(ux)
    return np.zeros_like(ux), np.stack([ux, uy, uz])


def _fft_k(N: int, d: int):
    """Angular wavenumbers 2 pi j / N on numpy's FFT layout, one array per grid axis."""
    k1 = 2.0 * np.pi * np.fft.fftfreq(N) * 1.0  # fftfreq gives j/N
    return np.meshgrid(*(k1,) * d, indexing="ij")


def _half_space_shell(d: int, kmin: float, kmax: float):
    """Integer vectors j (x first) with kmin <= |j| <= kmax in a fixed half space, fixed order."""
    r = int(np.floor(kmax))
    out = []
    rng1 = range(-r, r + 1)
    if d == 2:
        for jy in rng1:
            for jx in rng1:
                if jy > 0 or (jy == 0 and jx > 0):
                    n = np.hypot(jx, jy)
                    if kmin <= n <= kmax:
                        out.append((jx, jy))
    else:
        for jz in rng1:
            for jy in rng1:
                for jx in rng1:
                    if jz > 0 or (jz == 0 and (jy > 0 or (jy == 0 and jx > 0))):
                        n = np.sqrt(jx * jx + jy * jy + jz * jz)
                        if kmin <= n <= kmax:
                            out.append((jx, jy, jz))
    return out


def poisson_pressure(u: np.ndarray) -> np.ndarray:
    """p_hat = p'/cs^2 with lap p' = -div div (u u), zero mean (incompressible, rho_0 = 1)."""
    d = u.shape[0]
    N = u.shape[1]
    K = _fft_k(N, d)            # K[ax] varies along grid axis ax
    kc = [K[d - 1 - a] for a in range(d)]  # component alpha lives on grid axis d-1-alpha
    k2 = sum(k * k for k in kc)
    rhs = np.zeros(u.shape[1:], dtype=np.complex128)
    for i in range(d):
        for j in range(d):
            rhs += kc[i] * kc[j] * np.fft.fftn(u[i] * u[j])
    with np.errstate(divide="ignore", invalid="ignore"):
        p_hat = np.where(k2 > 0, -rhs / k2, 0.0)
    return np.real(np.fft.ifftn(p_hat)) / CS2


def random_phase(N: int, d: int, Re: float, seed: int, nu: float = 1.0 / 6.0,
                 kmin: float = 1.0, kmax: float = 8.0, with_pressure: bool = True):
    """Seeded divergence-free random-phase velocity, energy spectrum ~ k^-2 on kmin <= |j| <= kmax.

    2D: streamfunction with |psi_hat| ~ |j|^-5/2 and u = (d psi/dy, -d psi/dx).
    3D: random complex vectors projected onto the plane normal to j, |u_hat| ~ |j|^-2.
    Phases (and 3D directions) come from numpy's PCG64 ``default_rng(seed)``,
    drawn over a fixed half space of integer wavevectors so that the same seed
    gives the same large-scale flow at every N.  The field is rescaled so that
    the peak speed max_x |u| equals U = Re nu / N.  The initial pressure is the
    Poisson-consistent incompressible pressure (or zero).
    """
    rng = np.random.default_rng(seed)
    modes = _half_space_shell(d, kmin, kmax)
    shape = (N,) * d
    K = _fft_k(N, d)
    kc = [K[d - 1 - a] for a in range(d)]
    uh = [np.zeros(shape, dtype=np.complex128) for _ in range(d)]
    for jv in modes:
        jv = np.array(jv, dtype=np.float64)
        nrm = np.sqrt(jv @ jv)
        idx = tuple(int(jv[d - 1 - ax]) % N for ax in range(d))     # grid index of +j
        idxm = tuple((-int(jv[d - 1 - ax])) % N for ax in range(d))  # grid index of -j
        if d == 2:
            ph = rng.uniform(0.0, 2.0 * np.pi)
            psi = nrm ** -2.5 * np.exp(1j * ph)
            kx, ky = 2 * np.pi * jv[0] / N, 2 * np.pi * jv[1] / N
            vec = [1j * ky * psi, -1j * kx * psi]
        else:
            a = rng.standard_normal(3) + 1j * rng.standard_normal(3)
            e = jv / nrm
            a = a - (a @ e) * e
            a = a / np.sqrt(np.sum(np.abs(a) ** 2))
            vec = list(nrm ** -2.0 * a)
        for al in range(d):
            uh[al][idx] += vec[al]
            uh[al][idxm] += np.conj(vec[al])
    u = np.stack([np.real(np.fft.ifftn(uh[al])) for al in range(d)])
    speed = np.sqrt(np.sum(u * u, axis=0))
    u *= velocity_scale(N, Re, nu) / speed.max()
    p_hat = poisson_pressure(u) if with_pressure else np.zeros(shape)
    return p_hat, u


def random_populations(Q: int, shape, seed: int, scale: float = 1e-3) -> np.ndarray:
    """Gaussian populations for unit tests of a single sweep (not a physical state)."""
    return np.random.default_rng(seed).standard_normal((Q,) + tuple(shape)) * scale


def random_moments(d: int, shape, seed: int, scale: float = 1e-3) -> np.ndarray:
    """Gaussian (d+1)-component fields (history terms, residual moments) for unit tests."""
    return np.random.default_rng(seed).standard_normal((d + 1,) + tuple(shape)) * scale
