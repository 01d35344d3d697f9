"""Continuum reference for the random-phase workloads: dealiased pseudo-spectral incompressible
Navier-Stokes on the same periodic box (length N lattice units), integrating-factor RK4 in time.

The random-phase fields have no closed form, so the accuracy gates compare both the explicit
LBM and MSC-LBM against this solution (as the Taylor-Green closed form does for config 1).  It is
an independent solver of the macroscopic equations, not a restatement of the lattice method.

2D uses the vorticity form, 3D the rotational velocity form with the Leray projection; both use
the 2/3 rule on an M^d grid (M >= 4 kmax so the initial band and its first products are resolved)
and evaluate the velocity at the N^d lattice points by zero-padded spectral interpolation.
"""
import numpy as np


def _k(M: int, N: int, d: int):
    k1 = 2.0 * np.pi * np.fft.fftfreq(M, d=1.0 / M) / N  # angular wavenumbers of the box of length N
    K = np.meshgrid(*(k1,) * d, indexing="ij")
    kc = [K[d - 1 - a] for a in range(d)]  # component alpha on grid axis d-1-alpha
    j1 = np.abs(np.fft.fftfreq(M, d=1.0 / M))
    J = np.meshgrid(*(j1,) * d, indexing="ij")
    dealias = np.ones((M,) * d, dtype=bool)
    for ax in range(d):
        dealias &= J[ax] < M / 3.0
    return kc, dealias


def _to_coarse(field_N: np.ndarray, M: int) -> np.ndarray:
    """Normalised Fourier coefficients c(j) (field = sum c e^{ik.x}) restricted to the M grid."""
    N = field_N.shape[0]
    d = field_N.ndim
    c = np.fft.fftn(field_N) / N ** d
    idx = np.fft.fftfreq(M, d=1.0 / M).astype(int)
    return c[np.ix_(*([np.mod(idx, N)] * d))]


def _to_lattice(c: np.ndarray, N: int) -> np.ndarray:
    """Evaluate sum_j c(j) e^{ik.x} at the N^d lattice points (zero padding)."""
    M = c.shape[0]
    d = c.ndim
    idx = np.fft.fftfreq(M, d=1.0 / M).astype(int)
    full = np.zeros((N,) * d, dtype=np.complex128)
    full[np.ix_(*([np.mod(idx, N)] * d))] = c
    return np.real(np.fft.ifftn(full)) * N ** d


def _phys(c):
    return np.real(np.fft.ifftn(c)) * c.size


def _coef(f):
    return np.fft.fftn(f) / f.size


def navier_stokes_reference(u0: np.ndarray, nu: float, t_end: float, M: int = 128, n_steps: int = None):
    """Velocity at time t_end on the lattice points, from the lattice initial velocity u0."""
    d = u0.shape[0]
    N = u0.shape[1]
    kc, dealias = _k(M, N, d)
    k2 = sum(k * k for k in kc)
    k2_safe = np.where(k2 == 0, 1.0, k2)
    uc = [_to_coarse(u0[a], M) for a in range(d)]
    U = max(np.abs(u0).max(), 1e-300)
    kmax = 2 * np.pi * (M / 3.0) / N
    if n_steps is None:
        n_steps = max(200, int(np.ceil(t_end * U * kmax / 0.05)))
    dt = t_end / n_steps
    E = np.exp(-nu * k2 * dt / 2.0)
    E2 = E * E

    if d == 2:
        w = 1j * kc[0] * uc[1] - 1j * kc[1] * uc[0]

        def vel(wh):
            psi = wh / k2_safe
            psi = np.where(k2 == 0, 0.0, psi)
            return 1j * kc[1] * psi, -1j * kc[0] * psi

        def nonlin(wh):
            ux, uy = vel(wh)
            wx = _phys(1j * kc[0] * wh)
            wy = _phys(1j * kc[1] * wh)
            adv = _phys(ux) * wx + _phys(uy) * wy
            return -_coef(adv) * dealias

        for _ in range(n_steps):
            a1 = dt * nonlin(w)
            a2 = dt * nonlin(E * (w + a1 / 2))
            a3 = dt * nonlin(E * w + a2 / 2)
            a4 = dt * nonlin(E2 * w + E * a3)
            w = E2 * w + (E2 * a1 + 2 * E * (a2 + a3) + a4) / 6.0
        ux, uy = vel(w)
        return np.stack([_to_lattice(ux, N), _to_lattice(uy, N)])

    u = np.stack(uc)

    def nonlin3(uh):
        up = [_phys(uh[a]) for a in range(3)]
        wv = [_phys(1j * (kc[1] * uh[2] - kc[2] * uh[1])),
              _phys(1j * (kc[2] * uh[0] - kc[0] * uh[2])),
              _phys(1j * (kc[0] * uh[1] - kc[1] * uh[0]))]
        cr = [up[1] * wv[2] - up[2] * wv[1], up[2] * wv[0] - up[0] * wv[2], up[0] * wv[1] - up[1] * wv[0]]
        ch = np.stack([_coef(c) for c in cr]) * dealias
        kd = sum(kc[a] * ch[a] for a in range(3)) / k2_safe
        return np.stack([ch[a] - kc[a] * kd for a in range(3)])  # Leray projection of u x w

    for _ in range(n_steps):
        a1 = dt * nonlin3(u)
        a2 = dt * nonlin3(E * (u + a1 / 2))
        a3 = dt * nonlin3(E * u + a2 / 2)
        a4 = dt * nonlin3(E2 * u + E * a3)
        u = E2 * u + (E2 * a1 + 2 * E * (a2 + a3) + a4) / 6.0
    return np.stack([_to_lattice(u[a], N) for a in range(3)])
