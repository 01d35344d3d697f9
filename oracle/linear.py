"""Linearised Fourier symbol of one sweep and of one corrected iteration (Section 2.4), FP64.

Test infrastructure.  About the uniform rest state with zero base source and
omega+ = omega- = 1, one sweep acts on a Fourier mode e^{ik.x} through
T'(k) = gamma_q Z(k) E P with Z(k) = diag(e^{-ik.c_k}) (Eqs.
local-linear-response, symbol).  One MSC iteration f <- f_T + E H^{-1} P r
(Eq. shadow-update, inside the mask) linearises to
G(k) = T'(k) + E H(k)^{-1} P (T'(k) - I).

Off the collision operating point (general TRT collision, Eq. collision;
Section 4.6) the same linearisation holds with gamma_q E P replaced by the
rest Jacobian J of the collision (Eq. full-symbol): T'(k) = Z(k) J, and the
shadow-corrected iteration keeps the form of G(k) with that T'(k).  Its
largest spectral radius over the masked wavevectors says whether the shadow
correction contracts or diverges away from the operating point (the linear
Fourier analysis of Section 4.6).

Pins (tests/test_oracle_linear.py): gamma_q against Eq. zero-mode-scale
(P[I - T'(0)]E = (1 - gamma_q) I); the spectral radius of T'(k) and G(k)
against the observed contraction of the nonlinear oracle iteration on a
1e-8-amplitude single mode; ghost perturbations (P df = 0) vanish in one sweep;
the off-design symbols equal the operating-point ones at omega+ = omega- = 1,
and their spectral radius matches the observed contraction of the nonlinear
oracle march (general TRT sweep, shadow correction) on single modes that
converge and that diverge; the off-design envelope of Section 4.6 (no
divergence along the Lambda axis at nu = 1/6, divergence below a threshold nu
on the nu axis at Lambda = 1/4).
"""
import numpy as np

from .fullsymbol import rest_jacobian_exact
from .kinetics import lift_matrix, moment_matrix
from .lattice import Lattice
from .shadow import masked_indices, shadow_matrix


def gamma(a: float) -> float:
    """gamma_q = (1 - a/2) / (1 + a/2)   (Eq. local-linear-response)."""
    return (1.0 - a / 2.0) / (1.0 + a / 2.0)


def stream_phase(lat: Lattice, kvec) -> np.ndarray:
    """Z(k) = diag(exp(-i k . c_k))   (Eq. symbol)."""
    k = np.asarray(kvec, dtype=np.float64)
    return np.diag(np.exp(-1j * (lat.c.astype(np.float64) @ k)))


def sweep_symbol(lat: Lattice, kvec, a: float) -> np.ndarray:
    """T'(k) = gamma_q Z(k) E P   (Eq. symbol)."""
    return gamma(a) * stream_phase(lat, kvec) @ lift_matrix(lat) @ moment_matrix(lat)


def corrected_symbol(lat: Lattice, kvec, a: float, nu: float) -> np.ndarray:
    """G(k) = T'(k) + E H(k)^{-1} P (T'(k) - I) for a wavevector inside the mask."""
    T = sweep_symbol(lat, kvec, a)
    E = lift_matrix(lat)
    P = moment_matrix(lat)
    H = shadow_matrix(kvec, a, nu)
    return T + E @ np.linalg.solve(H, P @ (T - np.eye(lat.Q)))


def spectral_radius(M: np.ndarray) -> float:
    return float(np.max(np.abs(np.linalg.eigvals(M))))


def trt_sweep_symbol(lat: Lattice, kvec, a: float, omega, J=None) -> np.ndarray:
    """T'(k) = Z(k) J with J the rest Jacobian of the general TRT collision (Eqs. collision,
    full-symbol, symbol); omega = (omega+, omega-).  J may be passed in when it is already formed."""
    if J is None:
        J = rest_jacobian_exact(lat, a, omega)
    return stream_phase(lat, kvec) @ J


def trt_corrected_symbol(lat: Lattice, kvec, a: float, nu: float, omega, J=None) -> np.ndarray:
    """G(k) = T'(k) + E H(k)^{-1} P (T'(k) - I) with the off-design T'(k) of trt_sweep_symbol: one
    shadow-corrected iteration (Eq. shadow-update, H(k) at the viscosity nu of the shadow solve) with
    the general TRT sweep, for a wavevector inside the mask."""
    T = trt_sweep_symbol(lat, kvec, a, omega, J)
    E = lift_matrix(lat)
    P = moment_matrix(lat)
    H = shadow_matrix(kvec, a, nu)
    return T + E @ np.linalg.solve(H, P @ (T - np.eye(lat.Q)))


def masked_spectral_radius(lat: Lattice, N: int, a: float, nu: float, omega):
    """max over the masked wavevectors of an N^d grid (Eq. shadow-mask: |k_alpha| <= pi/2) of the
    spectral radius of trt_corrected_symbol, and the integer wavevector where it is reached."""
    js = masked_indices(N)
    J = rest_jacobian_exact(lat, a, omega)
    best, arg = -1.0, None
    for jvec in np.stack(np.meshgrid(*([js] * lat.d), indexing="ij"), axis=-1).reshape(-1, lat.d):
        r = spectral_radius(trt_corrected_symbol(lat, 2 * np.pi * jvec / N, a, nu, omega, J))
        if r > best:
            best, arg = r, tuple(int(j) for j in jvec)
    return best, arg
