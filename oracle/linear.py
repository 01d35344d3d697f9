"""Linearised Fourier symbol of one sweep and of one corrected iteration (Section 2.4), FP64.

Test infrastructure.  About the uniform rest state with zero base source and
omega+ = omega- = 1, one sweep acts on a Fourier mode e^{ik.x} through
T'(k) = gamma_q Z(k) E P with Z(k) = diag(e^{-ik.c_k}) (Eqs.
local-linear-response, symbol).  One MSC iteration f <- f_T + E H^{-1} P r
(Eq. shadow-update, inside the mask) linearises to
G(k) = T'(k) + E H(k)^{-1} P (T'(k) - I).

Pins (tests/test_oracle_linear.py): gamma_q against Eq. zero-mode-scale
(P[I - T'(0)]E = (1 - gamma_q) I); the spectral radius of T'(k) and G(k)
against the observed contraction of the nonlinear oracle iteration on a
1e-8-amplitude single mode; ghost perturbations (P df = 0) vanish in one sweep.
"""
import numpy as np

from .kinetics import lift_matrix, moment_matrix
from .lattice import Lattice
from .shadow import shadow_matrix


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
