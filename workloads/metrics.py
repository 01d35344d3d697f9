"""Error metrics and accuracy gates (Section 4.1)."""
import numpy as np


def rms_vector(u: np.ndarray) -> float:
    """Pointwise-vector RMS over all sites: sqrt(mean_x |u(x)|^2); u has a leading component axis."""
    return float(np.sqrt(np.mean(np.sum(np.asarray(u, dtype=np.float64) ** 2, axis=0))))


def velocity_error(u: np.ndarray, u_ref: np.ndarray) -> float:
    """Absolute velocity error: pointwise-vector RMS of u - u_ref."""
    return rms_vector(np.asarray(u, dtype=np.float64) - np.asarray(u_ref, dtype=np.float64))


def relative_error(u: np.ndarray, u_ref: np.ndarray) -> float:
    """Engineering error: absolute error over the numerical endpoint RMS, 1e-12 denominator floor."""
    return velocity_error(u, u_ref) / max(rms_vector(u), 1e-12)


def rel_l2(a: np.ndarray, b: np.ndarray) -> float:
    """Parity metric ||a - b||_2 / ||b||_2."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def matched_gate(e_scheme: float, e_explicit: float) -> bool:
    """Matched-accuracy gate e_abs <= 3 e_explicit."""
    return e_scheme <= 3.0 * e_explicit


def nint(x: float) -> int:
    """Nearest integer with halves rounded up: floor(x + 1/2) (Section 4.1)."""
    return int(np.floor(x + 0.5))
