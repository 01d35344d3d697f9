"""Full-symbol reference operator for off-design collisions (Section 4.1, Eq. full-symbol), FP64.

Test infrastructure.  At the uniform rest state (p_hat, u) = (1, 0) a forward difference of size
1e-7 builds the local Q x Q collision Jacobian J with the case's actual (omega+, omega-) (Eq.
collision, with the BDF reconstruction and source of the step: h = a (1, 0) so that s = 0 at
rest).  Streaming gives L(k) = Z(k) J with Z(k) = diag(exp(-i k . c_k)), and every wavevector's
correction solves [I - L(k)] df(k) = r(k); the next trial is f + df.  It corrects all Q population
fields at every wavevector (no mask), so it is the linearised Newton step about rest, used to
measure the contraction attainable away from the operating point.

The transforms are numpy FFTs on the full grid (every wavevector is corrected).  Pins
(tests/test_oracle_fullsymbol.py): at omega+- = 1, J equals gamma E P (Eq. symbol) to the
difference error; ghost vectors (P g = 0) are eigenvectors with the TRT relaxation factors
1 - omega+ (even) and 1 - omega- (odd), so |1 - omega+| = eta(nu) = |6 nu - 1| / (6 nu + 1)
(Eq. eta); in the linear regime one corrected iteration removes the residual to the difference
error of J.  rest_jacobian_exact is the derivative itself (complex step), pinned against the forward
difference and, at omega+- = 1, against gamma E P to rounding; it is the Jacobian the GPU's
full-symbol correction is compared with.
"""
import numpy as np

from .kinetics import collide_trt, feq, moments, reconstruct, source_moments
from .lattice import Lattice


def trt_rates(nu: float, Lambda: float):
    """(omega+, omega-) from nu = cs^2 (tau+ - 1/2) and Lambda = (tau+ - 1/2)(tau- - 1/2)   (Eq. trt)."""
    tp = 3.0 * nu + 0.5
    tm = Lambda / (tp - 0.5) + 0.5
    return 1.0 / tp, 1.0 / tm


def eta(nu: float) -> float:
    """Ghost survival |6 nu - 1| / (6 nu + 1)   (Eq. eta)."""
    return abs(6.0 * nu - 1.0) / (6.0 * nu + 1.0)


def _rest_collision(lat: Lattice, a: float, omega):
    """f -> C(f) at the rest state's history: h = a (1, 0), so that s = h - a m = 0 at m = (1, 0)."""
    F = lat.d + 1
    h = np.zeros(F)
    h[0] = a

    def coll(f):
        m = reconstruct(moments(lat, f), a, h)
        return collide_trt(lat, f, m, source_moments(a, h, m), omega[0], omega[1])

    return coll, feq(lat, np.ones(()), np.zeros(lat.d))


def rest_jacobian(lat: Lattice, a: float, omega, delta: float = 1e-7) -> np.ndarray:
    """Q x Q forward-difference Jacobian of the collision at rest (Eq. full-symbol)."""
    coll, f0 = _rest_collision(lat, a, omega)
    c0 = coll(f0)
    J = np.empty((lat.Q, lat.Q))
    for j in range(lat.Q):
        fj = f0.copy()
        fj[j] += delta
        J[:, j] = (coll(fj) - c0) / delta
    return J


def rest_jacobian_exact(lat: Lattice, a: float, omega) -> np.ndarray:
    """The derivative that rest_jacobian approximates, by complex-step differentiation of the same
    collision (Im C(f0 + i h e_j) / h with h = 1e-30: no subtraction, exact to rounding)."""
    coll, f0 = _rest_collision(lat, a, omega)
    hstep = 1e-30
    J = np.empty((lat.Q, lat.Q))
    for j in range(lat.Q):
        fj = f0.astype(np.complex128)
        fj[j] += 1j * hstep
        J[:, j] = np.imag(coll(fj)) / hstep
    return J


def wavevectors(lat: Lattice, shape):
    """k on the FFT grid of `shape`: component alpha on grid axis d-1-alpha (x is the last axis)."""
    d = lat.d
    ks = [2.0 * np.pi * np.fft.fftfreq(shape[ax]) for ax in range(d)]
    K = np.meshgrid(*ks, indexing="ij")
    return [K[d - 1 - al] for al in range(d)]


def correction_matrices(lat: Lattice, J: np.ndarray, shape) -> np.ndarray:
    """[I - Z(k) J]^{-1} for every wavevector of the grid, shape grid + (Q, Q)."""
    kv = wavevectors(lat, shape)
    phase = sum(np.multiply.outer(kv[al], lat.c[:, al].astype(np.float64)) for al in range(lat.d))
    Z = np.exp(-1j * phase)                                  # grid + (Q,)
    M = np.eye(lat.Q) - Z[..., :, None] * J               # I - diag(Z(k)) J at every k
    return np.linalg.inv(M)


def full_symbol_correction(lat: Lattice, r: np.ndarray, Minv: np.ndarray) -> np.ndarray:
    """df = F^{-1}[ (I - Z J)^{-1} F[r] ] over all Q fields and all wavevectors."""
    axes = tuple(range(1, lat.d + 1))
    rh = np.fft.fftn(r, axes=axes)                           # (Q,) + grid
    rh = np.moveaxis(rh, 0, -1)                              # grid + (Q,)
    dh = np.einsum("...ij,...j->...i", Minv, rh)
    df = np.fft.ifftn(np.moveaxis(dh, -1, 0), axes=axes)
    return np.real(df)
