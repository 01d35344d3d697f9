"""The complete fine-grid sweep T and its raw residual (Eqs. sweep, residual), FP64.

Test infrastructure.  Periodic domain, so the boundary assignment is the
identity (B = I, b = 0).  Push streaming (S g)_k(x + c_k) = g_k(x) is a
periodic roll of each direction by c_k.

Pins (tests/test_oracle_sweep.py): brute-force per-site loop on N = 4 / 8
grids; global mass and momentum balance sum_x P T(f) = sum_x (P f + s) exactly
for any nonlinear field; the mean-moment map of one Picard sweep is exactly
affine with slope gamma_q (derived from Eqs. local-linear-response and
zero-mode-scale); with a = h = 0 the sweep is the explicit LBM step.
"""
import numpy as np

from .kinetics import (collide_operating, collide_trt, moments, reconstruct,
                       source_moments)
from .lattice import Lattice


def stream(lat: Lattice, g: np.ndarray) -> np.ndarray:
    """Periodic push streaming: out_k(x + c_k) = g_k(x).

    Arrays are indexed [k, (z,) y, x]; component alpha of c_k shifts the axis
    that holds coordinate alpha (x is the last axis).
    """
    out = np.empty_like(g)
    d = lat.d
    grid_axis = tuple(d - 1 - a for a in range(d))  # component alpha lives on grid axis d-1-alpha
    for k in range(lat.Q):
        shifts = tuple(int(lat.c[k, a]) for a in range(d))
        out[k] = np.roll(g[k], shift=shifts, axis=grid_axis)
    return out


def sweep(lat: Lattice, f: np.ndarray, a: float, h: np.ndarray,
          omega=None) -> np.ndarray:
    """f_T = T(f) = S C(f; m, s) with m = R(f), s = h - a m   (Eq. sweep).

    ``omega=None`` uses the operating point (Eq. collision-operating);
    ``omega=(w_plus, w_minus)`` uses the general TRT collision (Eq. collision).
    """
    m = reconstruct(moments(lat, f), a, h)
    s = source_moments(a, h, m)
    if omega is None:
        c = collide_operating(lat, m, s)
    else:
        c = collide_trt(lat, f, m, s, omega[0], omega[1])
    return stream(lat, c)


def residual(f_T: np.ndarray, f: np.ndarray):
    """r = T(f) - f and its population RMS norm   (Eq. residual)."""
    r = f_T - f
    return r, float(np.sqrt(np.sum(r * r) / r.size))


def explicit_step(lat: Lattice, f: np.ndarray, omega=None) -> np.ndarray:
    """Explicit LBM step: the same collision and streaming with no BDF source (a = h = 0)."""
    zero = np.zeros((lat.d + 1,) + f.shape[1:])
    return sweep(lat, f, 0.0, zero, omega)
