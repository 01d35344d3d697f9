"""Periodic macroscopic shadow correction (Section 3.2), FP64 oracle.

Test infrastructure.  The transform is the paper's convention (Eq.
fft-convention): forward unnormalised with e^{-ik.x}, inverse with 1/N_Omega,
wavenumbers k_j = 2 pi j / N with signed j (Eq. wavenumbers), and the
rectangular mask |k_alpha| <= pi/2, i.e. |j_alpha| <= N/4 on integers, boundary
kept (Eq. shadow-mask).  The DFT is a naive separable sum evaluated only at the
masked modes (forward) and summed only over the masked modes (inverse), written
as products with explicit DFT matrices.

Pins (tests/test_oracle_shadow.py): the masked naive DFT against a brute-force
O(N^4) quadruple loop on N <= 8 and against numpy.fft on the masked modes; the
masked round trip reproduces band-limited fields; the closed-form Schur
elimination (Eq. schur) against a dense complex solve of H(k) built from Eqs.
shadow-cont / shadow-mom; r = 0 gives a zero correction; the k = 0 mean error
of one corrected iteration is multiplied by exactly -(1 - gamma_q)/2.
"""
import numpy as np

from .kinetics import linear_lift, moments
from .lattice import CS2, Lattice


def masked_indices(N: int) -> np.ndarray:
    """Signed integer wavenumber indices kept by the mask: -N/4 .. N/4 (Eq. shadow-mask)."""
    if N % 4:
        raise ValueError("N must be a multiple of 4")
    return np.arange(-(N // 4), N // 4 + 1, dtype=np.int64)


def wavenumber(j: np.ndarray, N: int) -> np.ndarray:
    """k_j = 2 pi j / N for a signed index j, |j| <= N/2   (Eq. wavenumbers)."""
    return 2.0 * np.pi * j / N


def dft_matrix(N: int, J: np.ndarray, sign: int) -> np.ndarray:
    """M[j, x] = exp(sign * 2 pi i j x / N) for j in J, x = 0..N-1 (phase reduced mod N)."""
    x = np.arange(N, dtype=np.int64)
    ph = np.mod(np.outer(J, x), N).astype(np.float64) * (2.0 * np.pi / N)
    return np.cos(ph) + 1j * sign * np.sin(ph)


def dft_forward_masked(g: np.ndarray) -> np.ndarray:
    """g_hat(k) = sum_x g(x) e^{-ik.x} at every masked k; g has grid shape (.., Ny, Nx).

    Output axes follow the grid axes with each axis replaced by the masked index
    list (ordered -N/4 .. N/4).
    """
    d = g.ndim
    out = g.astype(np.complex128)
    for ax in range(d):
        N = g.shape[ax]
        F = dft_matrix(N, masked_indices(N), -1)
        out = np.moveaxis(np.tensordot(F, out, axes=([1], [ax])), 0, ax)
    return out


def dft_inverse_masked(g_hat: np.ndarray, shape) -> np.ndarray:
    """g(x) = (1/N_Omega) sum_{masked k} g_hat(k) e^{+ik.x}; other modes are zero."""
    out = g_hat
    n_omega = 1
    for ax, N in enumerate(shape):
        G = dft_matrix(N, masked_indices(N), +1).T  # (N, |J|)
        out = np.moveaxis(np.tensordot(G, out, axes=([1], [ax])), 0, ax)
        n_omega *= N
    return out / n_omega


def mode_wavevectors(shape):
    """Wavevector components on the masked grid, ordered (k_x, k_y[, k_z]).

    ``shape`` is the grid shape (Ny, Nx) or (Nz, Ny, Nx); component alpha lives
    on grid axis d-1-alpha.
    """
    d = len(shape)
    axes_k = [wavenumber(masked_indices(N), N) for N in shape]
    mesh = np.meshgrid(*axes_k, indexing="ij")  # mesh[ax] varies along grid axis ax
    return [mesh[d - 1 - a] for a in range(d)]


def schur_solve(rp_hat: np.ndarray, rm_hat: np.ndarray, kvec, a: float, nu: float):
    """Closed-form block elimination of H(k) dm = r_hat   (Eq. schur).

    dp = (rp - i k.rm / (a + nu|k|^2)) / (a + cs^2 |k|^2 / (a + nu|k|^2))
    du = (rm - cs^2 i k dp) / (a + nu|k|^2)
    """
    k2 = sum(k * k for k in kvec)
    dvisc = a + nu * k2
    k_dot_rm = sum(kvec[al] * rm_hat[al] for al in range(len(kvec)))
    dp = (rp_hat - 1j * k_dot_rm / dvisc) / (a + CS2 * k2 / dvisc)
    du = np.stack([(rm_hat[al] - CS2 * 1j * kvec[al] * dp) / dvisc for al in range(len(kvec))])
    return dp, du


def shadow_matrix(kvec_point, a: float, nu: float) -> np.ndarray:
    """H(k) at one wavevector (Eqs. shadow-cont, shadow-mom): [[a, ik^T], [cs^2 ik, (a+nu|k|^2) I]]."""
    k = np.asarray(kvec_point, dtype=np.float64)
    d = k.size
    H = np.zeros((d + 1, d + 1), dtype=np.complex128)
    H[0, 0] = a
    H[0, 1:] = 1j * k
    H[1:, 0] = CS2 * 1j * k
    H[1:, 1:] = (a + nu * (k @ k)) * np.eye(d)
    return H


def shadow_dm(Pr: np.ndarray, a: float, nu: float) -> np.ndarray:
    """delta m_sh = F^{-1}[ chi H^{-1} F[P r] ]   (Eq. shadow-update, first two lines).

    ``Pr`` has shape (d+1, *grid): the zeroth and first moments of the raw residual.
    """
    shape = Pr.shape[1:]
    hats = [dft_forward_masked(Pr[i]) for i in range(Pr.shape[0])]
    kvec = mode_wavevectors(shape)
    dp, du = schur_solve(hats[0], np.stack(hats[1:]), kvec, a, nu)
    dm = [dft_inverse_masked(dp, shape).real]
    for al in range(du.shape[0]):
        dm.append(dft_inverse_masked(du[al], shape).real)
    return np.stack(dm)


def shadow_correction(lat: Lattice, r: np.ndarray, a: float, nu: float):
    """Population correction delta f_sh = E delta m_sh for the raw residual r (Eqs. lift, shadow-update).

    Returns (delta_m, delta_f).
    """
    dm = shadow_dm(moments(lat, r), a, nu)
    return dm, linear_lift(lat, dm)
