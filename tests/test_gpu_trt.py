"""Off-design collisions on the GPU: the general TRT sweep (Eq. collision) against the FP64 oracle,
the off-design march and explicit LBM, and the shadow correction's off-design contraction."""
import numpy as np
import pytest
import torch

from oracle import fullsymbol as FS
from oracle import kinetics as OK
from oracle import march as OM
from oracle import sweep as OSW
from oracle.lattice import D2Q9
from workloads.fields import random_moments, random_phase, random_populations, tgv2d
from tests.gpu_helpers import dev, host, rel_l2

pytestmark = pytest.mark.gpu
TOL = {"fp64": dict(f=1e-14, pr=1e-13, ss=1e-12), "fp32": dict(f=1e-6, pr=1e-5, ss=1e-5)}
OFF = [(0.12, 0.25), (1 / 6, 0.05), (0.25, 1.0)]


def _PL():
    from paper_2609_39474_b300 import lattice as PL
    return PL


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("lift", [False, True], ids=["nolift", "lift"])
@pytest.mark.parametrize("n", [8, 64, 256])
@pytest.mark.parametrize("nu,lam", OFF)
def test_trt_sweep_matches_oracle(n, lift, precision, nu, lam):
    PL = _PL()
    wp, wm = FS.trt_rates(nu, lam)
    f = random_populations(9, (n, n), seed=1, scale=1e-3)
    h = random_moments(2, (n, n), seed=2, scale=1e-4)
    dm = random_moments(2, (n, n), seed=3, scale=1e-4) if lift else None
    T = PL.storage_dtype(precision)
    f_s, h_s = dev(f, T), dev(h, T)
    dm_s = dev(dm, T) if lift else None
    a = 0.05
    f_out, pr, ss = PL.sweep_trt(n, precision, a, wp, wm, f_s, h_s, dm_s)
    torch.cuda.synchronize()
    trial = host(f_s) + (OK.linear_lift(D2Q9, host(dm_s)) if lift else 0.0)
    f_T = OSW.sweep(D2Q9, trial, a, host(h_s), omega=(wp, wm))
    r, _ = OSW.residual(f_T, trial)
    tol = TOL[precision]
    assert rel_l2(host(f_out), f_T) < tol["f"]
    assert rel_l2(host(pr), OK.moments(D2Q9, r)) < tol["pr"]
    assert abs(float(ss.item()) / float(np.sum(r * r)) - 1) < tol["ss"]


def test_trt_at_unit_rates_is_the_operating_point_sweep():
    PL = _PL()
    n = 64
    f = dev(random_populations(9, (n, n), seed=4, scale=1e-3))
    h = dev(random_moments(2, (n, n), seed=5, scale=1e-4))
    dm = dev(random_moments(2, (n, n), seed=6, scale=1e-4))
    a = 0.04
    g1 = PL.sweep(2, n, "fp64", a, f, h, dm)
    g2 = PL.sweep_trt(n, "fp64", a, 1.0, 1.0, f, h, dm)
    assert rel_l2(host(g2[0]), host(g1[0])) < 1e-14
    assert rel_l2(host(g2[1]), host(g1[1])) < 1e-12


@pytest.mark.parametrize("nu,lam", [(0.14, 0.25), (1 / 6, 0.05)])
def test_off_design_march_replay_parity(nu, lam):
    # (nu = 0.12 at this dt and field is already past the shadow correction's stability limit)
    PL = _PL()
    N, dt = 32, 12.0
    wp, wm = FS.trt_rates(nu, lam)
    p, u = random_phase(N, 2, 1.0, seed=7, kmax=4)
    prm = OM.MarchParams(dt=dt, eps=1e-11, kmax=400, omega=(wp, wm), nu=nu)
    st = OM.init_state(D2Q9, p, u)
    recs = OM.march(st, prm, 5)
    assert all(r.converged for r in recs)
    L = PL.MscLattice(2, N, "fp64")
    L.set_params(dt=dt, eps=prm.eps, nu=nu, kmax=400, replay=True, omega=(wp, wm))
    L.set_replay_counts([r.iters for r in recs])
    L.init_fields(p, u)
    L.march(5)
    assert L.stats()["status"] == 0
    assert rel_l2(host(L.fields()[1]), st.m_n[1:]) < 1e-12
    # the explicit LBM with the same collision
    f0 = OK.feq(D2Q9, p, u)
    L.init_fields(p, u)
    L.explicit_march(13)
    assert rel_l2(L.populations(), OM.explicit_march(D2Q9, f0, 13, omega=(wp, wm))) < 1e-13


def test_shadow_correction_off_design_contraction():
    # one interior BDF2 step of Taylor-Green at N = 32 (as the oracle scan): the shadow correction
    # contracts at the operating point, degrades as nu falls and fails to converge at nu = 0.10
    # (Section 4.6: divergence by nu ~ 0.09)
    PL = _PL()
    from paper_2609_39474_b300 import diagnostics as DG
    N, dt = 32, 20.0
    p, u = tgv2d(N, 1.0)
    rho = {}
    for nu in (1 / 6, 0.12, 0.10):
        wp, wm = FS.trt_rates(nu, 0.25)
        L = PL.MscLattice(2, N, "fp64")
        L.set_params(dt=dt, eps=1e-12, nu=nu, kmax=80, omega=(wp, wm))
        L.init_fields(p, u)
        L.march(1)
        L.march(1)
        s = L.stats()
        rho[nu] = (s["status"], DG.rho_observed(L.residual_history(), 10))
    assert rho[1 / 6][0] == 0 and rho[1 / 6][1] < 0.15
    assert rho[0.12][0] == 0 and 0.2 < rho[0.12][1] < 0.6
    assert rho[0.10][0] != 0 and rho[0.10][1] > 1.0


def _mode_fields(N, jvec, amp):
    x = np.arange(N)
    ph = 2 * np.pi * (jvec[0] * x[None, :] + jvec[1] * x[:, None]) / N
    return amp * np.cos(ph), np.stack([0.3 * amp * np.sin(ph), -0.7 * amp * np.cos(ph + 0.4)])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("nu,lam,jvec", [(0.1, 0.25, (8, 8)), (0.12, 0.25, (8, -8)), (0.14, 0.25, (8, 0)),
                                         (1 / 6, 2.0, (4, 2)), (0.25, 0.05, (4, 2))])
def test_off_design_contraction_matches_the_linear_symbol(nu, lam, jvec, precision):
    # The linear Fourier analysis of Section 4.6 on the GPU march: a 1e-12 single mode, one BDF1 step
    # with the general TRT sweep and the shadow correction, no acceptance (eps = 0, 60 inner
    # iterations).  Each inner residual shrinks or grows by the spectral radius of the oracle's
    # linearised corrected iteration G(k) (the mask corner diverges at nu = 0.10 and 0.12), and the
    # whole residual history matches the oracle march.
    from oracle import linear as OL
    from paper_2609_39474_b300 import diagnostics as DG
    PL = _PL()
    N, dt, K = 32, 20.0, 60
    omega = FS.trt_rates(nu, lam)
    k = 2 * np.pi * np.array(jvec) / N
    rho = OL.spectral_radius(OL.trt_corrected_symbol(D2Q9, k, 1.0 / dt, nu, omega))
    p, u = _mode_fields(N, jvec, 1e-12)
    L = PL.MscLattice(2, N, precision)
    L.set_params(dt=dt, eps=0.0, nu=nu, kmax=K, omega=omega)
    L.init_fields(p, u)
    L.march(1)
    s = L.stats()
    R = L.residual_history()
    L.close()
    assert s["status"] != 0 and s["steps_done"] == 0 and len(R) == K
    assert (rho > 1) == (nu <= 0.12)
    Ro = np.asarray(OM.physical_step(OM.init_state(D2Q9, p, u),
                                     OM.MarchParams(dt=dt, nu=nu, eps=0.0, kmax=K, omega=omega)).residuals)
    if precision == "fp64":
        assert abs(DG.rho_observed(R, 10) / rho - 1) < 1e-6
        # to 1e-9 of each residual, or to rounding of the mode (1e-14 R_0) once it has decayed
        assert np.all(np.abs(R - Ro) < 1e-9 * Ro + 1e-14 * Ro[0])
    else:
        # binary32 populations round at ~1e-7 of the mode's amplitude (~1e-6 R_0): the history to 1e-3
        # above that floor, and the rate where at least 20 residuals stay above 1e-4 R_0
        assert np.all(np.abs(R - Ro) < 1e-3 * Ro + 1e-5 * Ro[0])
        above = R[:int(np.argmax(R < 1e-4 * R[0]))] if np.any(R < 1e-4 * R[0]) else R
        if len(above) >= 20:
            assert abs(DG.rho_observed(above, 10) / rho - 1) < 2e-3
