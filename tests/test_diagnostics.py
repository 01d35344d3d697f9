"""Host-side march diagnostics (Eqs. rho-observed, swork) against the oracle and hand values."""
import math

import numpy as np

from oracle import march as OM
from paper_2609_39474_b300 import diagnostics as D


def test_rho_observed_matches_the_oracle_and_a_geometric_sequence():
    rng = np.random.default_rng(4)
    for n in (3, 5, 12, 40):
        R = np.exp(np.cumsum(rng.normal(-0.3, 0.2, n)))
        for m in (8, 10):
            assert math.isclose(D.rho_observed(R, m), OM.rho_observed(R, m), rel_tol=1e-12)
    # an exactly geometric history returns its ratio; fewer than three residuals give None
    assert math.isclose(D.rho_observed([1.0 * 0.3 ** k for k in range(15)]), 0.3, rel_tol=1e-12)
    assert D.rho_observed([1.0, 0.5]) is None


def test_rho_observed_uses_only_the_tail():
    # m_rho = 10: only the last ten ratios count (the first ratios here are 0.9, the tail 0.5)
    R = [0.9 ** k for k in range(6)]
    for _ in range(10):
        R.append(R[-1] * 0.5)
    assert math.isclose(D.rho_observed(R, 10), 0.5, rel_tol=1e-12)


def test_step_residuals_and_work_ratio():
    hist = [1.0, 0.1, 0.5, 0.05, 0.005, 0.2, 0.02]
    assert D.step_residuals(hist, [2, 3, 2]) == [[1.0, 0.1], [0.5, 0.05, 0.005], [0.2, 0.02]]
    # 16 steps of 2 sweeps to T_end = 157286: W = 32 maps + 16 corrections
    assert math.isclose(D.work_ratio(157286, 32, 16), 157286 / 48)
    assert math.isclose(D.work_ratio(100, 30, 10, corrector=False), 100 / 30)
