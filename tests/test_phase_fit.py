"""The logistic fit of recovery data used for phase transitions and their widths
(paper_1704_09012_gb300.phase.fit_logistic), pinned on data whose transition is known."""
import math

import numpy as np
import pytest

from paper_1704_09012_gb300.phase import fit_logistic


def _p(r, rho50, w):
    return 1.0 / (1.0 + np.exp((r - rho50) / w))


def test_fit_recovers_a_known_transition_from_exact_expectations():
    r = np.round(np.arange(0.01, 0.4, 0.01), 10)
    n = 10 ** 6
    k = n * _p(r, 0.2, 0.015)                       # expected counts: the MLE is the truth
    rho50, w, width = fit_logistic(r, k, n)
    assert rho50 == pytest.approx(0.2, abs=1e-6)
    assert w == pytest.approx(0.015, rel=1e-4)
    assert width == pytest.approx(2 * math.log(9) * 0.015, rel=1e-4)


def test_fit_on_sampled_recoveries_and_width_shrinks_with_sharper_data():
    rng = np.random.default_rng(0)
    r = np.round(np.arange(0.01, 0.4, 0.01), 10)
    widths = []
    for w_true in (0.03, 0.01):
        k = rng.binomial(2000, _p(r, 0.25, w_true))
        rho50, w, width = fit_logistic(r, k, 2000)
        assert rho50 == pytest.approx(0.25, abs=3 * w_true / math.sqrt(2000) * 10)
        assert w == pytest.approx(w_true, rel=0.15)
        widths.append(width)
    assert widths[1] < widths[0]


def test_fit_of_a_step_hits_the_lower_width_bound():
    r = np.round(np.arange(0.01, 0.21, 0.01), 10)
    k = np.where(r <= 0.12, 10, 0)                  # all recovered up to 0.12, none after
    rho50, w, _ = fit_logistic(r, k, 10)
    assert 0.12 <= rho50 <= 0.13
    assert 2 * math.log(9) * w < 0.01 / 5          # far below the rho grid step
