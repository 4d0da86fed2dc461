"""ESS and R-hat estimators against closed forms (AR(1) processes) and brute force."""
import numpy as np
import pytest

from paper_2511_06407_b300 import diagnostics as dg


def ar1(rho, m, n, seed):
    rng = np.random.default_rng(seed)
    x = np.empty((m, n))
    x[:, 0] = rng.standard_normal(m) / np.sqrt(1 - rho * rho)
    e = rng.standard_normal((m, n))
    for t in range(1, n):
        x[:, t] = rho * x[:, t - 1] + e[:, t]
    return x


@pytest.mark.parametrize("rho", [0.0, 0.5, 0.9])
def test_ess_of_ar1_matches_closed_form(rho):
    """For an AR(1) process the integrated autocorrelation time is (1 + rho) / (1 - rho)."""
    m, n = 4, 20000
    x = ar1(rho, m, n, seed=int(rho * 10))
    want = m * n * (1 - rho) / (1 + rho)
    for est in (dg.ess_chains(x), dg.ess_bulk(x)):
        assert abs(est / want - 1) < 0.15, (rho, est, want)


def test_autocovariance_matches_direct_sum():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((3, 37))
    got = dg._autocov(x)
    xc = x - x.mean(axis=1, keepdims=True)
    for t in (0, 1, 5, 36):
        want = (xc[:, : 37 - t] * xc[:, t:]).sum(axis=1) / 37
        np.testing.assert_allclose(got[:, t], want, rtol=1e-12, atol=1e-14)


def test_bulk_ess_is_invariant_to_monotone_maps():
    x = ar1(0.7, 4, 2000, seed=3)
    assert dg.ess_bulk(x) == pytest.approx(dg.ess_bulk(np.exp(x)), rel=1e-12)
    assert dg.rhat(x) == pytest.approx(dg.rhat(np.exp(x)), rel=1e-12)


def test_rhat_flags_chains_that_disagree():
    x = ar1(0.5, 4, 2000, seed=4)
    assert dg.rhat(x) < 1.01
    y = x + np.array([0.0, 0.0, 0.0, 3.0])[:, None]
    assert dg.rhat(y) > 1.1
    assert dg.ess_bulk(y) < 0.2 * dg.ess_bulk(x)


def test_tail_ess_matches_indicator_autocorrelation():
    """The 5 % indicator of a Gaussian AR(1) has lag-t autocorrelation
    (Phi2(q, q; rho^t) - p^2) / (p (1 - p)), q = Phi^-1(p), Phi2 the bivariate normal CDF."""
    from scipy.stats import multivariate_normal, norm
    rho, p = 0.5, 0.05
    q = norm.ppf(p)
    corr = [(multivariate_normal(cov=[[1, rho ** t], [rho ** t, 1]]).cdf([q, q]) - p * p) / (p * (1 - p))
            for t in range(1, 40)]
    tau = 1 + 2 * sum(corr)
    x = ar1(rho, 8, 20000, seed=5)
    assert abs(dg.ess_tail(x) / (x.size / tau) - 1) < 0.15


def test_summary_and_mcse():
    x = ar1(0.5, 8, 1000, seed=6)
    want = 8000 / 3
    s = dg.summary(np.stack([x.T, 2 * x.T + 1], axis=2), names=["a", "b"])
    assert [r["name"] for r in s["rows"]] == ["a", "b"]
    assert s["min_ess"] <= s["rows"][0]["ess_bulk"] and s["max_rhat"] < 1.02
    se = dg.mcse_mean(x)
    assert abs(se / (np.std(x) / np.sqrt(want)) - 1) < 0.2
