"""The package's model-evidence post-processing (bme.evidence, run on the sampler's recorded
log-likelihoods) against the oracle's thermodynamic integration, and its standard error against
the spread of replicated estimates (CPU only)."""
import numpy as np

from oracle.bme import thermodynamic_integration
from paper_2511_06407_b300 import bme


def _samples(rng, taus_per_chain, n_iter, sd=1.0):
    """ln P samples whose mean at temperature tau is -3 + 2 tau^0.5 (white noise of SD sd)."""
    mu = -3.0 + 2.0 * np.sqrt(taus_per_chain)
    return mu[None, :] + sd * rng.standard_normal((n_iter, len(taus_per_chain)))


def test_evidence_matches_the_oracle_trapezoid_and_ignores_chain_order():
    rng = np.random.default_rng(0)
    taus = np.repeat(bme.power_schedule(8), 3)  # 8 temperatures x 3 chains
    ll = _samples(rng, taus, 400)
    est, se, table = bme.evidence(taus, ll)
    t, means, vars_ = (np.array(c) for c in zip(*table))
    np.testing.assert_allclose(t, np.unique(taus), rtol=0, atol=0)
    for s, tau in enumerate(t):
        assert means[s] == ll[:, taus == tau].mean()
    ref, ref_var = thermodynamic_integration(t, means, vars_)
    assert abs(est - ref) <= 1e-14 * abs(ref)
    assert abs(se ** 2 - ref_var) <= 1e-12 * ref_var
    # the estimate does not depend on the order of the chains; the standard error's batches may
    # span two chains of one temperature, so it moves with the order by its own sampling noise only
    perm = rng.permutation(len(taus))
    est2, se2, _ = bme.evidence(taus[perm], ll[:, perm])
    assert abs(est2 - est) <= 1e-13 * abs(est)
    assert abs(se2 - se) <= 0.25 * se


def test_evidence_standard_error_matches_replicated_spread():
    """Over 300 independent replicates, the spread of the estimates agrees with the reported
    standard error (white-noise samples: batch means are unbiased for the variance of the mean)."""
    rng = np.random.default_rng(1)
    taus = np.repeat(bme.piecewise_schedule()[::10], 2)  # 11 temperatures x 2 chains
    ests, ses = [], []
    for _ in range(300):
        est, se, _ = bme.evidence(taus, _samples(rng, taus, 200))
        ests.append(est)
        ses.append(se)
    ratio = np.std(ests, ddof=1) / np.mean(ses)
    assert 0.85 < ratio < 1.15, ratio
    # and the estimate is centred on the trapezoid of the true means
    t = np.unique(taus)
    truth, _ = thermodynamic_integration(t, -3.0 + 2.0 * np.sqrt(t))
    assert abs(np.mean(ests) - truth) < 4 * np.std(ests, ddof=1) / np.sqrt(len(ests))
