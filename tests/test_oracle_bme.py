"""Pins for the oracle's thermodynamic-integration estimator (BME appendix): a closed-form
integrand, the variance formula on independent draws, and the analytic marginal likelihood of a
Gaussian-likelihood GP (CPU only)."""
import numpy as np
import scipy.stats as st

from oracle.bme import gaussian_tempered_loglik_mean, thermodynamic_integration
from oracle.kernels import kernel_derivs
from paper_2511_06407_b300 import workloads as wl


def test_trapezoid_on_a_closed_form_integrand():
    tau = np.linspace(0, 1, 201)
    est, _ = thermodynamic_integration(tau[::-1], tau ** 2)  # order does not matter
    assert abs(est - 1.0 / 3.0) < 1e-5                       # trapezoid error h^2/6 = 4e-6


def test_variance_formula_matches_replicated_estimates():
    """Var = sum_s w_s^2 V_s matches the spread of replicated estimates; the appendix's printed
    formula (no cross terms) is too small by 37% on this schedule."""
    rng = np.random.default_rng(0)
    tau = np.array([0.0, 0.1, 0.35, 0.7, 1.0])
    v = np.array([4.0, 1.0, 2.0, 0.5, 3.0])
    reps = [thermodynamic_integration(tau, rng.normal(0, np.sqrt(v)))[0] for _ in range(20000)]
    _, var = thermodynamic_integration(tau, np.zeros(5), v)
    assert abs(np.var(reps) / var - 1.0) < 0.05
    dt = np.diff(tau)
    printed = 0.25 * (v[0] * dt[0] ** 2 + v[-1] * dt[-1] ** 2) + sum(
        0.25 * v[s] * (dt[s - 1] ** 2 + dt[s] ** 2) for s in range(1, 4))
    assert np.var(reps) / printed > 1.3


def test_gaussian_gp_evidence_is_the_integral_of_the_tempered_means():
    """ln N(y; 0, K + s2 I) (the exact evidence) equals the integral over tau of the closed-form
    E_tau[ln P(y | f)]; the trapezoid rule on a fine power schedule converges to it."""
    prob = wl.gp_regression(12, seed=3, noise_var=0.2)
    K = kernel_derivs("se", prob["X"], prob["u_fixed"], 1e-6)[0]
    y = prob["y"]
    exact = st.multivariate_normal(np.zeros(len(y)), K + 0.2 * np.eye(len(y))).logpdf(y)
    errs = []
    for S in (17, 65, 257):
        tau = (np.arange(S) / (S - 1.0)) ** 5
        means = [gaussian_tempered_loglik_mean(K, y, 0.2, t) for t in tau]
        errs.append(abs(thermodynamic_integration(tau, means)[0] - exact))
    assert errs[2] < errs[1] < errs[0] and errs[2] < 2e-3 * abs(exact), errs
