"""Bayesian model evidence by thermodynamic integration (oracle), the BME appendix.

ln BME = integral_0^1 E_{P_tau}[ln P(X | a)] d tau, P_tau ∝ P(X | a)^tau G_theta(a) Pi(theta)
(Eq. MC_integration). With inverse temperatures 0 = tau_1 < ... < tau_S = 1 (the appendix orders
them from 1 down to 0; the trapezoid weights use |tau_s - tau_{s-1}|) and per-temperature means
E_s of the sampled ln P(X | a):
  ln BME ~ sum_{s=2..S} (E_s + E_{s-1}) / 2 (tau_s - tau_{s-1}) = sum_s w_s E_s
with trapezoid weights w_1 = dt_1 / 2, w_s = (dt_{s-1} + dt_s) / 2, w_S = dt_{S-1} / 2. With the
E_s independent and V_s the variance of E_s, Var = sum_s w_s^2 V_s. The appendix prints
  sum_{s=2..S-1} V_s (dt_{s-1}^2 + dt_s^2) / 4 + (V_1 dt_1^2 + V_S dt_{S-1}^2) / 4,
which drops the cross term V_s dt_{s-1} dt_s / 2 of every interior w_s^2 and so underestimates
the variance of its own estimator (a test replicating the estimate shows it); the oracle uses
sum_s w_s^2 V_s.
"""
import numpy as np


def thermodynamic_integration(tau, means, variances=None):
    """(estimate, variance or None) for temperatures `tau` (any order) and per-temperature means."""
    tau = np.asarray(tau, dtype=np.float64)
    means = np.asarray(means, dtype=np.float64)
    order = np.argsort(tau)
    t, e = tau[order], means[order]
    dt = np.diff(t)
    est = float(np.sum(0.5 * (e[1:] + e[:-1]) * dt))
    if variances is None:
        return est, None
    v = np.asarray(variances, dtype=np.float64)[order]
    w = np.zeros(len(t))
    w[1:] += 0.5 * dt
    w[:-1] += 0.5 * dt
    return est, float(np.sum(w * w * v))


def gaussian_tempered_loglik_mean(K, y, noise_var, tau):
    """E_{P_tau}[ln N(y | f, s2 I)] for f ~ N(0, K) tempered by tau (closed form: P_tau is
    Gaussian with precision K^-1 + tau/s2 I and mean Sigma_tau (tau/s2) y)."""
    N = len(y)
    A = np.linalg.inv(K) + (tau / noise_var) * np.eye(N)
    Sig = np.linalg.inv(A)
    Sig = 0.5 * (Sig + Sig.T)
    m = Sig @ ((tau / noise_var) * y)
    r = y - m
    return -0.5 * N * np.log(2 * np.pi * noise_var) - 0.5 * (r @ r + np.trace(Sig)) / noise_var
