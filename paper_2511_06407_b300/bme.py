"""Bayesian model evidence from tempered chains by thermodynamic integration (host-side
post-processing of rmhmc_sample's loglik output; the BME appendix, Eq. MC_integration).

All chains of one model may carry different inverse temperatures tau (rmhmc_init_model's tau);
evidence() groups them by tau, averages the recorded untempered log-likelihoods per temperature,
and integrates over tau with the trapezoid rule. The estimate's variance is sum_s w_s^2 V_s
(trapezoid weights w_s, V_s the variance of temperature s's mean from batch means over the samples
of all chains at that temperature, temperatures independent); the appendix's printed formula drops
the cross term V_s dt_{s-1} dt_s / 2 of every interior temperature.
"""
import numpy as np


def power_schedule(S, power=5.0):
    """tau_s = (s / (S - 1))^power, s = 0..S-1 (Calderhead and Girolami's schedule)."""
    return (np.arange(S) / (S - 1.0)) ** power


def piecewise_schedule():
    """The 101 inverse temperatures of the paper's own thermodynamic-integration runs (Sec. 2.5),
    from 1 down to 0 in four linear pieces (steps 0.02, 0.005, 0.002, 0.001 from s = 1, 41, 71, 91):
    finer near tau = 0, where the tempered mean of ln P changes fastest."""
    s = np.arange(1, 102, dtype=np.float64)
    return np.select([s <= 41, s <= 71, s <= 91],
                     [1.0 - 0.02 * (s - 1), 0.2 - 0.005 * (s - 41), 0.05 - 0.002 * (s - 71)],
                     0.01 - 0.001 * (s - 91))


def _batch_var_of_mean(x, n_batches=10):
    x = np.asarray(x, dtype=np.float64)
    n = len(x) // n_batches * n_batches
    if n < n_batches * 2:
        return float(np.var(x, ddof=1) / max(len(x), 1))
    b = x[:n].reshape(n_batches, -1).mean(axis=1)
    return float(np.var(b, ddof=1) / n_batches)


def evidence(tau_per_chain, loglik):
    """tau_per_chain: (n_chains,), loglik: (n_iter, n_chains) untempered ln P(y | F) samples.
    Returns (ln BME estimate, its standard error, per-temperature (tau, mean, var) table).
    The variance of each temperature's mean comes from 10 batch means over its chains' series laid
    end to end (a batch may span two chains), so the standard error, unlike the estimate, moves
    with the order of the chains by its own sampling noise."""
    tau_per_chain = np.asarray(tau_per_chain, dtype=np.float64)
    loglik = np.asarray(loglik, dtype=np.float64)
    taus = np.unique(tau_per_chain)
    means, vars_ = [], []
    for t in taus:
        x = loglik[:, tau_per_chain == t]
        # chain-major order so that batch means follow each chain's time series
        means.append(float(x.mean()))
        vars_.append(_batch_var_of_mean(x.T.reshape(-1)))
    means, vars_ = np.array(means), np.array(vars_)
    dt = np.diff(taus)
    w = np.zeros(len(taus))
    w[1:] += 0.5 * dt
    w[:-1] += 0.5 * dt
    est = float(np.sum(w * means))
    var = float(np.sum(w * w * vars_))
    return est, float(np.sqrt(var)), list(zip(taus.tolist(), means.tolist(), vars_.tolist()))
