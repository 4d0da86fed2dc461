"""Effective sample size and R-hat of sampled chains (host-side analysis of rmhmc_sample output).

ESS follows Geyer (1992): the autocorrelations rho_t are summed in pairs P_k = rho_2k + rho_2k+1
while P_k > 0 (initial positive sequence), the pairs are made non-increasing (initial monotone
sequence), and tau = -1 + 2 sum_k P_k, ESS = (number of draws) / tau. For several chains the
autocorrelation combines the within-chain autocovariances with the between-chain variance, and the
draws are split in halves and rank-normalised before the estimate ("bulk" ESS and split R-hat of
Vehtari, Gelman, Simpson, Carpenter and Burkner 2021); the "tail" ESS is the smaller ESS of the
indicators of the 5 % and 95 % quantiles. Autocovariances are computed by FFT.
"""
import numpy as np
from scipy.special import ndtri
from scipy.stats import rankdata


def _autocov(x):
    """Autocovariance (biased, lag 0..n-1) of each row of x (m x n), by zero-padded FFT."""
    m, n = x.shape
    xc = x - x.mean(axis=1, keepdims=True)
    nfft = 1 << int(np.ceil(np.log2(2 * n)))
    f = np.fft.rfft(xc, nfft, axis=1)
    return np.fft.irfft(f * np.conj(f), nfft, axis=1)[:, :n] / n


def ess_chains(chains):
    """Geyer ESS of draws x (m chains x n draws), chains combined as in Vehtari et al. (2021)
    (without splitting or rank normalisation: see ess_bulk)."""
    x = np.atleast_2d(np.asarray(chains, dtype=np.float64))
    m, n = x.shape
    if n < 4:
        return float("nan")
    acov = _autocov(x)
    chain_var = acov[:, 0] * n / (n - 1.0)
    W = chain_var.mean()
    var_plus = W * (n - 1.0) / n
    if m > 1:
        var_plus += x.mean(axis=1).var(ddof=1)
    if not var_plus > 0.0:
        return float(m * n)  # constant draws
    rho = 1.0 - (W - acov.mean(axis=0)) / var_plus
    rho[0] = 1.0
    # Geyer's initial positive sequence of pair sums, then made monotone
    npairs = n // 2
    P = rho[0:2 * npairs:2] + rho[1:2 * npairs:2]
    k = 0
    while k < npairs and P[k] > 0.0:
        k += 1
    P = np.minimum.accumulate(P[:k]) if k else P[:0]
    tau = -1.0 + 2.0 * P.sum()
    tau = max(tau, 1.0 / np.log10(m * n))  # the cap of Vehtari et al. for antithetic chains
    return float(m * n / tau)


def _split(x):
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    h = x.shape[1] // 2
    return np.concatenate([x[:, :h], x[:, x.shape[1] - h:]], axis=0)


def _rank_normal(x):
    r = rankdata(x, method="average").reshape(x.shape)
    return ndtri((r - 0.375) / (x.size + 0.25))


def ess_bulk(chains):
    """Bulk ESS: Geyer ESS of the split, rank-normalised draws (m x n)."""
    s = _split(chains)
    return ess_chains(_rank_normal(s))


def ess_tail(chains):
    """Tail ESS: the smaller ESS of the indicators of the 5 % and 95 % quantiles."""
    s = _split(chains)
    lo, hi = np.quantile(s, [0.05, 0.95])
    return min(ess_chains((s <= lo).astype(np.float64)), ess_chains((s <= hi).astype(np.float64)))


def rhat(chains):
    """Rank-normalised split R-hat (the larger of the bulk and the folded-draws values)."""
    s = _split(chains)

    def basic(z):
        m, n = z.shape
        W = z.var(axis=1, ddof=1).mean()
        B = n * z.mean(axis=1).var(ddof=1)
        return float(np.sqrt(((n - 1.0) / n * W + B / n) / W)) if W > 0 else float("nan")

    folded = np.abs(s - np.median(s))
    return max(basic(_rank_normal(s)), basic(_rank_normal(folded)))


def mcse_mean(chains):
    """Monte-Carlo standard error of the posterior mean: sd / sqrt(ESS) (ESS without ranks)."""
    x = np.atleast_2d(np.asarray(chains, dtype=np.float64))
    return float(x.std(ddof=1) / np.sqrt(ess_chains(x)))


def summary(samples, names=None):
    """Per-coordinate bulk ESS, tail ESS and R-hat of samples (n_iter x n_chains x k), plus the
    minimum ESS over coordinates."""
    s = np.asarray(samples, dtype=np.float64)
    if s.ndim == 2:
        s = s[:, :, None]
    rows = []
    for j in range(s.shape[2]):
        ch = s[:, :, j].T
        rows.append({"name": names[j] if names else str(j), "ess_bulk": ess_bulk(ch),
                     "ess_tail": ess_tail(ch), "rhat": rhat(ch)})
    return {"rows": rows, "min_ess": min(min(r["ess_bulk"], r["ess_tail"]) for r in rows),
            "max_rhat": max(r["rhat"] for r in rows)}
