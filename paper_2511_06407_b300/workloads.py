"""Seeded synthetic workloads (inputs only; none of the sampler's arithmetic lives here).

Both the CUDA path and the CPU oracle receive problems built here, as plain dicts:
  {"X": (N, n_cov) float64, "y": (N,) float64, "lik": "bernoulli"|"gaussian", "noise_var": float,
   "kernels": [{"kind": "se"|"linear"|"overlap", "cols": tuple, "jitter": float,
                "prior_a": (a_c, a_theta), "prior_b": (b_c, b_theta)}, ...],
   "sample_hypers": bool, "u_fixed": (2n,) or None}

The latent functions behind the labels are drawn in weight space, so no kernel matrix is formed:
  SE       random Fourier features (Rahimi and Recht 2007), 4096 features:
           f(x) = sqrt(2c/M) sum_j cos(w_j . x + b_j), w_j ~ N(0, I / l^2), b_j ~ U[0, 2 pi)
  linear   f(x) = sqrt(c) (w . x + sqrt(b) w_0),  w ~ N(0, I)
  overlap  exp(-h/l) = prod over columns of (rho + (1 - rho) [x_i = x'_i]), rho = exp(-1/l):
           per-column features [sqrt(rho), sqrt(1 - rho) e_category], tensor product over columns,
           f = w . phi(x), w ~ N(0, I)
The paper's own workloads (a 500-sample simulated logistic problem, Sec. 2.5, and the NMES data,
Sec. 2.6, which is not available here) are stood in for by these generators, with the paper's
sizes (N = 500, continuous / binary / ordinal covariates) where they apply.
"""
import numpy as np

DEFAULT_PRIOR_A = (2.0, 2.0)
DEFAULT_PRIOR_B = (2.0, 2.0)
DEFAULT_JITTER = 1e-6


def _kernel(kind, cols):
    return {"kind": kind, "cols": tuple(int(c) for c in cols), "jitter": DEFAULT_JITTER,
            "prior_a": DEFAULT_PRIOR_A, "prior_b": DEFAULT_PRIOR_B}


def _rff_draw(rng, X, lengthscale, amplitude, n_features=4096):
    W = rng.standard_normal((n_features, X.shape[1])) / lengthscale
    b = rng.uniform(0.0, 2.0 * np.pi, n_features)
    return np.sqrt(2.0 * amplitude / n_features) * np.cos(X @ W.T + b).sum(axis=1)


def _linear_draw(rng, X, amplitude, offset):
    w = rng.standard_normal(X.shape[1])
    w0 = rng.standard_normal()
    return np.sqrt(amplitude) * (X @ w + np.sqrt(offset) * w0)


def _overlap_draw(rng, X, amplitude, lengthscale, n_levels):
    rho = np.exp(-1.0 / lengthscale)
    cols = X.shape[1]
    feats = np.ones((X.shape[0], 1))
    for c in range(cols):
        phi = np.zeros((X.shape[0], n_levels + 1))
        phi[:, 0] = np.sqrt(rho)
        phi[np.arange(X.shape[0]), 1 + X[:, c].astype(int)] = np.sqrt(1.0 - rho)
        feats = (feats[:, :, None] * phi[:, None, :]).reshape(X.shape[0], -1)
    w = rng.standard_normal(feats.shape[1])
    return np.sqrt(amplitude) * feats @ w


def _bernoulli(rng, F):
    return (rng.uniform(size=F.shape) < 1.0 / (1.0 + np.exp(-F))).astype(np.float64)


def gp_classification(N, seed=0, lengthscale=0.5, amplitude=1.0):
    """GP binary classification: x ~ U[-1, 1]^2, SE kernel (log amplitude, log lengthscale),
    f_true from the GP at (lengthscale, amplitude), y ~ Bernoulli(sigmoid(f_true)).
    N = 50 gives d = 52; N = 400 gives d = 402."""
    rng = np.random.default_rng(seed)
    X = rng.uniform(-1.0, 1.0, (N, 2))
    f = _rff_draw(rng, X, lengthscale, amplitude)
    y = _bernoulli(rng, f)
    return {"X": X, "y": y, "lik": "bernoulli", "noise_var": 1.0,
            "kernels": [_kernel("se", (0, 1))], "sample_hypers": True, "u_fixed": None,
            "f_true": f}


def gp_regression(N, seed=0, lengthscale=0.5, amplitude=1.0, noise_var=0.1, sample_hypers=False):
    """Gaussian-likelihood GP regression on x ~ U[-1, 1]^2 (closed-form posterior when the
    hyperparameters are held fixed at u_fixed = (log amplitude, log lengthscale))."""
    rng = np.random.default_rng(seed)
    X = rng.uniform(-1.0, 1.0, (N, 2))
    f = _rff_draw(rng, X, lengthscale, amplitude)
    y = f + np.sqrt(noise_var) * rng.standard_normal(N)
    u_fixed = None if sample_hypers else np.array([np.log(amplitude), np.log(lengthscale)])
    return {"X": X, "y": y, "lik": "gaussian", "noise_var": noise_var,
            "kernels": [_kernel("se", (0, 1))], "sample_hypers": sample_hypers,
            "u_fixed": u_fixed, "f_true": f}


def propensity(N, seed=0, n_kernels=3):
    """Additive multiple-kernel propensity model (the NMES-like stand-in): 8 covariates,
    4 continuous ~ N(0,1) (cols 0-3), 2 binary ~ Bernoulli(0.5) (cols 4-5), 2 ordinal uniform on
    {0..4} (cols 6-7). Kernels, in order: SE on the continuous, linear on the binary,
    categorical-overlap on the ordinal (the first n_kernels of them). Treatment
    ~ Bernoulli(sigmoid(sum of the GP draws)) with every amplitude, lengthscale and offset 1."""
    rng = np.random.default_rng(seed)
    Xc = rng.standard_normal((N, 4))
    Xb = (rng.uniform(size=(N, 2)) < 0.5).astype(np.float64)
    Xo = rng.integers(0, 5, size=(N, 2)).astype(np.float64)
    X = np.concatenate([Xc, Xb, Xo], axis=1)
    draws = [_rff_draw(rng, Xc, 1.0, 1.0), _linear_draw(rng, Xb, 1.0, 1.0),
             _overlap_draw(rng, Xo, 1.0, 1.0, 5)]
    kernels = [_kernel("se", (0, 1, 2, 3)), _kernel("linear", (4, 5)), _kernel("overlap", (6, 7))]
    F = np.sum(draws[:n_kernels], axis=0)
    y = _bernoulli(rng, F)
    return {"X": X, "y": y, "lik": "bernoulli", "noise_var": 1.0,
            "kernels": kernels[:n_kernels], "sample_hypers": True, "u_fixed": None, "f_true": F}


def solin_logistic(D, N=500, seed=0, M=30, L=8.0, sd=1.5, bias=-0.5, n_linear=0):
    """The simulated logistic-regression data of Sec. 2.5 for the primal (reduced-rank) model:
    X ~ N(0, 1)^{N x D}; the true log-odds f*(x) = sum_k sum_{m=4..16} a*_km sin(pi m (x_k + L)/(2L))
    + b*, a*_km ~ N(0, c*/m), b* = -0.5, c* set so that the empirical SD of f* is 1.5; labels
    y ~ Bernoulli(sigmoid(f*)) coded {0, 1}. (The true function is drawn from the paper's own
    sinusoidal data-generating recipe; the model's features are evaluated separately by the
    sampler.) Optional linear covariates ~ N(0, 1) enter the truth with unit weights."""
    rng = np.random.default_rng(seed)
    Xg = rng.standard_normal((N, D))
    Xl = rng.standard_normal((N, n_linear))
    m = np.arange(1, M + 1)
    a = rng.standard_normal((D, M)) / np.sqrt(m)[None, :]
    a[:, (m < 4) | (m > 16)] = 0.0
    f0 = np.zeros(N)
    for k in range(D):
        f0 += np.sin(np.pi * m[None, :] * (Xg[:, k:k + 1] + L) / (2.0 * L)) @ a[k]
    f0 += Xl.sum(axis=1)
    f = f0 * (sd / f0.std()) + bias
    y = _bernoulli(rng, f)
    return {"model": "primal", "Xg": Xg, "Xl": Xl, "y": y, "M": M, "L": L, "lik": "bernoulli",
            "noise_var": 1.0, "bias_var": 1.0, "prior_a": (2.0, 2.0, 2.0), "prior_b": (2.0, 2.0, 2.0),
            "f_true": f}


def _sinusoid_draw(rng, X, M, L, sd):
    """sum_k sum_{m=4..16} a_km sin(pi m (x_k + L) / (2L)), a_km ~ N(0, c/m), scaled to SD sd (the
    data recipe of Sec. 2.5)."""
    m = np.arange(1, M + 1)
    a = rng.standard_normal((X.shape[1], M)) / np.sqrt(m)[None, :]
    a[:, (m < 4) | (m > 16)] = 0.0
    f = np.zeros(X.shape[0])
    for k in range(X.shape[1]):
        f += np.sin(np.pi * m[None, :] * (X[:, k:k + 1] + L) / (2.0 * L)) @ a[k]
    return f * (sd / f.std())


def meanvar_regression(D, N=500, seed=0, M=30, L=8.0, delta=0.05, n_linear=0):
    """Example 1 of Sec. 2.1 (covariate-dependent mean and variance, J = 2) on synthetic data in
    the layout of Sec. 2.6 (the NMES records are not available): X ~ N(0, 1)^{N x D}, true mean
    f1* (SD 1) and log-variance f2* (SD 0.7, mean log 0.3) drawn with the recipe of Sec. 2.5,
    y = f1* + sqrt(delta + exp f2*) eps, eps ~ N(0, 1). Optional linear covariates ~ N(0, 1) add
    to both functions with unit and 0.3 weights."""
    rng = np.random.default_rng(seed)
    Xg = rng.standard_normal((N, D))
    Xl = rng.standard_normal((N, n_linear))
    f1 = _sinusoid_draw(rng, Xg, M, L, 1.0) + Xl.sum(axis=1)
    f2 = _sinusoid_draw(rng, Xg, M, L, 0.7) + np.log(0.3) + 0.3 * Xl.sum(axis=1)
    y = f1 + np.sqrt(delta + np.exp(f2)) * rng.standard_normal(N)
    return {"model": "primal", "J": 2, "delta": delta, "Xg": Xg, "Xl": Xl, "y": y, "M": M, "L": L,
            "lik": "meanvar", "noise_var": 1.0, "bias_var": 1.0, "prior_a": (2.0, 2.0, 2.0),
            "prior_b": (2.0, 2.0, 2.0), "f_true": np.stack([f1, f2])}


def uneven_batch(n_problems=128, seed=0, n_min=32, n_max=512):
    """Problems of uneven dimension: N ~ U{n_min..n_max}, 1-3 kernels (SE, linear, overlap in that
    order) on the propensity covariates; problem i uses seed + i."""
    out = []
    for i in range(n_problems):
        rng = np.random.default_rng(seed + i)
        N = int(rng.integers(n_min, n_max + 1))
        nk = int(rng.integers(1, 4))
        out.append(propensity(N, seed=seed + i, n_kernels=nk))
    return out


def dims(problem):
    """(N, number of latent blocks or coefficients, d)."""
    if problem.get("model") == "primal":
        N = problem["Xg"].shape[0]
        P = problem["M"] * problem["Xg"].shape[1] + problem["Xl"].shape[1] + 1
        return N, P, problem.get("J", 1) * P + 3
    N = problem["X"].shape[0]
    n = len(problem["kernels"])
    return N, n, n * N + (2 * n if problem["sample_hypers"] else 0)


def initial_state(problem, n_chains):
    """f = 0 (a = 0, b = 0 for the primal model) and u = 0 (every hyperparameter 1) for every chain,
    as an (n_chains, d) array."""
    _, _, d = dims(problem)
    return np.zeros((n_chains, d))


def random_state(problem, n_chains, seed, f_scale=0.5, u_scale=0.3):
    """Random positions for parity tests: f ~ N(0, f_scale^2), u ~ N(0, u_scale^2)."""
    rng = np.random.default_rng(seed)
    _, _, d = dims(problem)
    q = f_scale * rng.standard_normal((n_chains, d))
    N, n, _ = dims(problem)
    if problem.get("model") == "primal":
        q[:, d - 3:] = u_scale * rng.standard_normal((n_chains, 3))
        return q
    if problem["sample_hypers"]:
        q[:, n * N:] = u_scale * rng.standard_normal((n_chains, 2 * n))
    return q


def random_momentum(problem, n_chains, seed):
    rng = np.random.default_rng(seed)
    _, _, d = dims(problem)
    return rng.standard_normal((n_chains, d))
