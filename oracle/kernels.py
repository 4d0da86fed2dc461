"""Kernel matrices of the additive GP prior and their hyperparameter derivatives (oracle).

Each latent block f_k ~ N(0, K_k(u_k)) (Eq. BMKL, one GP per kernel; dual/latent-value form).
Hyperparameters are log-parametrised, u_k = (log c, log theta):

  SE       k(x, x') = c * (exp(-|x - x'|^2 / (2 theta^2)) + delta [x == x'])   theta = lengthscale
  linear   k(x, x') = c * (x . x' + theta + delta [x == x'])                   theta = offset
  overlap  k(x, x') = c * (exp(-h(x, x') / theta) + delta [x == x'])         h = # mismatching cols

"[x == x']" is the diagonal (same sample index), i.e. a jitter delta*c*I. Because every kernel is
c * (...), each derivative with respect to u_0 = log c returns the same matrix, so only the
derivatives with respect to u_1 = log theta are needed: D_m = d^m K / d u_1^m, m = 0..3 (D_0 = K,
jitter included only in D_0).
"""
import numpy as np

KINDS = ("se", "linear", "overlap")


def kernel_derivs(kind, Xk, u, jitter):
    """Return [K, D1, D2, D3] (each N x N, float64) for kernel `kind` on columns Xk (N x p)."""
    Xk = np.asarray(Xk, dtype=np.float64)
    N = Xk.shape[0]
    c = np.exp(u[0])
    th = np.exp(u[1])
    eye = np.eye(N)
    if kind == "se":
        diff = Xk[:, None, :] - Xk[None, :, :]
        sq = np.sum(diff * diff, axis=2)
        r = sq / (th * th)
        E = np.exp(-0.5 * r)
        K = c * (E + jitter * eye)
        D1 = c * E * r
        D2 = c * E * (r * r - 2.0 * r)
        D3 = c * E * (r ** 3 - 6.0 * r * r + 4.0 * r)
    elif kind == "linear":
        G = Xk @ Xk.T
        K = c * (G + th + jitter * eye)
        D1 = np.full((N, N), c * th)
        D2 = D1.copy()
        D3 = D1.copy()
    elif kind == "overlap":
        h = np.sum(Xk[:, None, :] != Xk[None, :, :], axis=2).astype(np.float64)
        s = h / th
        E = np.exp(-s)
        K = c * (E + jitter * eye)
        D1 = c * E * s
        D2 = c * E * (s * s - s)
        D3 = c * E * (s ** 3 - 3.0 * s * s + s)
    else:
        raise ValueError(f"unknown kernel kind {kind!r}")
    return [K, D1, D2, D3]


def dK(mats, idx):
    """Mixed derivative d^|idx| K / d u_idx[0] ... for a tuple of hyper indices in {0, 1}.

    Derivatives in u_0 = log c leave c * (...) unchanged, so only the number of u_1 indices
    matters."""
    return mats[sum(1 for i in idx if i == 1)]
