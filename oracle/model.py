"""Negative log posterior U(q) of the dual-form hierarchical GP model and its derivatives (oracle).

Model (Eq. data_likelihood with J = 1, Eq. BMKL additive kernels, Eq. hpar_prior):
  F = sum_k f_k,   f_k ~ N(0, K_k(u_k)),   y_m | F_m ~ likelihood,
  theta = exp(u) ~ InvGamma(a, b) on every hyperparameter (log-parametrised, Jacobian included),
  tempered posterior P_tau ∝ P(y | F)^tau * prior (Sec. "MC integration for BME"): tau scales the
  likelihood and all its derivatives only.

Coordinates q = (f_1[0:N], ..., f_n[0:N], u_1[0:2], ..., u_n[0:2]); d = nN + 2n, or d = nN when the
hyperparameters are held fixed.

U(q) = tau * sum_m l(F_m, y_m)
       + sum_k [ 1/2 f_k^T K_k^-1 f_k + 1/2 log|K_k| + N/2 log 2pi ]     (f^T K^-1 f = |L^-1 f|^2)
       - sum_{k,h} log p(u_kh),      log p(u) = a log b - lgamma(a) - a u - b exp(-u)

Likelihoods (exact negative log likelihoods):
  bernoulli (y in {0,1}):  l = softplus(F) - y F   (= log(1 + exp(-y~ F)), y~ = 2y - 1; Sec. 2.5)
  gaussian:                l = (y - F)^2 / (2 s2) + 1/2 log(2 pi s2)

The third derivatives are returned as slices dH_i = d/dq_i Hessian(q) (a d x d matrix per
coordinate); stacking all slices gives the full tensor the Betancourt formula contracts with
(Eq. Betancourt_formula). The hyperparameter terms the paper omits in Sec. 2.3 are written out
here in full.
"""
from contextlib import contextmanager
from dataclasses import dataclass, field
from math import lgamma, log, pi

import numpy as np
import scipy.linalg as sla

from .kernels import dK, kernel_derivs

LOG2PI = log(2.0 * pi)


@dataclass
class KernelSpec:
    kind: str
    cols: tuple
    jitter: float = 1e-6
    prior_a: tuple = (2.0, 2.0)
    prior_b: tuple = (2.0, 2.0)


@dataclass
class GPModel:
    X: np.ndarray
    y: np.ndarray
    kernels: list
    lik: str = "bernoulli"
    noise_var: float = 1.0
    sample_hypers: bool = True
    u_fixed: np.ndarray = field(default=None)

    @property
    def N(self):
        return self.X.shape[0]

    @property
    def n(self):
        return len(self.kernels)

    @property
    def P(self):
        return 2 * self.n if self.sample_hypers else 0

    @property
    def d(self):
        return self.n * self.N + self.P


def from_problem(problem):
    """GPModel from a workload dict (keys X, y, lik, noise_var, kernels, sample_hypers, u_fixed)."""
    ks = [KernelSpec(kind=k["kind"], cols=tuple(k["cols"]), jitter=k["jitter"],
                     prior_a=tuple(k["prior_a"]), prior_b=tuple(k["prior_b"]))
          for k in problem["kernels"]]
    return GPModel(X=np.asarray(problem["X"], dtype=np.float64),
                   y=np.asarray(problem["y"], dtype=np.float64), kernels=ks,
                   lik=problem["lik"], noise_var=problem["noise_var"],
                   sample_hypers=problem["sample_hypers"], u_fixed=problem["u_fixed"])


def split(model, q):
    """Latent blocks f (n x N) and hyperparameters u (n x 2)."""
    q = np.asarray(q, dtype=np.float64)
    N, n = model.N, model.n
    f = q[: n * N].reshape(n, N)
    if model.sample_hypers:
        u = q[n * N:].reshape(n, 2)
    else:
        u = np.asarray(model.u_fixed, dtype=np.float64).reshape(n, 2)
    return f, u


def f_index(model, k):
    return np.arange(k * model.N, (k + 1) * model.N)


def u_index(model, k, h):
    return model.n * model.N + 2 * k + h


def lik_derivs(model, F):
    """l, l', l'', l''' of the per-sample negative log likelihood at F."""
    y = np.asarray(model.y, dtype=np.float64)
    if model.lik == "bernoulli":
        s = 1.0 / (1.0 + np.exp(-F))
        l0 = np.logaddexp(0.0, F) - y * F
        return l0, s - y, s * (1.0 - s), s * (1.0 - s) * (1.0 - 2.0 * s)
    if model.lik == "gaussian":
        s2 = model.noise_var
        l0 = (y - F) ** 2 / (2.0 * s2) + 0.5 * np.log(2.0 * pi * s2)
        return l0, (F - y) / s2, np.full_like(F, 1.0 / s2), np.zeros_like(F)
    raise ValueError(model.lik)


_INVERSE = {"method": "lu"}


@contextmanager
def inverse_method(method):
    """Evaluate K^-1 and alpha with LAPACK's LU ('lu', the default) or Cholesky ('cholesky')
    routines. Both are backward stable; their difference measures how far cond(K) lets two valid
    FP64 evaluations of the same quantity drift apart (used to calibrate parity tolerances)."""
    old = _INVERSE["method"]
    _INVERSE["method"] = method
    try:
        yield
    finally:
        _INVERSE["method"] = old


class KernelState:
    """Per-kernel quantities at q: K and its u_1-derivatives, K^-1, alpha = K^-1 f."""

    def __init__(self, spec, Xk, f, u):
        self.mats = kernel_derivs(spec.kind, Xk, u, spec.jitter)
        K = self.mats[0]
        self.L = np.linalg.cholesky(K)
        if _INVERSE["method"] == "cholesky":
            cf = (self.L, True)
            self.Kinv = sla.cho_solve(cf, np.eye(len(f)), check_finite=False)
            self.alpha = sla.cho_solve(cf, f, check_finite=False)
        else:
            self.Kinv = np.linalg.inv(K)
            self.alpha = np.linalg.solve(K, f)
        self.Kinv = 0.5 * (self.Kinv + self.Kinv.T)
        self.logdet = 2.0 * np.sum(np.log(np.diag(self.L)))
        # f^T K^-1 f = |L^-1 f|^2 by forward substitution (backward stable; the product f . alpha
        # loses ~cond(K) u relative accuracy to cancellation)
        t = sla.solve_triangular(self.L, f, lower=True, check_finite=False)
        self.quad = float(t @ t)

    def d(self, *idx):
        return dK(self.mats, idx)


def _states(model, q):
    f, u = split(model, q)
    out = []
    for k, spec in enumerate(model.kernels):
        Xk = model.X[:, list(spec.cols)]
        out.append(KernelState(spec, Xk, f[k], u[k]))
    return f, u, out


def log_prior_u(a, b, u):
    """log density of u = log theta for theta ~ InvGamma(a, b) (Jacobian included)."""
    return a * log(b) - lgamma(a) - a * u - b * np.exp(-u)


def potential(model, q, tau=1.0):
    """U(q) = -log P_tau(q) (exact, all constants included)."""
    f, u, st = _states(model, q)
    F = f.sum(axis=0)
    l0, _, _, _ = lik_derivs(model, F)
    U = tau * np.sum(l0)
    for k, s in enumerate(st):
        U += 0.5 * s.quad + 0.5 * s.logdet + 0.5 * model.N * LOG2PI
    if model.sample_hypers:
        for k, spec in enumerate(model.kernels):
            for h in range(2):
                U -= log_prior_u(spec.prior_a[h], spec.prior_b[h], u[k, h])
    return float(U)


def gradient(model, q, tau=1.0):
    """dU/dq."""
    f, u, st = _states(model, q)
    F = f.sum(axis=0)
    _, l1, _, _ = lik_derivs(model, F)
    g = np.zeros(model.d)
    for k, s in enumerate(st):
        g[f_index(model, k)] = tau * l1 + s.alpha
        if model.sample_hypers:
            spec = model.kernels[k]
            for h in range(2):
                Kh = s.d(h)
                g[u_index(model, k, h)] = (-0.5 * s.alpha @ Kh @ s.alpha
                                           + 0.5 * np.trace(s.Kinv @ Kh)
                                           + spec.prior_a[h] - spec.prior_b[h] * np.exp(-u[k, h]))
    return g


def hessian(model, q, tau=1.0):
    """d^2 U / dq dq (symmetric d x d)."""
    f, u, st = _states(model, q)
    F = f.sum(axis=0)
    _, _, l2, _ = lik_derivs(model, F)
    d, N = model.d, model.N
    H = np.zeros((d, d))
    for a in range(model.n):
        for b in range(model.n):
            ia, ib = f_index(model, a), f_index(model, b)
            H[np.ix_(ia, ib)] += np.diag(tau * l2)
    for k, s in enumerate(st):
        ik = f_index(model, k)
        H[np.ix_(ik, ik)] += s.Kinv
        if not model.sample_hypers:
            continue
        spec = model.kernels[k]
        for h in range(2):
            col = -s.Kinv @ s.d(h) @ s.alpha
            j = u_index(model, k, h)
            H[ik, j] = col
            H[j, ik] = col
            for h2 in range(2):
                j2 = u_index(model, k, h2)
                Kh, Kh2, Khh = s.d(h), s.d(h2), s.d(h, h2)
                v = (s.alpha @ Kh @ s.Kinv @ Kh2 @ s.alpha
                     - 0.5 * s.alpha @ Khh @ s.alpha
                     + 0.5 * np.trace(s.Kinv @ Khh)
                     - 0.5 * np.trace(s.Kinv @ Kh @ s.Kinv @ Kh2))
                if h == h2:
                    v += spec.prior_b[h] * np.exp(-u[k, h])
                H[j, j2] = v
    return H


class ThirdDerivatives:
    """The third derivatives d/dq_i H(q), one d x d slice per coordinate i (Sec. 2.3).

    Blocks (same kernel k for every term that involves K_k; S_j = K^-1 K_j, gamma_j = S_j alpha):
      d/df_{c,m} H[f_a, f_b]   = tau l'''(F_m) e_m e_m^T                    (all a, b)
      d/du_j     H[f_k, f_k]   = -K^-1 K_j K^-1
      d/du_j     H[f_k, u_l]   = K^-1 (K_j K^-1 K_l + K_l K^-1 K_j - K_jl) alpha
                               (= d/df_k H[u_j, u_l] by symmetry of third derivatives)
      d/du_j     H[u_k, u_l]   = -g_j K_k g_l - g_k K_j g_l - g_k K_l g_j
                                 + (K_jk a) g_l + g_k (K_jl a) + (K_kl a) g_j - 1/2 a K_jkl a
                                 - 1/2 tr(S_j K^-1 K_kl) + 1/2 tr(K^-1 K_jkl)
                                 + 1/2 tr(S_j S_k S_l) + 1/2 tr(S_k S_j S_l)
                                 - 1/2 tr(K^-1 K_jk S_l) - 1/2 tr(S_k K^-1 K_jl)
                                 - [j = k = l] b exp(-u)
    """

    def __init__(self, model, q, tau=1.0):
        self.model = model
        self.tau = tau
        self.f, self.u, self.st = _states(model, q)
        F = self.f.sum(axis=0)
        _, _, _, self.l3 = lik_derivs(model, F)
        self._cache = {}

    def _fuu_vector(self, k, h, h2):
        """K^-1 (K_h K^-1 K_h2 + K_h2 K^-1 K_h - K_hh2) alpha (an N-vector), cached per q."""
        key = ("fuu", k, h, h2)
        if key not in self._cache:
            s = self.st[k]
            Kh, Kh2, Khh = s.d(h), s.d(h2), s.d(h, h2)
            M = Kh @ s.Kinv @ Kh2 + Kh2 @ s.Kinv @ Kh - Khh
            self._cache[key] = s.Kinv @ (M @ s.alpha)
        return self._cache[key]

    def _A(self, k, h):
        """K^-1 K_h K^-1, cached per q."""
        key = ("A", k, h)
        if key not in self._cache:
            s = self.st[k]
            self._cache[key] = s.Kinv @ s.d(h) @ s.Kinv
        return self._cache[key]

    def _uuu(self, k, j, kk, l):
        s = self.st[k]
        a, Ki = s.alpha, s.Kinv
        Kj, Kk, Kl = s.d(j), s.d(kk), s.d(l)
        gj, gk, gl = Ki @ Kj @ a, Ki @ Kk @ a, Ki @ Kl @ a
        Sj, Sk, Sl = Ki @ Kj, Ki @ Kk, Ki @ Kl
        Kjk, Kjl, Kkl, Kjkl = s.d(j, kk), s.d(j, l), s.d(kk, l), s.d(j, kk, l)
        v = (-gj @ Kk @ gl - gk @ Kj @ gl - gk @ Kl @ gj
             + (Kjk @ a) @ gl + gk @ (Kjl @ a) + (Kkl @ a) @ gj
             - 0.5 * a @ Kjkl @ a
             - 0.5 * np.trace(Sj @ Ki @ Kkl) + 0.5 * np.trace(Ki @ Kjkl)
             + 0.5 * np.trace(Sj @ Sk @ Sl) + 0.5 * np.trace(Sk @ Sj @ Sl)
             - 0.5 * np.trace(Ki @ Kjk @ Sl) - 0.5 * np.trace(Sk @ Ki @ Kjl))
        if j == kk == l:
            spec = self.model.kernels[k]
            v -= spec.prior_b[j] * np.exp(-self.u[k, j])
        return v

    def slice(self, i):
        """d/dq_i of the Hessian, as a dense d x d matrix."""
        m_ = self.model
        N, n, d = m_.N, m_.n, m_.d
        D = np.zeros((d, d))
        if i < n * N:
            c, m = divmod(i, N)
            for a in range(n):
                for b in range(n):
                    D[a * N + m, b * N + m] += self.tau * self.l3[m]
            if m_.sample_hypers:
                ic = f_index(m_, c)
                for h in range(2):
                    col = -self._A(c, h)[:, m]
                    j = u_index(m_, c, h)
                    D[ic, j] += col
                    D[j, ic] += col
                    for h2 in range(2):
                        D[j, u_index(m_, c, h2)] += self._fuu_vector(c, h, h2)[m]
            return D
        k, jh = divmod(i - n * N, 2)
        ik = f_index(m_, k)
        D[np.ix_(ik, ik)] = -self._A(k, jh)
        for h in range(2):
            col = self._fuu_vector(k, jh, h)
            j = u_index(m_, k, h)
            D[ik, j] = col
            D[j, ik] = col
            for h2 in range(2):
                D[j, u_index(m_, k, h2)] = self._uuu(k, jh, h, h2)
        return D

    def tensor(self):
        """All slices stacked: T[i] = d/dq_i Hessian (d x d x d)."""
        return np.stack([self.slice(i) for i in range(self.model.d)])
