"""Primal (reduced-rank) hierarchical GP model of the paper's experiments, and its derivatives
(oracle; test infrastructure only, never called by the product path).

Model (Eq. data_likelihood, Eq. BMKL, Eq. Solin_representation, Eq. hpar_prior; the reduced-rank
appendix for the features and the spectral weights; Sec. 2.5 and 2.6 for the sizes):
  F_ji = sum_{k < Dg} sum_{m=1..M} a_jkm phi_m(Xg_ik) + sum_{l < Dl} a_jl Xl_il + b_j,  j < J
  phi_m(x)  = sin(pi m (x + L) / (2 L))          (the appendix's 1/L prefactor dropped, as there)
  a_jkm ~ N(0, c_g V_m(s_g)),  V_m(s) = sqrt(pi s) exp(-pi^2 m^2 s / (16 L^2))
        (the spectral density sqrt(pi s) exp(-s w^2 / 4) of k(r) = exp(-r^2 / s) at w = pi m / (2L);
         the appendix prints pi m^2 s in the exponent, the density gives pi^2 m^2 s)
  a_jl ~ N(0, c_l)   (linear kernels, V = 1),      b_j ~ N(0, Sigma)
  c_g, s_g, c_l ~ InvGamma(alpha, beta), one set shared by every function (Sec. 2.1), sampled as
  u = log(theta) with the Jacobian.
J = 1: a Bernoulli-logit or Gaussian likelihood on F_1. J = 2: Example 1, the covariate-dependent
mean and variance, y_i ~ N(F_1i, delta + exp(F_2i)) with delta fixed.
Coordinates q = (a_1.. (k-major), a_1l, b_1, [the same for j = 2], u_cg, u_sg, u_cl);
d = J P + 3 with P = M Dg + Dl + 1 (= 30 D + 4 for the simulated data of Sec. 2.5: D Gaussian
kernels, no linear one, c_l then only meets its prior).

U(q) = tau sum_i l(F_.i, y_i) + sum_jkm E(a_jkm, h_m) + sum_jl E(a_jl, -u_cl) + sum_j b_j^2 / (2 Sigma)
       + J P / 2 log 2 pi + J / 2 log Sigma - sum_theta log p(u_theta)
with E(a, h) = 1/2 a^2 e^h - 1/2 h and h_m(u) = -log(c_g V_m) = -u_cg - 1/2 log pi - 1/2 u_sg +
kappa_m e^{u_sg}, kappa_m = pi^2 m^2 / (16 L^2).

Derivatives follow from the chain rule through h: with E_a = a e^h, E_aa = e^h, E_h = 1/2 a^2 e^h
- 1/2, E_ah = a e^h, E_hh = 1/2 a^2 e^h, E_aah = e^h, E_ahh = a e^h, E_hhh = 1/2 a^2 e^h, and h_j,
h_jk, h_jkl the derivatives of h in (u_cg, u_sg) (h_cg = -1; h_sg = -1/2 + kappa e^u_sg;
h_sg,sg = h_sg,sg,sg = kappa e^u_sg; the rest 0). The likelihood part of the Hessian is
Phi^T diag(tau l_jk) Phi per block (j, k) and of the third derivatives
sum_i tau l_jkl,i phi_i phi_i phi_i (Sec. 2.3).

Mean/variance likelihood (J = 2): with r = y - F_1, w = e^{F_2}, v = delta + w, rho = w / v and
z = r^2 / v, l = z / 2 + log(2 pi v) / 2 and
  l_1 = -r / v,              l_2 = rho (1 - z) / 2,
  l_11 = 1 / v,              l_12 = r rho / v,          l_22 = rho A / 2,  A = (1 - rho)(1 - z) + z rho,
  l_111 = 0,  l_112 = -rho / v,  l_122 = r rho (1 - 2 rho) / v,
  l_222 = [rho (1 - rho) A + rho (-rho (1 - rho) + z rho + 2 z rho (1 - 2 rho))] / 2
(d rho / d F_2 = rho (1 - rho), d z / d F_2 = -z rho).
"""
from dataclasses import dataclass
from math import lgamma, log, pi

import numpy as np

from .model import lik_derivs

LOG2PI = log(2.0 * pi)


@dataclass
class PrimalModel:
    Xg: np.ndarray              # N x Dg covariates with a Gaussian kernel each
    Xl: np.ndarray              # N x Dl covariates with a linear kernel each
    y: np.ndarray
    M: int = 30
    L: float = 8.0
    lik: str = "bernoulli"      # J = 1: "bernoulli" | "gaussian"; J = 2: "meanvar"
    noise_var: float = 1.0
    bias_var: float = 1.0       # Sigma
    prior_a: tuple = (2.0, 2.0, 2.0)   # (c_g, s_g, c_l)
    prior_b: tuple = (2.0, 2.0, 2.0)
    J: int = 1
    delta: float = 0.0          # the fixed variance floor of the mean/variance model

    @property
    def N(self):
        return self.Xg.shape[0]

    @property
    def Dg(self):
        return self.Xg.shape[1]

    @property
    def Dl(self):
        return self.Xl.shape[1]

    @property
    def P(self):
        """Number of coefficients of one function (a_km, a_l, b)."""
        return self.M * self.Dg + self.Dl + 1

    @property
    def d(self):
        return self.J * self.P + 3


def from_problem(problem):
    """PrimalModel from a workload dict (keys Xg, Xl, y, M, L, lik, noise_var, bias_var, prior_a,
    prior_b, and J, delta for the mean/variance model)."""
    return PrimalModel(Xg=np.asarray(problem["Xg"], dtype=np.float64),
                       Xl=np.asarray(problem["Xl"], dtype=np.float64).reshape(len(problem["y"]), -1),
                       y=np.asarray(problem["y"], dtype=np.float64), M=problem["M"], L=problem["L"],
                       lik=problem["lik"], noise_var=problem["noise_var"], bias_var=problem["bias_var"],
                       prior_a=tuple(problem["prior_a"]), prior_b=tuple(problem["prior_b"]),
                       J=int(problem.get("J", 1)), delta=float(problem.get("delta", 0.0)))


def features(model):
    """Phi (N x P): phi_m(Xg_ik) in column k M + m - 1, then Xl_il, then 1 (the bias)."""
    m = np.arange(1, model.M + 1)
    cols = [np.sin(pi * m[None, :] * (model.Xg[:, k:k + 1] + model.L) / (2.0 * model.L))
            for k in range(model.Dg)]
    return np.concatenate(cols + [model.Xl, np.ones((model.N, 1))], axis=1)


def spectral_weights(model, u_sg):
    """V_m(s_g) for m = 1..M."""
    m = np.arange(1, model.M + 1)
    s = np.exp(u_sg)
    return np.sqrt(pi * s) * np.exp(-pi * pi * m * m * s / (16.0 * model.L ** 2))


def _kappa(model):
    m = np.arange(1, model.M + 1)
    return pi * pi * m * m / (16.0 * model.L ** 2)


def split(model, q):
    """Coefficients (J x P) and hyperparameters (3)."""
    q = np.asarray(q, dtype=np.float64)
    JP = model.J * model.P
    return q[:JP].reshape(model.J, model.P), q[JP:JP + 3]


def data_derivs(model, F):
    """Per-sample negative log likelihood and its derivatives in the latent values F (J x N):
    (l, [l_j], {(j, k): l_jk}, {(j, k, l): l_jkl}) with sorted index tuples."""
    if model.J == 1:
        l0, l1, l2, l3 = lik_derivs(model, F[0])
        return l0, [l1], {(0, 0): l2}, {(0, 0, 0): l3}
    if model.J != 2 or model.lik != "meanvar":
        raise ValueError("J = 2 needs the mean/variance likelihood")
    y = np.asarray(model.y, dtype=np.float64)
    r = y - F[0]
    w = np.exp(F[1])
    v = model.delta + w
    rho = w / v
    z = r * r / v
    A = (1.0 - rho) * (1.0 - z) + z * rho
    l0 = 0.5 * z + 0.5 * np.log(2.0 * pi * v)
    l1 = [-r / v, 0.5 * rho * (1.0 - z)]
    l2 = {(0, 0): 1.0 / v, (0, 1): r * rho / v, (1, 1): 0.5 * rho * A}
    dA = -rho * (1.0 - rho) + z * rho + 2.0 * z * rho * (1.0 - 2.0 * rho)
    l3 = {(0, 0, 0): np.zeros_like(r), (0, 0, 1): -rho / v, (0, 1, 1): r * rho * (1.0 - 2.0 * rho) / v,
          (1, 1, 1): 0.5 * (rho * (1.0 - rho) * A + rho * dA)}
    return l0, l1, l2, l3


def _h(model, u):
    """h_m = -log(c_g V_m) and its derivatives in (u_cg, u_sg): h (M,), dh (M, 2), d2h (M, 2, 2),
    d3h (M, 2, 2, 2)."""
    kap = _kappa(model)
    es = kap * np.exp(u[1])
    h = -u[0] - 0.5 * log(pi) - 0.5 * u[1] + es
    M = model.M
    dh = np.zeros((M, 2))
    dh[:, 0] = -1.0
    dh[:, 1] = -0.5 + es
    d2h = np.zeros((M, 2, 2))
    d2h[:, 1, 1] = es
    d3h = np.zeros((M, 2, 2, 2))
    d3h[:, 1, 1, 1] = es
    return h, dh, d2h, d3h


def _hyper_terms(model, u):
    """-sum log p(u) and its first three derivatives (diagonal)."""
    a, b = np.asarray(model.prior_a), np.asarray(model.prior_b)
    e = b * np.exp(-u)
    v = -np.sum([a[j] * log(b[j]) - lgamma(a[j]) for j in range(3)]) + np.sum(a * u + e)
    return v, a - e, e, -e


def _data(model, q):
    w, u = split(model, q)
    Phi = features(model)
    F = w @ Phi.T                                            # J x N
    return w, u, Phi, data_derivs(model, F)


def potential(model, q, tau=1.0):
    w, u, Phi, (l0, _, _, _) = _data(model, q)
    Dg, M, Dl = model.Dg, model.M, model.Dl
    h, _, _, _ = _h(model, u)
    U = tau * np.sum(l0)
    for j in range(model.J):
        a = w[j, :M * Dg].reshape(Dg, M)
        al = w[j, M * Dg:M * Dg + Dl]
        b = w[j, -1]
        U += np.sum(0.5 * a * a * np.exp(h)[None, :] - 0.5 * h[None, :])
        U += np.sum(0.5 * al * al * np.exp(-u[2]) + 0.5 * u[2])
        U += 0.5 * b * b / model.bias_var + 0.5 * log(model.bias_var)
    U += 0.5 * model.J * model.P * LOG2PI
    U += _hyper_terms(model, u)[0]
    return float(U)


def gradient(model, q, tau=1.0):
    w, u, Phi, (_, l1, _, _) = _data(model, q)
    Dg, M, P, Dl, J = model.Dg, model.M, model.P, model.Dl, model.J
    g = np.zeros(model.d)
    h, dh, _, _ = _h(model, u)
    eh = np.exp(h)
    el = np.exp(-u[2])
    for j in range(J):
        o = j * P
        g[o:o + P] = Phi.T @ (tau * l1[j])
        a = w[j, :M * Dg].reshape(Dg, M)
        g[o:o + M * Dg] += (a * eh[None, :]).ravel()
        Eh = 0.5 * a * a * eh[None, :] - 0.5
        g[J * P:J * P + 2] += np.einsum("km,mj->j", Eh, dh)
        al = w[j, M * Dg:M * Dg + Dl]
        g[o + M * Dg:o + M * Dg + Dl] += al * el
        g[J * P + 2] += np.sum(-0.5 * al * al * el + 0.5)
        g[o + P - 1] += w[j, -1] / model.bias_var
    g[J * P:] += _hyper_terms(model, u)[1]
    return g


def hessian(model, q, tau=1.0):
    w, u, Phi, (_, _, l2, _) = _data(model, q)
    Dg, M, P, Dl, J = model.Dg, model.M, model.P, model.Dl, model.J
    H = np.zeros((model.d, model.d))
    for (j, k), ljk in l2.items():
        B = Phi.T @ (tau * ljk[:, None] * Phi)
        H[j * P:(j + 1) * P, k * P:(k + 1) * P] = B
        H[k * P:(k + 1) * P, j * P:(j + 1) * P] = B.T
    h, dh, d2h, _ = _h(model, u)
    eh = np.exp(h)
    iu = [J * P, J * P + 1]
    el = np.exp(-u[2])
    for jf in range(J):
        o = jf * P
        a = w[jf, :M * Dg].reshape(Dg, M)
        for k in range(Dg):
            for m in range(M):
                i = o + k * M + m
                H[i, i] += eh[m]                                  # E_aa
                for j in range(2):
                    v = a[k, m] * eh[m] * dh[m, j]                # E_ah h_j
                    H[i, iu[j]] += v
                    H[iu[j], i] += v
                Eh = 0.5 * a[k, m] ** 2 * eh[m] - 0.5
                Ehh = 0.5 * a[k, m] ** 2 * eh[m]
                for j in range(2):
                    for j2 in range(2):
                        H[iu[j], iu[j2]] += Ehh * dh[m, j] * dh[m, j2] + Eh * d2h[m, j, j2]
        al = w[jf, M * Dg:M * Dg + Dl]
        for l in range(Dl):
            i = o + M * Dg + l
            H[i, i] += el
            H[i, J * P + 2] += -al[l] * el
            H[J * P + 2, i] += -al[l] * el
        H[J * P + 2, J * P + 2] += np.sum(0.5 * al * al * el)
        H[o + P - 1, o + P - 1] += 1.0 / model.bias_var
    H[J * P:, J * P:] += np.diag(_hyper_terms(model, u)[2])
    return H


class ThirdDerivatives:
    """d/dq_i of the Hessian for every coordinate i (d x d x d), term by term as in the module
    docstring: the likelihood part on the coefficients, the per-coefficient prior parts on
    (a_jkm, u_cg, u_sg) and (a_jl, u_cl), and the diagonal hyperprior part."""

    def __init__(self, model, q, tau=1.0):
        self.model, self.q, self.tau = model, np.asarray(q, dtype=np.float64), tau

    def tensor(self):
        model, tau = self.model, self.tau
        w, u, Phi, (_, _, _, l3) = _data(model, self.q)
        Dg, M, P, Dl, d, J = model.Dg, model.M, model.P, model.Dl, model.d, model.J
        T = np.zeros((d, d, d))
        for (j, k, l), ljkl in l3.items():
            B = np.einsum("n,ni,nj,nk->ijk", tau * ljkl, Phi, Phi, Phi)
            for (a, b, c) in {(j, k, l), (j, l, k), (k, j, l), (k, l, j), (l, j, k), (l, k, j)}:
                T[a * P:(a + 1) * P, b * P:(b + 1) * P, c * P:(c + 1) * P] = B
        h, dh, d2h, d3h = _h(model, u)
        eh = np.exp(h)
        JP = J * P
        el = np.exp(-u[2])
        for jf in range(J):
            o = jf * P
            a = w[jf, :M * Dg].reshape(Dg, M)
            for k in range(Dg):
                for m in range(M):
                    x = a[k, m]
                    E = {"aah": eh[m], "ahh": x * eh[m], "hhh": 0.5 * x * x * eh[m], "ah": x * eh[m],
                         "hh": 0.5 * x * x * eh[m], "h": 0.5 * x * x * eh[m] - 0.5}
                    # local variables: 0 = a_jkm, 1 = u_cg, 2 = u_sg
                    idx = [o + k * M + m, JP, JP + 1]
                    t = np.zeros((3, 3, 3))
                    hj, hjk, hjkl = dh[m], d2h[m], d3h[m]
                    for j in range(2):
                        t[0, 0, 1 + j] = E["aah"] * hj[j]
                        for j2 in range(2):
                            t[0, 1 + j, 1 + j2] = E["ahh"] * hj[j] * hj[j2] + E["ah"] * hjk[j, j2]
                            for j3 in range(2):
                                t[1 + j, 1 + j2, 1 + j3] = (
                                    E["hhh"] * hj[j] * hj[j2] * hj[j3]
                                    + E["hh"] * (hjk[j, j2] * hj[j3] + hjk[j, j3] * hj[j2] + hjk[j2, j3] * hj[j])
                                    + E["h"] * hjkl[j, j2, j3])
                    # symmetrise the entries written with a sorted leading index
                    for p in range(3):
                        for r in range(3):
                            for s in range(3):
                                key = tuple(sorted((p, r, s)))
                                T[idx[p], idx[r], idx[s]] += t[key]
            al = w[jf, M * Dg:M * Dg + Dl]
            for l in range(Dl):
                # E(a, h) with h = -u_cl: h_j = -1, higher derivatives 0
                x = al[l]
                vals = {(0, 0, 1): el * -1.0, (0, 1, 1): x * el, (1, 1, 1): -0.5 * x * x * el}
                idx = [o + M * Dg + l, JP + 2]
                for p in range(2):
                    for r in range(2):
                        for s in range(2):
                            key = tuple(sorted((p, r, s)))
                            if key in vals:
                                T[idx[p], idx[r], idx[s]] += vals[key]
        t3 = _hyper_terms(model, u)[3]
        for j in range(3):
            T[JP + j, JP + j, JP + j] += t3[j]
        return T

    def slice(self, i):
        return self.tensor()[i]
