"""Primal (reduced-rank) hierarchical GP model of the paper's experiments, and its derivatives
(oracle; test infrastructure only, never called by the product path).

Model (Eq. data_likelihood with J = 1, Eq. BMKL, Eq. Solin_representation, Eq. hpar_prior; the
reduced-rank appendix for the features and the spectral weights; Sec. 2.5 for the sizes):
  F_i = sum_{k < Dg} sum_{m=1..M} a_km phi_m(Xg_ik) + sum_{l < Dl} a_l Xl_il + b
  phi_m(x)  = sin(pi m (x + L) / (2 L))          (the appendix's 1/L prefactor dropped, as there)
  a_km ~ N(0, c_g V_m(s_g)),  V_m(s) = sqrt(pi s) exp(-pi^2 m^2 s / (16 L^2))
        (the spectral density sqrt(pi s) exp(-s w^2 / 4) of k(r) = exp(-r^2 / s) at w = pi m / (2L);
         the appendix prints pi m^2 s in the exponent, the density gives pi^2 m^2 s)
  a_l  ~ N(0, c_l)   (linear kernels, V = 1),      b ~ N(0, Sigma)
  c_g, s_g, c_l ~ InvGamma(alpha, beta), sampled as u = log(theta) with the Jacobian.
Coordinates q = (a_km (k-major), a_l, b, u_cg, u_sg, u_cl); d = M Dg + Dl + 4 (= 30 D + 4 for the
simulated data of Sec. 2.5: D Gaussian kernels, no linear one, c_l then only meets its prior).

U(q) = tau sum_i l(F_i, y_i) + sum_km E(a_km, h_m) + sum_l E(a_l, -u_cl) + b^2 / (2 Sigma)
       + (number of coefficients + 1)/2 log 2 pi + 1/2 log Sigma - sum_theta log p(u_theta)
with E(a, h) = 1/2 a^2 e^h - 1/2 h and h_m(u) = -log(c_g V_m) = -u_cg - 1/2 log pi - 1/2 u_sg +
kappa_m e^{u_sg}, kappa_m = pi^2 m^2 / (16 L^2).

Derivatives follow from the chain rule through h: with E_a = a e^h, E_aa = e^h, E_h = 1/2 a^2 e^h
- 1/2, E_ah = a e^h, E_hh = 1/2 a^2 e^h, E_aah = e^h, E_ahh = a e^h, E_hhh = 1/2 a^2 e^h, and h_j,
h_jk, h_jkl the derivatives of h in (u_cg, u_sg) (h_cg = -1; h_sg = -1/2 + kappa e^u_sg;
h_sg,sg = h_sg,sg,sg = kappa e^u_sg; the rest 0). The likelihood part of the Hessian is
Phi^T diag(tau l'') Phi and of the third derivatives sum_i tau l'''_i phi_i phi_i phi_i (Sec. 2.3).
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
    lik: str = "bernoulli"
    noise_var: float = 1.0
    bias_var: float = 1.0       # Sigma
    prior_a: tuple = (2.0, 2.0, 2.0)   # (c_g, s_g, c_l)
    prior_b: tuple = (2.0, 2.0, 2.0)

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
        """Number of coefficients (a_km, a_l, b)."""
        return self.M * self.Dg + self.Dl + 1

    @property
    def d(self):
        return self.P + 3


def from_problem(problem):
    """PrimalModel from a workload dict (keys Xg, Xl, y, M, L, lik, noise_var, bias_var, prior_a,
    prior_b)."""
    return PrimalModel(Xg=np.asarray(problem["Xg"], dtype=np.float64),
                       Xl=np.asarray(problem["Xl"], dtype=np.float64).reshape(len(problem["y"]), -1),
                       y=np.asarray(problem["y"], dtype=np.float64), M=problem["M"], L=problem["L"],
                       lik=problem["lik"], noise_var=problem["noise_var"], bias_var=problem["bias_var"],
                       prior_a=tuple(problem["prior_a"]), prior_b=tuple(problem["prior_b"]))


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
    q = np.asarray(q, dtype=np.float64)
    P = model.P
    return q[:P], q[P:P + 3]


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


def potential(model, q, tau=1.0):
    w, u = split(model, q)
    Phi = features(model)
    l0, _, _, _ = lik_derivs(model, Phi @ w)
    Dg, M = model.Dg, model.M
    a = w[:M * Dg].reshape(Dg, M)
    al = w[M * Dg:M * Dg + model.Dl]
    b = w[-1]
    h, _, _, _ = _h(model, u)
    U = tau * np.sum(l0)
    U += np.sum(0.5 * a * a * np.exp(h)[None, :] - 0.5 * h[None, :])
    U += np.sum(0.5 * al * al * np.exp(-u[2]) + 0.5 * u[2])
    U += 0.5 * b * b / model.bias_var + 0.5 * log(model.bias_var)
    U += 0.5 * (model.P) * LOG2PI
    U += _hyper_terms(model, u)[0]
    return float(U)


def gradient(model, q, tau=1.0):
    w, u = split(model, q)
    Phi = features(model)
    _, l1, _, _ = lik_derivs(model, Phi @ w)
    Dg, M, P = model.Dg, model.M, model.P
    g = np.zeros(model.d)
    g[:P] = Phi.T @ (tau * l1)
    a = w[:M * Dg].reshape(Dg, M)
    h, dh, _, _ = _h(model, u)
    eh = np.exp(h)
    g[:M * Dg] += (a * eh[None, :]).ravel()
    Eh = 0.5 * a * a * eh[None, :] - 0.5                     # (Dg, M)
    g[P:P + 2] += np.einsum("km,mj->j", Eh, dh)
    al = w[M * Dg:M * Dg + model.Dl]
    el = np.exp(-u[2])
    g[M * Dg:M * Dg + model.Dl] += al * el
    g[P + 2] += np.sum(-0.5 * al * al * el + 0.5)
    g[P - 1] += w[-1] / model.bias_var
    g[P:] += _hyper_terms(model, u)[1]
    return g


def hessian(model, q, tau=1.0):
    w, u = split(model, q)
    Phi = features(model)
    _, _, l2, _ = lik_derivs(model, Phi @ w)
    Dg, M, P, Dl = model.Dg, model.M, model.P, model.Dl
    H = np.zeros((model.d, model.d))
    H[:P, :P] = Phi.T @ (tau * l2[:, None] * Phi)
    a = w[:M * Dg].reshape(Dg, M)
    h, dh, d2h, _ = _h(model, u)
    eh = np.exp(h)
    iu = [P, P + 1]
    for k in range(Dg):
        for m in range(M):
            i = k * M + m
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
    al = w[M * Dg:M * Dg + Dl]
    el = np.exp(-u[2])
    for l in range(Dl):
        i = M * Dg + l
        H[i, i] += el
        H[i, P + 2] += -al[l] * el
        H[P + 2, i] += -al[l] * el
    H[P + 2, P + 2] += np.sum(0.5 * al * al * el)
    H[P - 1, P - 1] += 1.0 / model.bias_var
    H[P:, P:] += np.diag(_hyper_terms(model, u)[2])
    return H


class ThirdDerivatives:
    """d/dq_i of the Hessian for every coordinate i (d x d x d), term by term as in the module
    docstring: the likelihood part on the coefficients, the per-coefficient prior parts on
    (a_km, u_cg, u_sg) and (a_l, u_cl), and the diagonal hyperprior part."""

    def __init__(self, model, q, tau=1.0):
        self.model, self.q, self.tau = model, np.asarray(q, dtype=np.float64), tau

    def tensor(self):
        model, tau = self.model, self.tau
        w, u = split(model, self.q)
        Phi = features(model)
        _, _, _, l3 = lik_derivs(model, Phi @ w)
        Dg, M, P, Dl, d = model.Dg, model.M, model.P, model.Dl, model.d
        T = np.zeros((d, d, d))
        T[:P, :P, :P] = np.einsum("n,ni,nj,nk->ijk", tau * l3, Phi, Phi, Phi)
        a = w[:M * Dg].reshape(Dg, M)
        h, dh, d2h, d3h = _h(model, u)
        eh = np.exp(h)
        for k in range(Dg):
            for m in range(M):
                x = a[k, m]
                E = {"aah": eh[m], "ahh": x * eh[m], "hhh": 0.5 * x * x * eh[m], "ah": x * eh[m],
                     "hh": 0.5 * x * x * eh[m], "h": 0.5 * x * x * eh[m] - 0.5}
                # local variables: 0 = a_km, 1 = u_cg, 2 = u_sg
                idx = [k * M + m, P, P + 1]
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
        al = w[M * Dg:M * Dg + Dl]
        el = np.exp(-u[2])
        for l in range(Dl):
            # E(a, h) with h = -u_cl: h_j = -1, higher derivatives 0
            x = al[l]
            vals = {(0, 0, 1): el * -1.0, (0, 1, 1): x * el, (1, 1, 1): -0.5 * x * x * el}
            idx = [M * Dg + l, P + 2]
            for p in range(2):
                for r in range(2):
                    for s in range(2):
                        key = tuple(sorted((p, r, s)))
                        if key in vals:
                            T[idx[p], idx[r], idx[s]] += vals[key]
        t3 = _hyper_terms(model, u)[3]
        for j in range(3):
            T[P + j, P + j, P + j] += t3[j]
        return T

    def slice(self, i):
        return self.tensor()[i]
