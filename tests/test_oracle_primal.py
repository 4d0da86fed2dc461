"""Pins of the primal (reduced-rank) model oracle, J = 1 and the mean/variance model J = 2, against
things other than itself: the Fourier transform of the Gaussian kernel, the reduced-rank
approximation of the kernel, scipy densities, and finite differences of the likelihood, of U, its
gradient and its Hessian, plus the Hamiltonian gradient."""
from math import pi

import numpy as np
import pytest
from scipy import integrate, stats

from oracle import primal
from oracle.geometry import Geometry
from paper_2511_06407_b300 import workloads as wl


def small_model(lik="bernoulli", Dl=1, M=6, N=40, seed=3):
    if lik == "meanvar":
        return primal.from_problem(wl.meanvar_regression(2, N=N, seed=seed, M=M, n_linear=Dl))
    prob = wl.solin_logistic(2, N=N, seed=seed, M=M, n_linear=Dl)
    m = primal.from_problem(prob)
    if lik == "gaussian":
        rng = np.random.default_rng(seed)
        m.lik, m.noise_var = "gaussian", 0.3
        m.y = prob["f_true"] + np.sqrt(0.3) * rng.standard_normal(N)
    return m


def rand_q(m, seed, scale=0.4):
    rng = np.random.default_rng(seed)
    q = scale * rng.standard_normal(m.d)
    q[-3:] = 0.3 * rng.standard_normal(3)
    return q


@pytest.mark.parametrize("s", [0.5, 1.0, 3.0])
def test_spectral_weights_are_the_fourier_transform_of_the_kernel(s):
    """V_m(s) = S(pi m / 2L) with S(w) = int exp(-r^2/s) exp(-i w r) dr, by quadrature. A wrong
    exponent (the appendix's printed pi m^2 s instead of pi^2 m^2 s) fails here."""
    m = small_model(M=12)
    V = primal.spectral_weights(m, np.log(s))
    for mm in (1, 5, 12):
        w = pi * mm / (2 * m.L)
        S, _ = integrate.quad(lambda r: np.exp(-r * r / s) * np.cos(w * r), -np.inf, np.inf)
        assert V[mm - 1] == pytest.approx(S, rel=1e-9)


def test_reduced_rank_features_reproduce_the_kernel():
    """sum_m V_m phi_m(x) phi_m(x') -> L exp(-(x - x')^2 / s) inside [-L, L] (Solin and Sarkka):
    the sinusoidal features with the 1/sqrt(L) normalisation dropped (a rescaling of c_g)."""
    prob = wl.solin_logistic(1, N=7, seed=0, M=80)
    m = primal.from_problem(prob)
    m.Xg = np.linspace(-2.0, 2.0, 7)[:, None]
    Phi = primal.features(m)[:, :m.M]
    for s in (0.5, 1.0, 2.0):
        V = primal.spectral_weights(m, np.log(s))
        K = (Phi * V) @ Phi.T
        x = m.Xg[:, 0]
        want = m.L * np.exp(-(x[:, None] - x[None, :]) ** 2 / s)
        np.testing.assert_allclose(K, want, rtol=0, atol=1e-9 * m.L)


@pytest.mark.parametrize("lik", ["bernoulli", "gaussian", "meanvar"])
def test_potential_matches_scipy_densities(lik):
    m = small_model(lik)
    q = rand_q(m, 1)
    tau = 0.7
    W, u = q[:m.J * m.P].reshape(m.J, m.P), q[m.J * m.P:]
    F = W @ primal.features(m).T
    if lik == "bernoulli":
        ll = stats.bernoulli.logpmf(m.y, 1.0 / (1.0 + np.exp(-F[0]))).sum()
    elif lik == "gaussian":
        ll = stats.norm.logpdf(m.y, F[0], np.sqrt(m.noise_var)).sum()
    else:  # Example 1: y ~ N(f_1, delta + exp f_2)
        ll = stats.norm.logpdf(m.y, F[0], np.sqrt(m.delta + np.exp(F[1]))).sum()
    cg, sg, cl = np.exp(u)
    Mg = m.M * m.Dg
    var = np.tile(cg * np.sqrt(pi * sg) * np.exp(-pi ** 2 * np.arange(1, m.M + 1) ** 2 * sg / (16 * m.L ** 2)), m.Dg)
    lp = 0.0
    for w in W:
        lp += stats.norm.logpdf(w[:Mg], 0.0, np.sqrt(var)).sum()
        lp += stats.norm.logpdf(w[Mg:Mg + m.Dl], 0.0, np.sqrt(cl)).sum()
        lp += stats.norm.logpdf(w[-1], 0.0, np.sqrt(m.bias_var))
    for j, th in enumerate((cg, sg, cl)):
        lp += stats.invgamma.logpdf(th, m.prior_a[j], scale=m.prior_b[j]) + u[j]   # + log |d theta / d u|
    assert primal.potential(m, q, tau) == pytest.approx(-(tau * ll + lp), rel=1e-12)


@pytest.mark.parametrize("lik", ["bernoulli", "gaussian", "meanvar"])
def test_gradient_and_hessian_match_finite_differences(lik):
    m = small_model(lik)
    q = rand_q(m, 2)
    tau = 0.8
    g = primal.gradient(m, q, tau)
    H = primal.hessian(m, q, tau)
    np.testing.assert_allclose(H, H.T, rtol=0, atol=1e-12 * np.abs(H).max())
    h = 1e-6
    for i in range(m.d):
        e = np.zeros(m.d)
        e[i] = h
        fd = (primal.potential(m, q + e, tau) - primal.potential(m, q - e, tau)) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-6, abs=1e-6)
        fdg = (primal.gradient(m, q + e, tau) - primal.gradient(m, q - e, tau)) / (2 * h)
        np.testing.assert_allclose(H[i], fdg, rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("lik", ["bernoulli", "gaussian", "meanvar"])
def test_third_derivatives_match_finite_differences(lik):
    m = small_model(lik, M=4, N=30)
    q = rand_q(m, 3)
    tau = 0.9
    T = primal.ThirdDerivatives(m, q, tau).tensor()
    np.testing.assert_allclose(T, T.transpose(1, 0, 2), atol=1e-12)
    np.testing.assert_allclose(T, T.transpose(0, 2, 1), atol=1e-12)
    h = 1e-5
    for i in range(m.d):
        e = np.zeros(m.d)
        e[i] = h
        fd = (primal.hessian(m, q + e, tau) - primal.hessian(m, q - e, tau)) / (2 * h)
        np.testing.assert_allclose(T[i], fd, rtol=1e-6, atol=1e-6)


def test_hamiltonian_gradient_matches_finite_differences_sqrt_map():
    """dH/dq with the sqrt(kappa^2 + lambda^2) map of Sec. 2.5 (kappa = 1) against FD of H(q, p)."""
    m = small_model(M=4, N=30)
    q = rand_q(m, 4)
    p = np.random.default_rng(5).standard_normal(m.d)
    geo = Geometry(m, q, 1.0, 1.0, "sqrt")
    got = geo.dHdq(p)
    h = 1e-6
    for i in range(m.d):
        e = np.zeros(m.d)
        e[i] = h
        Hp = Geometry(m, q + e, 1.0, 1.0, "sqrt", with_third=False).hamiltonian(p)
        Hm = Geometry(m, q - e, 1.0, 1.0, "sqrt", with_third=False).hamiltonian(p)
        assert got[i] == pytest.approx((Hp - Hm) / (2 * h), rel=1e-5, abs=1e-6)


def test_dimension_of_the_simulated_problem():
    """d = 30 D + 4 (D = 1 gives 34, D = 16 gives 484; Fig. 1)."""
    for D, want in ((1, 34), (16, 484)):
        prob = wl.solin_logistic(D, N=20, seed=0)
        assert primal.from_problem(prob).d == want == wl.dims(prob)[2]


def test_meanvar_likelihood_derivatives_match_finite_differences():
    """The per-sample derivatives of l(F_1, F_2) = (y - F_1)^2 / (2 v) + log(2 pi v) / 2,
    v = delta + exp F_2, against central differences of l itself (up to third order)."""
    m = small_model("meanvar", N=12)
    rng = np.random.default_rng(9)
    F = np.stack([rng.normal(size=m.N), rng.normal(-1.0, 0.7, size=m.N)])
    l0, l1, l2, l3 = primal.data_derivs(m, F)
    h = 1e-4

    def f(F1, F2):
        return primal.data_derivs(m, np.stack([F1, F2]))[0]

    # first derivatives
    for j in range(2):
        Fp, Fm = F.copy(), F.copy()
        Fp[j] += h
        Fm[j] -= h
        np.testing.assert_allclose(l1[j], (f(*Fp) - f(*Fm)) / (2 * h), rtol=1e-6, atol=1e-8)
    # second and third derivatives from differences of the analytic lower orders
    for (j, k), ljk in l2.items():
        Fp, Fm = F.copy(), F.copy()
        Fp[k] += h
        Fm[k] -= h
        d1p = primal.data_derivs(m, Fp)[1][j]
        d1m = primal.data_derivs(m, Fm)[1][j]
        np.testing.assert_allclose(ljk, (d1p - d1m) / (2 * h), rtol=1e-6, atol=1e-8)
    for (j, k, l), ljkl in l3.items():
        Fp, Fm = F.copy(), F.copy()
        Fp[l] += h
        Fm[l] -= h
        d2p = primal.data_derivs(m, Fp)[2][(j, k)]
        d2m = primal.data_derivs(m, Fm)[2][(j, k)]
        np.testing.assert_allclose(ljkl, (d2p - d2m) / (2 * h), rtol=1e-6, atol=1e-8)
