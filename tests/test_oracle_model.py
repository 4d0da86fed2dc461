"""Pins for the oracle's model: kernel matrices vs scikit-learn / scipy, U vs scipy densities,
gradient / Hessian / third derivatives vs central finite differences (CPU only)."""
import numpy as np
import pytest
import scipy.stats as st
from scipy.spatial.distance import cdist

from oracle import model as mdl
from oracle.kernels import kernel_derivs
from paper_2511_06407_b300 import workloads as wl


def fd_grad(fun, x, h=1e-5):
    x = np.asarray(x, dtype=np.float64)
    out = []
    for i in range(len(x)):
        e = np.zeros_like(x)
        e[i] = h * max(1.0, abs(x[i]))
        out.append((np.asarray(fun(x + e)) - np.asarray(fun(x - e))) / (2 * e[i]))
    return np.array(out)


def _problems():
    a = wl.gp_classification(6, seed=3)
    b = wl.propensity(7, seed=4, n_kernels=3)
    c = wl.gp_regression(5, seed=5, sample_hypers=True)
    d = wl.gp_regression(5, seed=6, sample_hypers=False)
    for p in (a, b, c, d):
        for k in p["kernels"]:
            k["jitter"] = 1e-2
    b["kernels"][1]["prior_a"] = (3.0, 1.5)
    b["kernels"][2]["prior_b"] = (0.5, 1.0)
    return [(a, 0.7), (b, 1.0), (c, 1.0), (d, 0.4)]


PROBLEMS = _problems()


@pytest.mark.parametrize("u", [(0.3, -0.2), (-0.5, 0.6)])
def test_se_kernel_matches_sklearn(u):
    RBF = pytest.importorskip("sklearn.gaussian_process.kernels").RBF
    X = np.random.default_rng(0).uniform(-1, 1, (9, 2))
    K, D1, _, _ = kernel_derivs("se", X, u, 1e-6)
    c, ell = np.exp(u[0]), np.exp(u[1])
    Kref, dref = RBF(length_scale=ell)(X, eval_gradient=True)
    np.testing.assert_allclose(K, c * (Kref + 1e-6 * np.eye(9)), rtol=1e-13, atol=1e-15)
    # sklearn's gradient is with respect to log(length_scale), our u_1
    np.testing.assert_allclose(D1, c * dref[:, :, 0], rtol=1e-12, atol=1e-15)


def test_linear_kernel_matches_sklearn():
    DotProduct = pytest.importorskip("sklearn.gaussian_process.kernels").DotProduct
    X = (np.random.default_rng(1).uniform(size=(8, 2)) < 0.5).astype(float)
    u = (0.2, -0.4)
    K, D1, _, _ = kernel_derivs("linear", X, u, 1e-6)
    c, b = np.exp(u[0]), np.exp(u[1])
    Kref, dref = DotProduct(sigma_0=np.sqrt(b))(X, eval_gradient=True)
    np.testing.assert_allclose(K, c * (Kref + 1e-6 * np.eye(8)), rtol=1e-13)
    # d/dlog(sigma_0) of sigma_0^2 is 2 sigma_0^2 = 2 d/dlog(b)
    np.testing.assert_allclose(D1, c * dref[:, :, 0] / 2.0, rtol=1e-13)


def test_overlap_kernel_matches_scipy_hamming():
    X = np.random.default_rng(2).integers(0, 5, (10, 2)).astype(float)
    u = (-0.1, 0.3)
    K, _, _, _ = kernel_derivs("overlap", X, u, 1e-6)
    h = cdist(X, X, metric="hamming") * X.shape[1]
    np.testing.assert_allclose(K, np.exp(u[0]) * (np.exp(-h / np.exp(u[1])) + 1e-6 * np.eye(10)),
                               rtol=1e-13)


@pytest.mark.parametrize("kind", ["se", "linear", "overlap"])
def test_kernel_higher_derivatives_fd(kind):
    rng = np.random.default_rng(7)
    X = rng.integers(0, 4, (6, 3)).astype(float) if kind == "overlap" else rng.normal(size=(6, 3))
    u = np.array([0.1, -0.3])
    mats = kernel_derivs(kind, X, u, 1e-3)
    h = 1e-5
    for m in range(3):
        plus = kernel_derivs(kind, X, u + [0, h], 1e-3)[m]
        minus = kernel_derivs(kind, X, u - [0, h], 1e-3)[m]
        fd = (plus - minus) / (2 * h)
        if m == 0:
            fd = fd  # jitter does not depend on u_1
        np.testing.assert_allclose(mats[m + 1], fd, rtol=1e-6, atol=1e-8)
    # derivative in u_0 = log c returns the same matrix
    fd_c = (kernel_derivs(kind, X, u + [h, 0], 1e-3)[0] - kernel_derivs(kind, X, u - [h, 0], 1e-3)[0]) / (2 * h)
    np.testing.assert_allclose(mats[0], fd_c, rtol=1e-7, atol=1e-10)


@pytest.mark.parametrize("pi", range(len(PROBLEMS)))
def test_potential_matches_scipy_densities(pi, oracle_model):
    prob, tau = PROBLEMS[pi]
    m = oracle_model(prob)
    q = wl.random_state(prob, 1, seed=11 + pi)[0]
    f, u = mdl.split(m, q)
    F = f.sum(axis=0)
    if m.lik == "bernoulli":
        loglik = st.bernoulli.logpmf(m.y, 1.0 / (1.0 + np.exp(-F))).sum()
    else:
        loglik = st.norm.logpdf(m.y, loc=F, scale=np.sqrt(m.noise_var)).sum()
    logp = tau * loglik
    for k, spec in enumerate(m.kernels):
        K = kernel_derivs(spec.kind, m.X[:, list(spec.cols)], u[k], spec.jitter)[0]
        logp += st.multivariate_normal(mean=np.zeros(m.N), cov=K).logpdf(f[k])
        if m.sample_hypers:
            for h in range(2):
                th = np.exp(u[k, h])
                logp += st.invgamma.logpdf(th, spec.prior_a[h], scale=spec.prior_b[h]) + u[k, h]
    assert mdl.potential(m, q, tau) == pytest.approx(-logp, rel=1e-12, abs=1e-10)


@pytest.mark.parametrize("pi", range(len(PROBLEMS)))
def test_gradient_fd(pi, oracle_model):
    prob, tau = PROBLEMS[pi]
    m = oracle_model(prob)
    q = wl.random_state(prob, 1, seed=21 + pi)[0]
    g = mdl.gradient(m, q, tau)
    fd = fd_grad(lambda x: mdl.potential(m, x, tau), q)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-6 * np.abs(g).max())


@pytest.mark.parametrize("pi", range(len(PROBLEMS)))
def test_hessian_fd(pi, oracle_model):
    prob, tau = PROBLEMS[pi]
    m = oracle_model(prob)
    q = wl.random_state(prob, 1, seed=31 + pi)[0]
    H = mdl.hessian(m, q, tau)
    np.testing.assert_allclose(H, H.T, rtol=0, atol=1e-12 * np.abs(H).max())
    fd = fd_grad(lambda x: mdl.gradient(m, x, tau), q)
    np.testing.assert_allclose(H, fd, rtol=1e-6, atol=1e-6 * np.abs(H).max())


@pytest.mark.parametrize("pi", range(len(PROBLEMS)))
def test_third_derivatives_fd(pi, oracle_model):
    prob, tau = PROBLEMS[pi]
    m = oracle_model(prob)
    q = wl.random_state(prob, 1, seed=41 + pi)[0]
    T3 = mdl.ThirdDerivatives(m, q, tau).tensor()
    fd = fd_grad(lambda x: mdl.hessian(m, x, tau), q)
    np.testing.assert_allclose(T3, fd, rtol=1e-6, atol=1e-6 * np.abs(T3).max())
    # a third-derivative tensor is symmetric in all three indices
    np.testing.assert_allclose(T3, T3.transpose(1, 0, 2), atol=1e-10 * np.abs(T3).max())
    np.testing.assert_allclose(T3, T3.transpose(2, 1, 0), atol=1e-10 * np.abs(T3).max())


@pytest.mark.parametrize("state", ["zero", "random"])
def test_potential_matches_40_digit_evaluation(oracle_model, state):
    """U of an ill-conditioned problem (SE kernel, jitter 1e-6, cond(K) ~ 1e7) against the same
    definition evaluated in 40-digit arithmetic (mpmath Cholesky), at f = 0 and at a random point
    off the prior manifold (huge K^-1 f): to within the first-order error that rounding K to FP64
    already commits (tests/conftest.potential_rounding_bound; 2e-11 relative at f = 0, 1e-9 at the
    random point)."""
    from conftest import potential_rounding_bound
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    prob = wl.gp_classification(24, seed=0)
    m = oracle_model(prob)
    q = wl.random_state(prob, 1, seed=10)[0]
    if state == "zero":
        q[:] = 0.0
    f, u = mdl.split(m, q)
    X, N = m.X, m.N
    c, th = mp.e ** mp.mpf(u[0, 0]), mp.e ** mp.mpf(u[0, 1])
    K = mp.matrix(N, N)
    for i in range(N):
        for j in range(N):
            sq = sum((mp.mpf(X[i, k]) - mp.mpf(X[j, k])) ** 2 for k in range(2))
            K[i, j] = c * mp.e ** (-sq / (2 * th * th)) + (c * mp.mpf(1e-6) if i == j else 0)
    L = mp.cholesky(K)
    t = mp.lu_solve(L, mp.matrix([mp.mpf(v) for v in f[0]]))
    quad = sum(t[i] ** 2 for i in range(N))
    logdet = 2 * sum(mp.log(L[i, i]) for i in range(N))
    lik = sum(mp.log(1 + mp.e ** mp.mpf(f[0][i])) - mp.mpf(m.y[i]) * mp.mpf(f[0][i]) for i in range(N))
    pri = sum(2 * mp.log(2) - mp.loggamma(2) - 2 * mp.mpf(u[0, h]) - 2 * mp.e ** (-mp.mpf(u[0, h]))
              for h in range(2))
    exact = float(lik + quad / 2 + logdet / 2 + mp.mpf(N) / 2 * mp.log(2 * mp.pi) - pri)
    assert np.linalg.cond(kernel_derivs("se", X, u[0], 1e-6)[0]) > 1e5
    err = abs(mdl.potential(m, q) - exact)
    bound = potential_rounding_bound(m, q)
    assert err <= max(1e-12 * abs(exact), bound), (err, bound)
    # a dropped or wrong term would be orders of magnitude above the bound
    assert bound < 1e-8 * abs(exact)
