"""Pins for the oracle's generalized leapfrog (Eq. leapfrog) and Algorithm 1: time reversibility,
volume preservation, eps^2 scaling of the energy error, the closed-form posterior of a
Gaussian-likelihood GP (Bishop, PRML ch. 6) and brute-force quadrature at N = 2 (CPU only)."""
import numpy as np
import pytest

from oracle.geometry import Geometry
from oracle.integrator import leapfrog, trajectory
from oracle.sampler import sample
from paper_2511_06407_b300 import workloads as wl


def _small(N=4, seed=3, n_kernels=2, jitter=0.05):
    p = wl.propensity(N, seed=seed, n_kernels=n_kernels)
    for k in p["kernels"]:
        k["jitter"] = jitter
    return p


def test_leapfrog_is_reversible(oracle_model):
    prob = _small()
    m = oracle_model(prob)
    q0 = wl.random_state(prob, 1, seed=1)[0]
    p0 = 0.5 * wl.random_momentum(prob, 1, seed=2)[0]
    q, p, _, _ = trajectory(m, q0, p0, 0.05, 3, 50)
    qb, pb, _, _ = trajectory(m, q, -p, 0.05, 3, 50)
    assert np.abs(q - q0).max() > 1e-3  # it moved
    np.testing.assert_allclose(qb, q0, atol=1e-10)
    np.testing.assert_allclose(-pb, p0, atol=1e-10)


def test_leapfrog_preserves_volume(oracle_model):
    prob = wl.gp_classification(2, seed=4)
    for k in prob["kernels"]:
        k["jitter"] = 0.05
    m = oracle_model(prob)
    q0 = wl.random_state(prob, 1, seed=5)[0]
    p0 = 0.5 * wl.random_momentum(prob, 1, seed=6)[0]
    d = m.d
    x0 = np.concatenate([q0, p0])

    def step(x):
        qn, pn, _ = leapfrog(m, x[:d], x[d:], 0.1, 50)
        return np.concatenate([qn, pn])

    h = 1e-6
    J = np.stack([(step(x0 + h * e) - step(x0 - h * e)) / (2 * h) for e in np.eye(2 * d)], axis=1)
    assert abs(np.linalg.det(J) - 1.0) < 1e-6


def test_energy_error_scales_as_eps_squared(oracle_model):
    prob = _small(N=3, seed=7)
    m = oracle_model(prob)
    q0 = wl.random_state(prob, 1, seed=8)[0]
    p0 = Geometry(m, q0, 1.0, with_third=False).sqrtG_z(wl.random_momentum(prob, 1, seed=9)[0])
    errs = []
    epss = [0.01, 0.005, 0.0025]
    for eps in epss:
        L = int(round(0.08 / eps))
        geo = Geometry(m, q0, 1.0)
        H0 = geo.hamiltonian(p0)
        q, p, worst = q0, p0, 0.0
        for _ in range(L):
            q, p, geo = leapfrog(m, q, p, eps, 50, geo=geo)
            worst = max(worst, abs(geo.hamiltonian(p) - H0))
        errs.append(worst)
    slope = np.polyfit(np.log(epss), np.log(errs), 1)[0]
    assert 1.8 <= slope <= 2.2, (errs, slope)


def _batch_se(x, nb=20):
    n = len(x) // nb * nb
    b = x[:n].reshape(nb, -1, *x.shape[1:]).mean(axis=1)
    return b.std(axis=0, ddof=1) / np.sqrt(nb)


@pytest.mark.slow
def test_gaussian_gp_posterior_moments(oracle_model):
    """Gaussian likelihood, fixed hyperparameters: f | y ~ N(K (K + s2 I)^-1 y,
    K - K (K + s2 I)^-1 K). Sample mean and variance within 4 Monte-Carlo standard errors."""
    prob = wl.gp_regression(3, seed=11, noise_var=0.2)
    m = oracle_model(prob)
    from oracle.kernels import kernel_derivs
    K = kernel_derivs("se", m.X, m.u_fixed, 1e-6)[0]
    A = np.linalg.solve(K + m.noise_var * np.eye(3), np.eye(3))
    mean = K @ A @ m.y
    cov = K - K @ A @ K
    res = sample(m, np.zeros(3), 1200, 50, seed=1, chain=0, eps=0.5, n_leapfrog=4, n_fp=4)
    Q = res["q"]
    assert res["accept"].mean() > 0.9
    se = _batch_se(Q)
    assert np.all(np.abs(Q.mean(axis=0) - mean) < 4 * se + 1e-12), (Q.mean(axis=0), mean, se)
    dev2 = (Q - mean) ** 2
    se2 = _batch_se(dev2)
    assert np.all(np.abs(dev2.mean(axis=0) - np.diag(cov)) < 4 * se2 + 1e-12)


def test_metropolis_hastings_keeps_the_posterior_at_a_coarse_step(oracle_model):
    """The accept/reject step makes Algorithm 1 exact at any step size: with one leapfrog per
    iteration at eps = 1.2 about a quarter of the proposals carry an energy error large enough to
    be rejected, and the chain still has the closed-form posterior mean and variance of the
    Gaussian-likelihood GP (an accept test with the energy difference reversed, which the fine-step
    moment check above cannot see, inflates the variances several times here)."""
    prob = wl.gp_regression(3, seed=11, noise_var=0.2)
    m = oracle_model(prob)
    from oracle.kernels import kernel_derivs
    K = kernel_derivs("se", m.X, m.u_fixed, 1e-6)[0]
    A = np.linalg.solve(K + m.noise_var * np.eye(3), np.eye(3))
    mean = K @ A @ m.y
    var = np.diag(K - K @ A @ K)
    res = sample(m, np.zeros(3), 2000, 50, seed=1, chain=0, eps=1.2, n_leapfrog=1, n_fp=2)
    Q = res["q"]
    assert 0.5 < res["accept"].mean() < 0.9  # a coarse step: a real share of rejections
    se = _batch_se(Q)
    assert np.all(np.abs(Q.mean(axis=0) - mean) < 4 * se + 1e-12), (Q.mean(axis=0), mean, se)
    dev2 = (Q - mean) ** 2
    se2 = _batch_se(dev2)
    assert np.all(np.abs(dev2.mean(axis=0) - var) < 4 * se2 + 1e-12), (dev2.mean(axis=0), var, se2)


def test_sampler_records_the_log_posterior_of_its_samples(oracle_model):
    """The log P that Algorithm 1 records for each kept sample is the log posterior at the recorded
    position: here scipy's densities (the GP prior's MVN and the Gaussian likelihood)."""
    import scipy.stats as st
    from oracle.kernels import kernel_derivs
    prob = wl.gp_regression(3, seed=11, noise_var=0.2)
    m = oracle_model(prob)
    K = kernel_derivs("se", m.X, m.u_fixed, 1e-6)[0]
    res = sample(m, np.zeros(3), 20, 5, seed=2, chain=0, eps=0.5, n_leapfrog=2, n_fp=2)
    assert res["accept"].any()
    for q, lp in zip(res["q"], res["logp"]):
        want = (st.multivariate_normal(np.zeros(3), K).logpdf(q)
                + st.norm.logpdf(m.y, loc=q, scale=np.sqrt(m.noise_var)).sum())
        assert lp == pytest.approx(want, rel=1e-12, abs=1e-10)


@pytest.mark.slow
def test_brute_force_quadrature_tiny_classification(oracle_model):
    """N = 2 Bernoulli-logistic GP with both hyperparameters sampled (d = 4): RMHMC posterior means
    of (f, u) against 4-D grid quadrature of exp(-U) (the oracle's U is pinned against scipy
    densities separately)."""
    from oracle import model as mdl
    prob = wl.gp_classification(2, seed=12)
    for k in prob["kernels"]:
        k["jitter"] = 1e-2
    m = oracle_model(prob)
    # quadrature on a product grid
    fg = np.linspace(-7, 7, 36)
    ug = np.linspace(-5, 7, 40)
    F1, F2, U0, U1 = np.meshgrid(fg, fg, ug, ug, indexing="ij")
    pts = np.stack([F1.ravel(), F2.ravel(), U0.ravel(), U1.ravel()], axis=1)
    # vectorised -U over the grid: 2 x 2 SE kernel in closed form
    x = m.X
    r2 = np.sum((x[0] - x[1]) ** 2)
    c = np.exp(pts[:, 2])
    ell = np.exp(pts[:, 3])
    j = 1e-2
    k11 = c * (1 + j)
    k12 = c * np.exp(-0.5 * r2 / ell ** 2)
    det = k11 * k11 - k12 * k12
    f1, f2 = pts[:, 0], pts[:, 1]
    quad = (k11 * f1 * f1 - 2 * k12 * f1 * f2 + k11 * f2 * f2) / det
    logp = -0.5 * quad - 0.5 * np.log(det) - np.log(2 * np.pi)
    F = np.stack([f1, f2], axis=1)
    logp += np.sum(m.y * F - np.logaddexp(0, F), axis=1)
    for h in range(2):
        logp += mdl.log_prior_u(2.0, 2.0, pts[:, 2 + h])
    # spot-check the vectorised density against the oracle's U at a few grid points
    for i in np.random.default_rng(0).integers(0, len(pts), 5):
        assert -mdl.potential(m, pts[i]) == pytest.approx(logp[i], rel=1e-10, abs=1e-10)
    w = np.exp(logp - logp.max())
    w /= w.sum()
    ref = w @ pts
    # alpha = 1 keeps g >= 1: with N = 2 the hyperparameters follow their heavy-tailed prior, where
    # the Hessian's curvature vanishes and g -> 1/alpha would make the velocities explode
    res = sample(m, np.zeros(4), 1500, 100, seed=3, chain=0, eps=0.4, n_leapfrog=4, n_fp=4,
                 alpha=1.0)
    Q = res["q"]
    se = _batch_se(Q, nb=25)
    assert res["accept"].mean() > 0.6
    assert np.all(np.abs(Q.mean(axis=0) - ref) < 4 * se + 0.02), (Q.mean(axis=0), ref, se)
