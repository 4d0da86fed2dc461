"""Pins for the oracle's SoftAbs map and Riemannian geometry: mpmath reference values, closed-form
limits, finite differences of the metric and the Hamiltonian, and the positive-definite special
case (CPU only)."""
import numpy as np
import pytest

mpmath = pytest.importorskip("mpmath")

from oracle import model as mdl
from oracle.geometry import Geometry
from oracle.softabs import divided_differences, g_and_gprime
from paper_2511_06407_b300 import workloads as wl

mpmath.mp.dps = 50


def _g_mp(lam, alpha):
    lam = mpmath.mpf(lam)
    if lam == 0:
        return 1 / mpmath.mpf(alpha), mpmath.mpf(0)
    x = alpha * lam
    g = lam * mpmath.coth(x)
    gp = mpmath.coth(x) - x / mpmath.sinh(x) ** 2
    return g, gp


@pytest.mark.parametrize("alpha", [1e6, 1.0, 37.5])
def test_g_matches_mpmath(alpha):
    xs = np.concatenate([[0.0], np.geomspace(1e-9, 60, 200), [9.99e-4, 1.001e-3, 19.99, 20.01]])
    lam = np.concatenate([xs, -xs]) / alpha
    g, gp = g_and_gprime(lam, alpha)
    for l, a, b in zip(lam, g, gp):
        gr, gpr = _g_mp(l, alpha)
        assert abs(a - float(gr)) <= 1e-15 * abs(float(gr)), (l, a, gr)
        assert abs(b - float(gpr)) <= 2e-15 * abs(float(gpr)) + 1e-300, (l, b, gpr)


def test_g_closed_form_limits():
    alpha = 1e6
    g, gp = g_and_gprime(np.array([0.0, 3.0, -2.5, 1e-2, -1e-2]), alpha)
    assert g[0] == 1.0 / alpha and gp[0] == 0.0
    np.testing.assert_array_equal(g[1:], [3.0, 2.5, 1e-2, 1e-2])
    np.testing.assert_array_equal(gp[1:], [1.0, -1.0, 1.0, -1.0])
    gs, gps = g_and_gprime(np.array([0.0, 3.0, -4.0]), 1.0, kind="sqrt")
    np.testing.assert_allclose(gs, [1.0, np.sqrt(10.0), np.sqrt(17.0)], rtol=1e-15)
    np.testing.assert_allclose(gps, [0.0, 3 / np.sqrt(10.0), -4 / np.sqrt(17.0)], rtol=1e-15)


def test_divided_differences_mpmath():
    alpha = 2.0
    lam = np.array([-3.0, -0.4, -1e-4, 0.0, 2e-5, 0.7, 0.7 + 1e-9, 5.0])
    T = divided_differences(lam, alpha)
    np.testing.assert_allclose(T, T.T, rtol=0, atol=0)
    for j in range(len(lam)):
        for l in range(len(lam)):
            if j == l:
                ref = _g_mp(lam[j], alpha)[1]
            elif abs(lam[j] - lam[l]) <= 1e-7 * max(1, abs(lam[j]), abs(lam[l])):
                ref = _g_mp(0.5 * (lam[j] + lam[l]), alpha)[1]
            else:
                gj, gl = _g_mp(lam[j], alpha)[0], _g_mp(lam[l], alpha)[0]
                ref = (gj - gl) / (mpmath.mpf(lam[j]) - mpmath.mpf(lam[l]))
            assert abs(T[j, l] - float(ref)) <= 1e-9 * max(1.0, abs(float(ref))), (j, l)


def _geo_problem(N=5, seed=3):
    p = wl.propensity(N, seed=seed, n_kernels=2)
    for k in p["kernels"]:
        k["jitter"] = 0.05
    return p


def _fd(fun, x, h=1e-6):
    out = []
    for i in range(len(x)):
        e = np.zeros_like(x)
        e[i] = h
        out.append((fun(x + e) - fun(x - e)) / (2 * h))
    return np.array(out)


@pytest.mark.parametrize("alpha,gkind", [(1e6, "coth"), (1.0, "sqrt"), (3.0, "coth")])
def test_betancourt_traces_match_fd_of_metric(alpha, gkind, oracle_model):
    """tr(W2 dH_i) = d/dq_i log|G| and tr(W1 dH_i) = -d/dq_i p^T G^-1 p (Eq. Betancourt_formula)."""
    prob = _geo_problem()
    m = oracle_model(prob)
    q = wl.random_state(prob, 1, seed=5)[0]
    p = wl.random_momentum(prob, 1, seed=6)[0]
    geo = Geometry(m, q, 0.8, alpha, gkind)

    def logdetG(x):
        return Geometry(m, x, 0.8, alpha, gkind, with_third=False).logdetG()

    def quad(x):
        return p @ Geometry(m, x, 0.8, alpha, gkind, with_third=False).Ginv_p(p)

    t2 = geo.traces(geo.W2())
    t1 = geo.traces(geo.W1(p))
    np.testing.assert_allclose(t2, _fd(logdetG, q), rtol=2e-6, atol=2e-6 * np.abs(t2).max())
    np.testing.assert_allclose(t1, -_fd(quad, q), rtol=2e-6, atol=2e-6 * np.abs(t1).max())


@pytest.mark.parametrize("alpha,gkind", [(1e6, "coth"), (1.0, "sqrt")])
def test_dHdq_matches_fd_of_hamiltonian(alpha, gkind, oracle_model):
    """dH/dq from the corrected-sign formula equals the finite difference of Eq. Hamiltonian
    (the printed Eq. d_Hamiltonian has the metric terms' signs swapped; that version fails)."""
    prob = _geo_problem(N=4, seed=8)
    m = oracle_model(prob)
    q = wl.random_state(prob, 1, seed=9)[0]
    p = wl.random_momentum(prob, 1, seed=10)[0]
    geo = Geometry(m, q, 1.0, alpha, gkind)
    fd = _fd(lambda x: Geometry(m, x, 1.0, alpha, gkind, with_third=False).hamiltonian(p), q)
    got = geo.dHdq(p)
    np.testing.assert_allclose(got, fd, rtol=2e-6, atol=2e-6 * np.abs(got).max())
    printed = geo.dU - 0.5 * geo.traces(geo.W2()) + 0.5 * geo.traces(geo.W1(p))
    assert np.abs(printed - fd).max() > 1e-3 * np.abs(fd).max()
    np.testing.assert_allclose(geo.dHdp(p), np.linalg.solve(geo.G(), p), rtol=1e-10)


def test_positive_definite_special_case(oracle_model):
    """H > 0 with every |alpha lambda| >> 1: G = H, T = 1, W2 = H^-1, W1 = (H^-1 p)(H^-1 p)^T."""
    prob = wl.gp_regression(6, seed=2, sample_hypers=False)
    m = oracle_model(prob)
    q = wl.random_state(prob, 1, seed=3)[0]
    p = wl.random_momentum(prob, 1, seed=4)[0]
    geo = Geometry(m, q, 1.0, 1e6, "coth")
    H = mdl.hessian(m, q)
    assert geo.lam.min() > 1e-3
    Hinv = np.linalg.inv(H)
    np.testing.assert_allclose(geo.G(), H, rtol=1e-12, atol=1e-12 * np.abs(H).max())
    np.testing.assert_allclose(geo.T, np.ones_like(geo.T), rtol=1e-12)
    np.testing.assert_allclose(geo.W2(), Hinv, rtol=1e-9, atol=1e-12 * np.abs(Hinv).max())
    v = Hinv @ p
    np.testing.assert_allclose(geo.W1(p), np.outer(v, v), rtol=1e-9, atol=1e-12 * np.abs(v).max() ** 2)


def test_momentum_root_is_symmetric_square_root(oracle_model):
    prob = _geo_problem()
    m = oracle_model(prob)
    geo = Geometry(m, wl.random_state(prob, 1, seed=1)[0], 1.0, 1e6, "coth", with_third=False)
    Z = np.eye(m.d)
    R = np.stack([geo.sqrtG_z(z) for z in Z], axis=1)
    np.testing.assert_allclose(R, R.T, atol=1e-10 * np.abs(R).max())
    np.testing.assert_allclose(R @ R, geo.G(), rtol=1e-9, atol=1e-10 * np.abs(geo.G()).max())
