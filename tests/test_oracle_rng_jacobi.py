"""Pins for the oracle's Philox4x64-10 (against numpy's library Philox) and its Box-Muller draws,
and for the separate cyclic Jacobi solver (against LAPACK eigh, and the sweep-count behaviour of
Sec. 2.4 / Sec. 3.1) (CPU only)."""
import numpy as np
import pytest
import scipy.stats as st

from oracle.jacobi import jacobi_eigh, offdiag_norm
from oracle.philox import mh_uniform, normals, philox4x64_10


@pytest.mark.parametrize("key,ctr", [((0, 0), (0, 0, 0, 0)), ((7, 9), (5, 3, 2, 1)),
                                     ((2**64 - 1, 12345), (2**64 - 2, 2**63, 77, 2**40))])
def test_philox_matches_numpy_library(key, ctr):
    # numpy's Philox increments the 256-bit counter before producing each block
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array(ctr, dtype=np.uint64))
    ref = [int(v) for v in bg.random_raw(4)]
    c = list(ctr)
    c[0] = (c[0] + 1) % 2**64
    assert philox4x64_10(c, key) == ref


def test_box_muller_normals_are_standard():
    z = np.concatenate([normals(seed=3, chain=c, iteration=i, d=101) for c in range(4) for i in range(25)])
    assert abs(z.mean()) < 4.0 / np.sqrt(len(z))
    assert abs(z.var() - 1.0) < 5.0 * np.sqrt(2.0 / len(z))
    assert st.kstest(z, "norm").pvalue > 1e-3
    # distinct chains and iterations give distinct streams
    assert not np.allclose(normals(0, 0, 0, 8), normals(0, 1, 0, 8))
    assert not np.allclose(normals(0, 0, 0, 8), normals(0, 0, 1, 8))
    # a prefix of a longer draw is the shorter draw
    np.testing.assert_array_equal(normals(5, 2, 7, 9), normals(5, 2, 7, 13)[:9])
    u = np.array([mh_uniform(1, c, i) for c in range(8) for i in range(200)])
    assert st.kstest(u, "uniform").pvalue > 1e-3


def _sym(d, seed):
    A = np.random.default_rng(seed).normal(size=(d, d))
    return 0.5 * (A + A.T)


@pytest.mark.parametrize("d", [2, 5, 17])
def test_jacobi_matches_eigh(d):
    H = _sym(d, d)
    lam, Psi, sweeps = jacobi_eigh(H)
    ref = np.linalg.eigvalsh(H)
    np.testing.assert_allclose(np.sort(lam), ref, rtol=1e-12, atol=1e-13 * np.abs(ref).max())
    np.testing.assert_allclose(Psi.T @ Psi, np.eye(d), atol=1e-13)
    np.testing.assert_allclose(Psi @ np.diag(lam) @ Psi.T, H, atol=1e-12 * np.abs(H).max())
    assert 1 <= sweeps <= 30


def test_jacobi_warm_start_needs_one_to_two_sweeps_cold_grows_with_d():
    """Sec. 3.1 / Fig. 1C: warm-started (dynamic) Jacobi takes 1-2 sweeps regardless of d, the
    static (cold) one takes more sweeps as d grows."""
    warm, cold = {}, {}
    for d in (8, 32, 64):
        H = _sym(d, 100 + d)
        _, Psi, cold[d] = jacobi_eigh(H)
        E = 1e-4 * _sym(d, 200 + d)  # an O(eps) change of H between substeps
        _, _, warm[d] = jacobi_eigh(H + E, Psi0=Psi)
        assert 1 <= warm[d] <= 2, (d, warm[d])
    assert cold[8] < cold[64] and cold[64] >= 5
    # an already-diagonal start takes zero sweeps
    _, _, s0 = jacobi_eigh(np.diag([3.0, -1.0, 2.0]))
    assert s0 == 0
    assert offdiag_norm(np.eye(3)) == 0.0


def test_metric_rule_needs_fewer_sweeps_on_a_gp_hessian_and_keeps_G_inverse():
    """On the Hessian of the dual GP model (K^-1 puts ~N eigenvalues in a near-degenerate cluster
    near 1/(c jitter)), the 'metric' stopping rule stops earlier than 'relative' from a warm start
    while G^-1 p (soft-abs metric, alpha = 1e6) stays as accurate."""
    from oracle import model as mdl
    from oracle.softabs import g_and_gprime
    from paper_2511_06407_b300 import workloads as wl
    prob = wl.gp_classification(40, seed=0)
    m = mdl.from_problem(prob)
    q0 = wl.random_state(prob, 1, seed=3, f_scale=0.2, u_scale=0.1)[0]
    _, P0, _ = jacobi_eigh(mdl.hessian(m, q0))
    q1 = q0 + 1e-3 * np.random.default_rng(1).standard_normal(m.d)
    H1 = mdl.hessian(m, q1)
    p = np.random.default_rng(2).standard_normal(m.d)
    lam_ref, Psi_ref = np.linalg.eigh(H1)
    g_ref, _ = g_and_gprime(lam_ref)
    ref = Psi_ref @ ((Psi_ref.T @ p) / g_ref)
    out = {}
    for rule in ("relative", "metric"):
        lam, Psi, sw = jacobi_eigh(H1, Psi0=P0, rule=rule)
        g, _ = g_and_gprime(lam)
        v = Psi @ ((Psi.T @ p) / g)
        out[rule] = (sw, np.linalg.norm(v - ref) / np.linalg.norm(ref))
    assert out["metric"][0] < out["relative"][0], out
    assert out["metric"][1] < 1e-8 and out["relative"][1] < 1e-8, out
