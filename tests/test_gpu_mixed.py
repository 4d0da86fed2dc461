"""The mixed-precision form (precision = "mixed": the Jacobi rotations and the d x d products
M = Psi^T H Psi and W = Psi C Psi^T in double-float pairs of FP32, about 48 significant bits;
Cholesky, the K^-1 algebra, log-determinants, the Hamiltonian and everything else FP64) against
the FP64 oracle.

Stated error per result: the metric gradient dH/dq within 1e-5 relative (or the calibrated
LU-vs-Cholesky spread of the FP64 oracle where the conditioning of K makes that larger, as in the
FP64 parity tests); the quantities the rotations do not touch (U, dU/dq, the Hessian) at the FP64
tolerance 1e-10; eigenvalues, G and H(q, p) within 1e-8 relative; G^-1 p (= dH/dp, the other
half of the metric gradient) within the same 1e-5: it is dominated by the smallest eigenpairs,
whose vectors carry the rounding of entries ~1e6 divided by their gaps; two FP64 LAPACK
eigensolvers already disagree by up to 4e-8 there (N = 400), and the double-float unit is 32x
the FP64 one, so ~1e-6 is the expected level; accept/reject decisions
identical to the oracle's on the N = 50 sampler case; posterior means and variances of a
fixed-hyperparameter GP regression within Monte-Carlo error of the closed-form posterior.
"""
import numpy as np
import pytest

import oracle_pool
from conftest import potential_rounding_bound
from oracle import model as mdl
from oracle.geometry import Geometry
from oracle.sampler import sample
from paper_2511_06407_b300 import workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

MIXED_BASE = {"U": 1e-10, "dU": 1e-10, "H": 1e-10, "lam": 1e-8, "G": 1e-8, "Ham": 1e-8,
              "dHdq": 1e-5, "Ginv_p": 1e-5}


@pytest.fixture(scope="module")
def rm():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2511_06407_b300 import build, rmhmc
    build.build()
    return rmhmc


def _geometry(rm, prob, Q, P, tau, integ):
    C, d = Q.shape
    m = rm.Model(prob, C, tau)
    m.set_state(torch.tensor(Q, device="cuda"), integ=integ)
    f64 = dict(dtype=torch.float64, device="cuda")
    out = {"U": torch.empty(C, **f64), "dU": torch.empty(C, d, **f64),
           "H": torch.empty(C, d, d, **f64), "lam": torch.empty(C, d, **f64),
           "G": torch.empty(C, d, d, **f64), "sweeps": torch.empty(C, dtype=torch.int32, device="cuda"),
           "dHdq": torch.empty(C, d, **f64), "Ginv_p": torch.empty(C, d, **f64),
           "Ham": torch.empty(C, **f64)}
    m.geometry(out["U"], out["dU"], out["H"], out["lam"], out["G"], out["sweeps"])
    m.hamiltonian_grad(torch.tensor(P, device="cuda"), out["dHdq"], out["Ginv_p"], out["Ham"])
    torch.cuda.synchronize()
    m.close()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _oracle(m, q, tau, p):
    geo = Geometry(m, q, tau, 1e6, "coth")
    return {"U": geo.U, "dU": geo.dU, "H": geo.H, "lam": geo.lam, "G": geo.G(),
            "dHdq": geo.dHdq(p), "Ginv_p": geo.Ginv_p(p), "Ham": geo.hamiltonian(p)}


def _compare(label, got, c, m, q, tau, p, keys, oracle=None):
    if oracle is None:
        ref = _oracle(m, q, tau, p)
        with mdl.inverse_method("cholesky"):
            alt = _oracle(m, q, tau, p)
    else:
        ref, alt = oracle
    fails, rows = [], []
    for k in keys:
        g = np.sort(got[k][c]) if k == "lam" else got[k][c]
        err = float(np.linalg.norm(np.asarray(g) - ref[k]))
        tol = max(MIXED_BASE[k] * float(np.linalg.norm(ref[k])),
                  8.0 * float(np.linalg.norm(np.asarray(ref[k]) - alt[k])))
        if k in ("U", "Ham"):
            tol = max(tol, potential_rounding_bound(m, q))
        scale = max(float(np.linalg.norm(ref[k])), 1e-300)
        rows.append(f"{k}={err / scale:.1e}/{tol / scale:.0e}")
        if not err <= tol:
            fails.append((label, c, k, err, tol))
    print(label, "chain", c, "sweeps", got["sweeps"][c], " ".join(rows))
    return fails


CASES = [("c0", lambda: wl.gp_classification(50, seed=0), 3, [1.0, 0.5, 0.8]),
         ("propensity3", lambda: wl.propensity(40, seed=1, n_kernels=3), 2, None),
         # N = 130: every product spans a 128 x 128 tile, so the whole tensor-core path runs
         ("tc130", lambda: wl.gp_classification(130, seed=4), 2, [1.0, 0.7]),
         ("regression_fixed", lambda: wl.gp_regression(30, seed=3), 2, None)]


@pytest.mark.parametrize("name,make,C,tau", CASES, ids=[c[0] for c in CASES])
def test_mixed_geometry_relative_rule(rm, oracle_model, name, make, C, tau):
    """Every eigenpair resolved (RELATIVE rule, cold start): eigenvalues and G too."""
    prob = make()
    Q = wl.random_state(prob, C, seed=10)
    Q[0] = 0.0
    P = wl.random_momentum(prob, C, seed=11)
    got = _geometry(rm, prob, Q, P, tau, rm.Integrator(precision="mixed", jacobi_rule="relative"))
    m = oracle_model(prob)
    taus = tau or [1.0] * C
    fails = []
    for c in range(C):
        fails += _compare(name + "/mixed", got, c, m, Q[c], taus[c], P[c], tuple(MIXED_BASE))
    assert not fails, fails


@pytest.mark.parametrize("name,make,C,tau", CASES[:3], ids=[c[0] for c in CASES[:3]])
def test_mixed_metric_rule_sampler_quantities(rm, oracle_model, name, make, C, tau):
    """The sampler's default METRIC rule: the quantities the Hamiltonian and its gradient use."""
    prob = make()
    Q = wl.random_state(prob, C, seed=12)
    P = wl.random_momentum(prob, C, seed=13)
    got = _geometry(rm, prob, Q, P, tau, rm.Integrator(precision="mixed"))
    m = oracle_model(prob)
    taus = tau or [1.0] * C
    fails = []
    for c in range(C):
        fails += _compare(name + "/mixed-metric", got, c, m, Q[c], taus[c], P[c],
                          ("U", "dU", "H", "dHdq", "Ginv_p", "Ham"))
    assert not fails, fails


def test_mixed_full_size_metric_gradient(rm, oracle_model):
    """N = 400 (d = 402), 64 chains: the launch configuration of the benchmark; the metric
    gradient, G^-1 p and H(q, p) of 8 chains spread over the batch."""
    prob = wl.gp_classification(400, seed=0)
    C = 64
    Q = wl.random_state(prob, C, seed=5, f_scale=0.5, u_scale=0.2)
    P = wl.random_momentum(prob, C, seed=6)
    got = _geometry(rm, prob, Q, P, None, rm.Integrator(precision="mixed"))
    m = oracle_model(prob)
    fails = []
    chains = list(range(0, C, 8))
    res = oracle_pool.run(oracle_pool.quantities_job,
                          [(prob, Q[c], 1.0, P[c], method, "evd") for c in chains for method in ("lu", "cholesky")])
    for i, c in enumerate(chains):
        fails += _compare("N400/mixed", got, c, m, Q[c], 1.0, P[c], ("dHdq", "Ginv_p", "Ham"),
                          oracle=(res[2 * i], res[2 * i + 1]))
    assert not fails, fails


def test_mixed_sampler_decisions_c0(rm, oracle_model):
    """Algorithm 1 on the N = 50 problem from f = 0, u = 0 (eps = 0.01, L = 10, 6 fixed-point
    iterations, seed 0): the same accept/reject decisions as the FP64 oracle and the same chain
    within 1e-6."""
    prob = wl.gp_classification(50, seed=0)
    m = oracle_model(prob)
    n_iter, eps = 6, 0.01
    ref = sample(m, np.zeros(m.d), n_iter, 0, seed=0, chain=0, eps=eps, n_leapfrog=10, n_fp=6)
    integ = rm.Integrator(eps=eps, n_leapfrog=10, n_fp=6, precision="mixed")
    model = rm.Model(prob, 1)
    model.set_state(torch.zeros(1, m.d, dtype=torch.float64, device="cuda"), integ=integ)
    f64 = dict(dtype=torch.float64, device="cuda")
    qs, lp = torch.empty(n_iter, 1, m.d, **f64), torch.empty(n_iter, 1, **f64)
    acc = torch.empty(n_iter, 1, dtype=torch.int32, device="cuda")
    cs = torch.empty(1, dtype=torch.int32, device="cuda")
    model.sample(n_iter, 0, 0, qs, lp, acc, chain_status=cs, integ=integ)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(acc.cpu().numpy()[:, 0].astype(bool), ref["accept"])
    assert ref["accept"].any()  # (rejected proposals that left the PD region flag the status, as in FP64)
    q = qs.cpu().numpy()[:, 0]
    for i in range(n_iter):
        assert np.linalg.norm(q[i] - ref["q"][i]) <= 1e-6 * max(np.linalg.norm(ref["q"][i]), 1.0), i


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_posterior_moments_match_closed_form(rm, oracle_model, precision):
    """GP regression with fixed hyperparameters (N = 20, Gaussian likelihood): the posterior of f
    is N(K (K + s2 I)^-1 y, K - K (K + s2 I)^-1 K). 64 chains x 150 kept iterations; every
    coordinate's posterior mean and variance must lie within 5 standard errors (spread of the 64
    independent per-chain estimates) of the closed form."""
    prob = wl.gp_regression(20, seed=21)
    m = oracle_model(prob)
    _, _, (st,) = mdl._states(m, np.zeros(m.d))
    K, s2, y = st.mats[0], m.noise_var, m.y
    A = np.linalg.solve(K + s2 * np.eye(m.N), np.column_stack([y, K]))
    mean, cov = K @ A[:, 0], K - K @ A[:, 1:]
    var = np.diag(cov)
    C, n_iter, n_burn = 64, 150, 20
    integ = rm.Integrator(eps=0.3, n_leapfrog=5, n_fp=4, precision=precision)
    model = rm.Model(prob, C)
    model.set_state(torch.zeros(C, m.d, dtype=torch.float64, device="cuda"), integ=integ)
    f64 = dict(dtype=torch.float64, device="cuda")
    qs = torch.empty(n_iter, C, m.d, **f64)
    acc = torch.empty(n_iter, C, dtype=torch.int32, device="cuda")
    cs = torch.empty(C, dtype=torch.int32, device="cuda")
    model.sample(n_iter, n_burn, 3, qs, accept=acc, chain_status=cs, integ=integ)
    torch.cuda.synchronize()
    assert not cs.cpu().numpy().any()
    q = qs.cpu().numpy()                        # (n_iter, C, N)
    print(precision, "acceptance", acc.cpu().numpy().mean())
    chain_mean = q.mean(axis=0)                 # (C, N)
    chain_var = q.var(axis=0, ddof=1)
    se_mean = chain_mean.std(axis=0, ddof=1) / np.sqrt(C)
    se_var = chain_var.std(axis=0, ddof=1) / np.sqrt(C)
    z_mean = np.abs(chain_mean.mean(axis=0) - mean) / se_mean
    z_var = np.abs(chain_var.mean(axis=0) - var) / se_var
    print(precision, "max z mean", z_mean.max(), "max z var", z_var.max())
    assert z_mean.max() < 5.0 and z_var.max() < 5.0


def test_mixed_warm_updates_with_and_without_prerotation(rm, oracle_model):
    """Warm-started eigen-updates in the mixed form at N = 130 (d = 132: the d x d products span
    tensor-core tiles, so the first-order pre-rotation applies): 5 leapfrogs (eps = 0.01, 4
    fixed-point iterations, 24 warm eigen-updates) of 2 chains, with the pre-rotation and without,
    against the oracle's trajectory from the same (q, p): within 1e-6 relative or 16x the oracle's
    LU-vs-Cholesky spread (the mixed form's trajectory bound). With the pre-rotation the Jacobi
    that follows it runs fewer rounds per eigen-update."""
    from oracle.integrator import trajectory
    from oracle.philox import normals
    prob = wl.gp_classification(130, seed=4)
    m = oracle_model(prob)
    C = 2
    Q = wl.random_state(prob, C, seed=9, f_scale=0.3, u_scale=0.2)
    P = np.stack([Geometry(m, Q[c], 1.0, with_third=False).sqrtG_z(normals(3, c, 0, m.d)) for c in range(C)])
    refs = []
    for c in range(C):
        qr, pr, _, _ = trajectory(m, Q[c], P[c], 0.01, 5, 4)
        with mdl.inverse_method("cholesky"):
            qa, pa, _, _ = trajectory(m, Q[c], P[c], 0.01, 5, 4)
        refs.append((qr, pr, qa, pa))
    rounds = {}
    for prerot in (True, False):
        model = rm.Model(prob, C)
        model.set_prerotation(prerot)
        integ = rm.Integrator(eps=0.01, n_fp=4, precision="mixed")
        model.set_state(torch.tensor(Q, device="cuda"), torch.tensor(P, device="cuda"), integ)
        model.profile(True)
        model.profile(False)  # resets the Jacobi counters
        q = torch.empty(C, m.d, dtype=torch.float64, device="cuda")
        p = torch.empty_like(q)
        st = torch.empty(C, dtype=torch.int32, device="cuda")
        model.leapfrog(5, q, p, status_out=st, integ=integ)
        torch.cuda.synchronize()
        cnt = model.jacobi_counters()
        rounds[prerot] = cnt["rounds"] / max(cnt["updates"], 1)
        q, p, st = q.cpu().numpy(), p.cpu().numpy(), st.cpu().numpy()
        model.close()
        assert np.all(st == 0), st
        for c in range(C):
            qr, pr, qa, pa = refs[c]
            for name, g, r, a in (("q", q[c], qr, qa), ("p", p[c], pr, pa)):
                err = np.linalg.norm(g - r)
                tol = max(1e-6 * np.linalg.norm(r), 16.0 * np.linalg.norm(r - a))
                print(f"prerotation {prerot} chain {c} {name}: {err / np.linalg.norm(r):.1e} / "
                      f"{tol / np.linalg.norm(r):.0e}")
                assert err <= tol, (prerot, c, name, err, tol)
    print("Jacobi rounds per eigen-update: with pre-rotation", rounds[True], "without", rounds[False])
    assert rounds[True] < rounds[False]


def test_gemm_tile_widths_give_identical_results(rm):
    """The mixed form's tensor-core GEMMs with 128 x 32 output tiles (the autotuner's other tile
    width) against 128 x 64: every output element is the same exact sum of the same slice products,
    so U, dU, the Hessian, dH/dq and G^-1 p of the N = 130 problem (K^-1 algebra and the d x d
    products on the tensor cores, symmetric and general outputs) must agree bit for bit."""
    prob = wl.gp_classification(130, seed=4)
    Q = wl.random_state(prob, 2, seed=10)
    P = wl.random_momentum(prob, 2, seed=11)
    outs = []
    for nt in (64, 32):
        m = rm.Model(prob, 2)
        m.set_gemm_tile(nt)
        integ = rm.Integrator(precision="mixed", jacobi_rule="relative")
        m.set_state(torch.tensor(Q, device="cuda"), integ=integ)
        f64 = dict(dtype=torch.float64, device="cuda")
        d = m.d
        U, dU, H = torch.empty(2, **f64), torch.empty(2, d, **f64), torch.empty(2, d, d, **f64)
        dHdq, Gp = torch.empty(2, d, **f64), torch.empty(2, d, **f64)
        m.geometry(U, dU, H)
        m.hamiltonian_grad(torch.tensor(P, device="cuda"), dHdq, Gp)
        torch.cuda.synchronize()
        outs.append([x.cpu().numpy() for x in (U, dU, H, dHdq, Gp)])
        m.close()
    for a, b in zip(*outs):
        np.testing.assert_array_equal(a, b)
