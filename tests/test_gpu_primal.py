"""The primal (reduced-rank) model of the paper's experiments on the GPU (rmhmc_init_primal)
against the FP64 oracle (oracle/primal.py).

The primal Hessian has no K^-1, so the LU-versus-Cholesky calibration of the dual tests does not
apply: the GPU must meet base * ||x_oracle|| with base = 1e-10 for U, dU/dq, the Hessian, the
eigenvalues, G and H(q, p), and 1e-8 for dH/dq and G^-1 p (1e-5 for dH/dq and 1e-6 for G^-1 p
in the mixed form). Accept/reject decisions must be identical.
"""
import numpy as np
import pytest

from oracle.geometry import Geometry
from oracle.integrator import trajectory
from oracle.philox import normals
from oracle.sampler import sample
from paper_2511_06407_b300 import workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

BASE = {"U": 1e-10, "dU": 1e-10, "H": 1e-10, "lam": 1e-10, "G": 1e-10, "Ham": 1e-10,
        "dHdq": 1e-8, "Ginv_p": 1e-8}


@pytest.fixture(scope="module")
def rm():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2511_06407_b300 import build, rmhmc
    build.build()
    return rmhmc


def _problem(D=2, N=60, M=8, n_linear=1, seed=3):
    return wl.solin_logistic(D, N=N, seed=seed, M=M, n_linear=n_linear)


def _geometry(rm, prob, Q, P, tau, integ, with_G=True):
    C, d = Q.shape
    m = rm.Model(prob, C, tau)
    m.set_state(torch.tensor(Q, device="cuda"), integ=integ)
    f64 = dict(dtype=torch.float64, device="cuda")
    out = {"U": torch.empty(C, **f64), "dU": torch.empty(C, d, **f64), "H": torch.empty(C, d, d, **f64),
           "lam": torch.empty(C, d, **f64), "sweeps": torch.empty(C, dtype=torch.int32, device="cuda"),
           "dHdq": torch.empty(C, d, **f64), "Ginv_p": torch.empty(C, d, **f64), "Ham": torch.empty(C, **f64)}
    if with_G:
        out["G"] = torch.empty(C, d, d, **f64)
    m.geometry(out["U"], out["dU"], out["H"], out["lam"], out.get("G"), out["sweeps"])
    m.hamiltonian_grad(torch.tensor(P, device="cuda"), out["dHdq"], out["Ginv_p"], out["Ham"])
    torch.cuda.synchronize()
    m.close()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _compare(label, got, c, geo, p, keys, base):
    ref = {"U": geo.U, "dU": geo.dU, "H": geo.H, "lam": geo.lam, "G": geo.G(), "Ham": geo.hamiltonian(p),
           "Ginv_p": geo.Ginv_p(p)}
    if geo.third is not None:
        ref["dHdq"] = geo.dHdq(p)
    fails, rows = [], []
    for k in keys:
        g = np.sort(got[k][c]) if k == "lam" else got[k][c]
        err = float(np.linalg.norm(np.asarray(g) - ref[k]))
        scale = max(float(np.linalg.norm(ref[k])), 1e-300)
        rows.append(f"{k}={err / scale:.1e}")
        if not err <= base[k] * scale:
            fails.append((label, c, k, err / scale))
    print(label, "chain", c, "sweeps", got["sweeps"][c], " ".join(rows))
    return fails


@pytest.mark.parametrize("gkind,alpha", [("sqrt", 1.0), ("coth", 1e6)])
def test_primal_geometry_and_gradient_parity(rm, oracle_model, gkind, alpha):
    prob = _problem()
    C = 3
    Q = wl.random_state(prob, C, seed=10, f_scale=0.4, u_scale=0.3)
    Q[0] = 0.0  # the paper's initial state: a = 0, b = 0, every hyperparameter 1
    P = wl.random_momentum(prob, C, seed=11)
    tau = [1.0, 0.6, 0.3]
    got = _geometry(rm, prob, Q, P, tau, rm.Integrator(g_kind=gkind, alpha=alpha, jacobi_rule="relative"))
    m = oracle_model(prob)
    fails = []
    for c in range(C):
        geo = Geometry(m, Q[c], tau[c], alpha, gkind)
        fails += _compare(f"primal/{gkind}", got, c, geo, P[c], tuple(BASE), BASE)
    assert not fails, fails


def test_primal_full_size_d484(rm, oracle_model):
    """Sec. 2.5's largest model: D = 16 Gaussian kernels, M = 30, N = 500 (d = 484), 16 chains.
    dH/dq is checked through directional derivatives of the oracle's H(q, p) (the full
    third-derivative tensor is 0.9 GB at this size)."""
    prob = wl.solin_logistic(16, N=500, seed=0)
    C = 16
    Q = wl.random_state(prob, C, seed=5, f_scale=0.2, u_scale=0.2)
    P = wl.random_momentum(prob, C, seed=6)
    integ = rm.Integrator(g_kind="sqrt", alpha=1.0)
    got = _geometry(rm, prob, Q, P, None, integ, with_G=False)
    m = oracle_model(prob)
    fails = []
    rng = np.random.default_rng(7)
    for c in (0, 9):
        geo = Geometry(m, Q[c], 1.0, 1.0, "sqrt", with_third=False)
        fails += _compare("primal/d484", got, c, geo, P[c], ("U", "dU", "H", "Ginv_p", "Ham"), BASE)
        for _ in range(3):
            v = rng.standard_normal(m.d)
            h = 1e-5
            Hp = Geometry(m, Q[c] + h * v, 1.0, 1.0, "sqrt", with_third=False).hamiltonian(P[c])
            Hm = Geometry(m, Q[c] - h * v, 1.0, 1.0, "sqrt", with_third=False).hamiltonian(P[c])
            fd = (Hp - Hm) / (2 * h)
            dd = float(got["dHdq"][c] @ v)
            print(f"directional dH/dq chain {c}: gpu {dd:.10e} fd {fd:.10e}")
            if abs(dd - fd) > 1e-6 * max(abs(fd), np.linalg.norm(got["dHdq"][c]) * np.linalg.norm(v)):
                fails.append(("directional", c, dd, fd))
    assert not fails, fails


def test_primal_trajectory_parity(rm, oracle_model):
    """One 8-leapfrog trajectory of the D = 1 model (d = 34, eps = 0.01, 6 fixed-point iterations,
    g = sqrt(1 + lambda^2))."""
    prob = wl.solin_logistic(1, N=100, seed=1)
    m = oracle_model(prob)
    q0 = wl.random_state(prob, 1, seed=4, f_scale=0.2, u_scale=0.2)[0]
    p0 = Geometry(m, q0, 1.0, 1.0, "sqrt", with_third=False).sqrtG_z(normals(0, 0, 0, m.d))
    _, _, _, path = trajectory(m, q0, p0, 0.01, 8, 6, alpha=1.0, gkind="sqrt")
    model = rm.Model(prob, 1)
    integ = rm.Integrator(eps=0.01, n_fp=6, g_kind="sqrt", alpha=1.0)
    model.set_state(torch.tensor(q0[None], device="cuda"), torch.tensor(p0[None], device="cuda"), integ)
    q = torch.empty(1, m.d, dtype=torch.float64, device="cuda")
    p = torch.empty_like(q)
    fails = []
    for k in range(8):
        model.leapfrog(1, q, p, integ=integ)
        torch.cuda.synchronize()
        for name, g, ref in (("q", q, path[k][0]), ("p", p, path[k][1])):
            e = np.linalg.norm(g.cpu().numpy()[0] - ref) / np.linalg.norm(ref)
            print(f"leapfrog {k} {name} rel err {e:.2e}")
            if e > 1e-9:
                fails.append((k, name, e))
    assert not fails, fails


def test_primal_sampler_decisions(rm, oracle_model):
    """Algorithm 1 on the D = 1 model from a = 0, b = 0, theta = 1 (eps = 0.2, L = 10, seed 0; one
    proposal of six is rejected): the same accept/reject decisions and the same chain as the oracle."""
    prob = wl.solin_logistic(1, N=100, seed=1)
    m = oracle_model(prob)
    n_iter, eps = 6, 0.2
    ref = sample(m, np.zeros(m.d), n_iter, 0, seed=0, chain=0, eps=eps, n_leapfrog=10, n_fp=6,
                 alpha=1.0, gkind="sqrt")
    integ = rm.Integrator(eps=eps, n_leapfrog=10, n_fp=6, g_kind="sqrt", alpha=1.0)
    model = rm.Model(prob, 1)
    model.set_state(torch.zeros(1, m.d, dtype=torch.float64, device="cuda"), integ=integ)
    f64 = dict(dtype=torch.float64, device="cuda")
    qs, lp = torch.empty(n_iter, 1, m.d, **f64), torch.empty(n_iter, 1, **f64)
    acc = torch.empty(n_iter, 1, dtype=torch.int32, device="cuda")
    model.sample(n_iter, 0, 0, qs, lp, acc, integ=integ)
    torch.cuda.synchronize()
    print("accept oracle", ref["accept"], "gpu", acc.cpu().numpy()[:, 0])
    np.testing.assert_array_equal(acc.cpu().numpy()[:, 0].astype(bool), ref["accept"])
    assert ref["accept"].any() and not ref["accept"].all()
    q = qs.cpu().numpy()[:, 0]
    for i in range(n_iter):
        assert np.linalg.norm(q[i] - ref["q"][i]) <= 1e-8 * max(np.linalg.norm(ref["q"][i]), 1.0), i


def test_primal_mixed_precision(rm, oracle_model):
    prob = _problem(D=3, N=80, M=12)
    C = 2
    Q = wl.random_state(prob, C, seed=12, f_scale=0.3, u_scale=0.2)
    P = wl.random_momentum(prob, C, seed=13)
    got = _geometry(rm, prob, Q, P, None, rm.Integrator(g_kind="sqrt", alpha=1.0, precision="mixed"))
    m = oracle_model(prob)
    base = dict(BASE, dHdq=1e-5, Ginv_p=1e-6, Ham=1e-8)
    fails = []
    for c in range(C):
        geo = Geometry(m, Q[c], 1.0, 1.0, "sqrt")
        fails += _compare("primal/mixed", got, c, geo, P[c], ("U", "dU", "H", "dHdq", "Ginv_p", "Ham"), base)
    assert not fails, fails


@pytest.mark.parametrize("gkind,alpha", [("sqrt", 1.0), ("coth", 1e6)])
def test_meanvar_geometry_and_gradient_parity(rm, oracle_model, gkind, alpha):
    """The mean/variance model (Example 1, J = 2: y ~ N(F_1, delta + exp F_2), both functions on
    the same features, shared hyperparameters): every geometric quantity."""
    prob = wl.meanvar_regression(2, N=60, seed=4, M=8, n_linear=1)
    C = 3
    Q = wl.random_state(prob, C, seed=14, f_scale=0.3, u_scale=0.2)
    Q[0] = 0.0
    P = wl.random_momentum(prob, C, seed=15)
    tau = [1.0, 0.5, 0.2]
    got = _geometry(rm, prob, Q, P, tau, rm.Integrator(g_kind=gkind, alpha=alpha, jacobi_rule="relative"))
    m = oracle_model(prob)
    assert m.J == 2 and got["U"].shape == (C,)
    fails = []
    for c in range(C):
        geo = Geometry(m, Q[c], tau[c], alpha, gkind)
        fails += _compare(f"meanvar/{gkind}", got, c, geo, P[c], tuple(BASE), BASE)
    assert not fails, fails


def test_meanvar_sampler_decisions(rm, oracle_model):
    """Algorithm 1 on the J = 2 model (D = 1, N = 80, M = 12, d = 29) from all-zero coefficients
    and theta = 1 (eps = 0.05, L = 10, g = sqrt(1 + l^2)): the first proposal diverges and is
    rejected, the next five are accepted, as in the oracle, along the same chain."""
    prob = wl.meanvar_regression(1, N=80, seed=1, M=12)
    m = oracle_model(prob)
    n_iter, eps = 6, 0.05
    ref = sample(m, np.zeros(m.d), n_iter, 0, seed=0, chain=0, eps=eps, n_leapfrog=10, n_fp=6,
                 alpha=1.0, gkind="sqrt")
    integ = rm.Integrator(eps=eps, n_leapfrog=10, n_fp=6, g_kind="sqrt", alpha=1.0)
    model = rm.Model(prob, 1)
    model.set_state(torch.zeros(1, m.d, dtype=torch.float64, device="cuda"), integ=integ)
    f64 = dict(dtype=torch.float64, device="cuda")
    qs, lp = torch.empty(n_iter, 1, m.d, **f64), torch.empty(n_iter, 1, **f64)
    acc = torch.empty(n_iter, 1, dtype=torch.int32, device="cuda")
    model.sample(n_iter, 0, 0, qs, lp, acc, integ=integ)
    torch.cuda.synchronize()
    print("accept oracle", ref["accept"], "gpu", acc.cpu().numpy()[:, 0])
    np.testing.assert_array_equal(acc.cpu().numpy()[:, 0].astype(bool), ref["accept"])
    assert ref["accept"].any() and not ref["accept"].all()
    q = qs.cpu().numpy()[:, 0]
    for i in range(n_iter):
        assert np.linalg.norm(q[i] - ref["q"][i]) <= 1e-8 * max(np.linalg.norm(ref["q"][i]), 1.0), i
