"""Uneven batches in one CUDA graph, the Jacobi autotuner, and the continuous-batching server."""
import numpy as np
import pytest

from paper_2511_06407_b300 import workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rm():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2511_06407_b300 import build, rmhmc
    build.build()
    return rmhmc


def _uneven_problems():
    return [(wl.gp_classification(30, seed=1), 3), (wl.propensity(24, seed=2, n_kernels=2), 2),
            (wl.propensity(41, seed=3, n_kernels=3), 4)]


def _make(rm, prob, C, seed, integ):
    s = torch.cuda.Stream()
    m = rm.Model(prob, C, stream=s)
    q = torch.tensor(wl.random_state(prob, C, seed=seed, f_scale=0.2, u_scale=0.1), device="cuda")
    p = torch.tensor(0.3 * wl.random_momentum(prob, C, seed=seed + 100), device="cuda")
    with torch.cuda.stream(s):
        m.set_state(q, p, integ=integ)
    return m, s


def _state(m, s, integ):
    q = torch.empty(m.n_chains, m.d, dtype=torch.float64, device="cuda")
    p = torch.empty_like(q)
    with torch.cuda.stream(s):
        m.leapfrog(0, q, p, integ=integ)
    torch.cuda.synchronize()
    return q.cpu().numpy(), p.cpu().numpy()


def test_uneven_batch_graph_equals_individual_leapfrogs(rm):
    """Three problems of different d (30, 52, 129) advanced by one captured CUDA graph per leapfrog
    give exactly the states of the same models advanced one by one."""
    integ = rm.Integrator(eps=0.01, n_fp=4)
    probs = _uneven_problems()
    solo = [_make(rm, p, C, 10 + i, integ) for i, (p, C) in enumerate(probs)]
    group = [_make(rm, p, C, 10 + i, integ) for i, (p, C) in enumerate(probs)]
    for m, s in solo:
        with torch.cuda.stream(s):
            m.leapfrog(3, integ=integ)
    batch = rm.Batch([m for m, _ in group])
    batch.leapfrog(2, integ)      # captures the graph, replays twice
    batch.leapfrog(1, integ)      # replays the captured graph
    torch.cuda.synchronize()
    for (ms, ss), (mg, sg) in zip(solo, group):
        qs, ps = _state(ms, ss, integ)
        qg, pg = _state(mg, sg, integ)
        np.testing.assert_array_equal(qs, qg)
        np.testing.assert_array_equal(ps, pg)
    batch.close()


def test_uneven_batch_chains_match_the_oracle(rm, oracle_model):
    """The batched form on a small uneven batch (6 problems, N ~ U{20..60}, 1-3 additive kernels,
    2 chains each, d from 51 to 153), advanced by the batch's captured graph for 2 leapfrogs: every
    chain against the FP64 oracle's generalized leapfrog from the same (q, p), under the parity
    rule (16 x the oracle's LU-vs-Cholesky spread after several leapfrogs, 1e-8 relative floor)."""
    from oracle import model as mdl
    from oracle.integrator import trajectory
    integ = rm.Integrator(eps=0.002, n_fp=4)  # (0.01 leaves the PD region for two of these problems)
    probs = wl.uneven_batch(6, seed=3, n_min=20, n_max=60)
    made = [_make(rm, p, 2, 30 + i, integ) for i, p in enumerate(probs)]
    batch = rm.Batch([m for m, _ in made])
    batch.leapfrog(2, integ)
    torch.cuda.synchronize()
    fails = []
    for i, (prob, (m, s)) in enumerate(zip(probs, made)):
        qg, pg = _state(m, s, integ)
        om = oracle_model(prob)
        Q0 = wl.random_state(prob, 2, seed=30 + i, f_scale=0.2, u_scale=0.1)
        P0 = 0.3 * wl.random_momentum(prob, 2, seed=130 + i)
        for c in range(2):
            qr, pr, _, _ = trajectory(om, Q0[c], P0[c], 0.002, 2, 4)
            with mdl.inverse_method("cholesky"):
                qa, pa, _, _ = trajectory(om, Q0[c], P0[c], 0.002, 2, 4)
            for name, g, r, a in (("q", qg[c], qr, qa), ("p", pg[c], pr, pa)):
                err = np.linalg.norm(g - r)
                tol = max(1e-8 * np.linalg.norm(r), 16.0 * np.linalg.norm(r - a))
                print(f"problem {i} (d={om.d}) chain {c} {name}: {err / np.linalg.norm(r):.1e} / "
                      f"{tol / np.linalg.norm(r):.0e}")
                if not err <= tol:
                    fails.append((i, c, name, err, tol))
    batch.close()
    assert not fails, fails


def test_autotune_picks_a_cluster_and_schedule_and_keeps_the_state(rm, oracle_model):
    """The autotuner times one leapfrog per (cluster size, rotation schedule) and then restores the
    state: the potential at q is recomputed bit for bit and dH/dq still matches the oracle."""
    from oracle.geometry import Geometry
    integ = rm.Integrator(eps=0.01, n_fp=4)
    prob = wl.gp_classification(40, seed=4)
    m, s = _make(rm, prob, 4, 7, integ)
    U0 = torch.empty(4, dtype=torch.float64, device="cuda")
    with torch.cuda.stream(s):
        m.geometry(U=U0)
        c, sched, tile, pre = m.autotune(integ)
        U1 = torch.empty_like(U0)
        m.geometry(U=U1)
        dHdq = torch.empty(4, m.d, dtype=torch.float64, device="cuda")
        P = wl.random_momentum(prob, 4, seed=8)
        m.hamiltonian_grad(torch.tensor(P, device="cuda"), dHdq=dHdq)
    torch.cuda.synchronize()
    assert c in (1, 2, 4, 8) and sched in ("cyclic", "dynamic") and tile in (64, 32)
    np.testing.assert_array_equal(U0.cpu().numpy(), U1.cpu().numpy())
    q = wl.random_state(prob, 4, seed=7, f_scale=0.2, u_scale=0.1)
    ref = Geometry(oracle_model(prob), q[2], 1.0).dHdq(P[2])
    assert np.linalg.norm(dHdq.cpu().numpy()[2] - ref) <= 1e-6 * np.linalg.norm(ref)


def test_server_results_are_the_same_alone_and_in_the_mix(rm):
    from paper_2511_06407_b300.serve import Job, Server
    integ = rm.Integrator(eps=0.01, n_leapfrog=3, n_fp=4)
    probs = _uneven_problems()
    taus = [np.linspace(0.2, 1.0, C) for _, C in probs]

    def jobs(arrivals):
        return [Job(p, C, n_iter=3, n_burn=1, seed=5 + i, tau=taus[i], integ=integ, arrival=a, job_id=i)
                for i, ((p, C), a) in enumerate(zip(probs, arrivals))]

    mixed, stats = Server(hbm_budget_bytes=2**30).run(jobs([0.0, 0.0, 0.01]))
    assert stats["jobs"] == 3 and stats["max_concurrent_jobs"] >= 2
    assert stats["p50_latency_s"] > 0 and stats["p99_latency_s"] >= stats["p50_latency_s"]
    for i in range(3):
        alone, _ = Server(hbm_budget_bytes=2**30).run([jobs([0.0, 0.0, 0.0])[i]])
        np.testing.assert_array_equal(alone[0].q_samples, mixed[i].q_samples)
        np.testing.assert_array_equal(alone[0].logp, mixed[i].logp)
        np.testing.assert_array_equal(alone[0].accept, mixed[i].accept)


def test_server_admits_by_hbm_budget(rm):
    """With a budget that fits one job at a time, jobs run one after another (never two resident)."""
    from paper_2511_06407_b300.serve import Job, Server
    integ = rm.Integrator(eps=0.01, n_leapfrog=2, n_fp=3)
    prob = wl.gp_classification(30, seed=1)
    need = rm.plan_bytes(prob, 2)
    js = [Job(prob, 2, n_iter=2, seed=i, integ=integ, arrival=0.0, job_id=i) for i in range(3)]
    done, stats = Server(hbm_budget_bytes=int(need * 1.5)).run(js)
    assert stats["max_concurrent_jobs"] == 1 and stats["jobs"] == 3
    for a, b in zip(done, done[1:]):
        assert b.admitted >= a.finished - 1e-3


def test_native_server_jobs_equal_one_sample_call(rm):
    """rmhmc_server_*: two jobs submitted together run concurrently, one iteration per call, and
    each one's samples, log densities, accept flags and chain status equal those of a single
    rmhmc_sample(n_iter, n_burn, seed) call on a model of its own; the bookkeeping (states, times,
    budget in use) is consistent, and a job larger than the whole budget is refused."""
    integ = rm.Integrator(eps=0.01, n_leapfrog=2, n_fp=3)
    probs = [wl.gp_classification(30, seed=1), wl.gp_classification(45, seed=2)]
    C, n_iter, n_burn = 3, 3, 1
    f64 = dict(dtype=torch.float64, device="cuda")
    i32 = dict(dtype=torch.int32, device="cuda")
    srv = rm.NativeServer(2**30, depth=2)
    ids, outs = [], []
    for i, p in enumerate(probs):
        d = wl.dims(p)[2]
        o = (torch.empty(n_iter, C, d, **f64), torch.empty(n_iter, C, **f64), torch.empty(n_iter, C, **i32),
             torch.zeros(C, **i32))
        ids.append(srv.submit(p, C, integ, n_iter, n_burn, 11 + i, None, None, *o))
        outs.append(o)
    srv.wait()
    st = srv.stats()
    assert st["active"] == 0 and st["queued"] == 0 and st["bytes_in_use"] == 0 and st["max_active"] >= 1
    for jid in ids:
        state, err, (t_sub, t_adm, t_fin) = srv.poll(jid)
        assert state == "done" and err == 0 and 0 <= t_sub <= t_adm <= t_fin
    for i, p in enumerate(probs):
        m = rm.Model(p, C)
        d = m.d
        m.set_state(torch.zeros(C, d, **f64), integ=integ)
        q, lp = torch.empty(n_iter, C, d, **f64), torch.empty(n_iter, C, **f64)
        acc, cs = torch.empty(n_iter, C, **i32), torch.zeros(C, **i32)
        m.sample(n_iter, n_burn, 11 + i, q, lp, acc, chain_status=cs, integ=integ)
        torch.cuda.synchronize()
        m.close()
        for got, want in zip(outs[i], (q, lp, acc, cs)):
            np.testing.assert_array_equal(got.cpu().numpy(), want.cpu().numpy())
    srv.close()
    small = rm.NativeServer(4096)
    with pytest.raises(rm.RmhmcError):
        small.submit(probs[0], C, integ, 1, 0, 0)
    small.close()


def test_served_tempered_job_matches_the_oracle(rm):
    """A served job against the FP64 oracle's Algorithm 1 directly: the N = 30 problem, 2 chains at
    inverse temperatures 1 and 0.5, 1 burn-in + 4 recorded iterations (L = 3, eps = 0.01, 3
    fixed-point iterations) from f = 0, u = 0, seed 5, submitted together with a second job. Same
    accept/reject decisions, the samples and log posteriors within the parity rule (16 x the oracle's
    LU-vs-Cholesky spread, or a floor: 1e-8 relative for the first trajectory's sample, growing by
    3e-9 per leapfrog run since the start, and 1e-10 for log P; log P also its first-order change with the sample's
    own deviation and the error of rounding K to FP64),
    and the recorded untempered ln P(y|F) per sample."""
    import oracle_pool
    from conftest import potential_rounding_bound
    from oracle import model as mdl
    prob = wl.gp_classification(30, seed=1)
    taus = np.array([1.0, 0.5])
    C, n_iter, n_burn, seed = 2, 4, 1, 5
    integ = rm.Integrator(eps=0.01, n_leapfrog=3, n_fp=3)
    f64 = dict(dtype=torch.float64, device="cuda")
    i32 = dict(dtype=torch.int32, device="cuda")
    d = wl.dims(prob)[2]
    srv = rm.NativeServer(2**30, depth=2)
    out = (torch.empty(n_iter, C, d, **f64), torch.empty(n_iter, C, **f64), torch.empty(n_iter, C, **i32),
           torch.zeros(C, **i32), torch.empty(n_iter, C, **f64))
    srv.submit(prob, C, integ, n_iter, n_burn, seed, taus, None, *out)
    other = wl.gp_classification(45, seed=2)  # a second job in the mix
    o2 = (torch.empty(2, 3, wl.dims(other)[2], **f64), torch.empty(2, 3, **f64), torch.empty(2, 3, **i32),
          torch.zeros(3, **i32))
    srv.submit(other, 3, integ, 2, 0, 9, None, None, *o2)
    srv.wait()
    srv.close()
    q, lp, acc, cs, ll = (x.cpu().numpy() for x in out)
    assert not cs.any(), cs
    jobs = []
    for c in range(C):
        kw = dict(n_iter=n_iter, n_burn=n_burn, seed=seed, chain=c, eps=0.01, n_leapfrog=3, n_fp=3,
                  tau=float(taus[c]))
        jobs += [(prob, "lu", kw), (prob, "cholesky", kw)]
    res = oracle_pool.run(oracle_pool.sample_job, jobs)
    m = mdl.from_problem(prob)
    for c in range(C):
        ref, alt = res[2 * c], res[2 * c + 1]
        np.testing.assert_array_equal(acc[:, c].astype(bool), ref["accept"])
        for i in range(n_iter):
            # the 1e-8 trajectory target grows by 3e-9 per leapfrog run so far: the samples are the
            # ends of (n_burn + i + 1) x 3 leapfrogs, each adding the eigen-update's rounding (the
            # measured drift is ~1.3e-9 relative per leapfrog on this problem)
            base_q = max(1e-8, 3e-9 * (n_burn + i + 1) * 3)
            for name, g, r, a, base in (("q", q[i, c], ref["q"][i], alt["q"][i], base_q),
                                        ("logp", lp[i, c], ref["logp"][i], alt["logp"][i], 1e-10)):
                err = float(np.linalg.norm(np.asarray(g) - r))
                tol = max(base * float(np.linalg.norm(r)), 16.0 * float(np.linalg.norm(np.asarray(r) - a)))
                if name == "logp":
                    # log P at the kept sample also moves with the sample's own (validated) deviation,
                    # to first order |dU . dq|, and rounding K to FP64 bounds any evaluation of U
                    dq = q[i, c] - ref["q"][i]
                    du = mdl.gradient(m, ref["q"][i], float(taus[c]))
                    tol = max(tol, 2.0 * abs(float(du @ dq)) + potential_rounding_bound(m, ref["q"][i]))
                assert err <= tol, (c, i, name, err, tol)
            # the recorded untempered log-likelihood -sum l(F) of the kept sample (Bernoulli-logistic)
            f, _ = mdl.split(m, q[i, c])
            want = -float(np.sum(mdl.lik_derivs(m, f.sum(axis=0))[0]))
            assert abs(ll[i, c] - want) <= 1e-10 * max(1.0, abs(want)), (c, i, ll[i, c], want)
