"""The benchmark's CPU-baseline legs on the host (no GPU): the oracle timed on one chain with the
host's BLAS threads, and the many-chain form (one chain per process, single-threaded BLAS, a pool
started with spawn). Each runs one leapfrog per chain here, to check that it completes and that the
rates it reports are consistent with what it did."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_single_chain_leg_counts_its_leapfrogs():
    rate, n, secs = bench.oracle_leapfrogs(0.0, max_leapfrogs=1)
    assert n == 1 and secs > 0
    assert abs(rate - bench.SUBSTEPS_PER_LEAPFROG * n / secs) <= 1e-9 * rate


def test_per_core_leg_runs_spawned_processes():
    rate, procs, leapfrogs, secs = bench.oracle_per_core(0.0, max_procs=2)
    assert procs == min(2, os.cpu_count() or 1)
    assert leapfrogs >= procs and secs > 0
    # the sum of the processes' rates is at least what one process over the longest time gives
    assert rate >= bench.SUBSTEPS_PER_LEAPFROG * leapfrogs / secs / procs


def _measured_mixed_profile():
    """Category times (ms) and rates (TFLOP/s) of a measured mixed-form run (64 chains, N = 400,
    5 leapfrogs) as {name: (ms, flops, launches)}."""
    ms = {"cholesky": 86.216, "trinv": 36.026, "model": 26.797, "contract": 4.849, "vector": 25.2,
          "reorth": 5.915, "jacobi_df": 545.957, "gemm_tc": 106.821}
    tf = {"cholesky": 0.47509, "trinv": 1.13697, "vector": 0.10236, "jacobi_df": 1.45503, "gemm_tc": 639.9625}
    return {k: (v, tf.get(k, 0.0) * 1e12 * v * 1e-3, 5) for k, v in ms.items()}


def test_category_rooflines_of_a_measured_mixed_run():
    peaks = {"fp64": 1.2006, "df": 6.4826, "bf16": 1372.4}
    out = bench.category_rooflines(_measured_mixed_profile(), peaks, mixed=True)
    cats = out["categories"]
    assert abs(sum(c["share"] for c in cats.values()) - 1.0) < 1e-12
    assert list(cats)[0] == "jacobi_df"  # ordered by time
    assert abs(cats["jacobi_df"]["frac"] - 1.45503 / 6.4826) < 1e-9
    assert abs(cats["gemm_tc"]["frac"] - 639.9625 / 1372.4) < 1e-9
    # no pipe for the memory-bound phases, nor for the mixed Cholesky / L^-1
    for name in ("model", "contract", "vector", "reorth", "cholesky", "trinv"):
        assert "frac" not in cats[name]
    assert abs(cats["trinv"]["achieved_fp64_equivalent"] - 1.13697) < 1e-9
    st = out["step"]
    ideal = 545.957 * 1.45503 / 6.4826 + 106.821 * 639.9625 / 1372.4
    assert abs(st["ideal_ms"] - ideal) < 1e-6
    assert abs(st["measured_ms"] - sum(v[0] for v in _measured_mixed_profile().values())) < 1e-9
    assert st["frac"] < st["frac_counted"] < 1.0


def test_prerotation_is_rated_against_the_double_float_peak():
    """The pre-rotation's counted work (double-float multiply-adds) is rated against the measured
    Dot2 peak, per category and, when it dominates the step, in the headline roofline (whose traffic
    stays null: no capture of it feeds the table of DRAM bytes)."""
    ms = {"gemm_tc": 203.472, "jacobi_df": 185.624, "cholesky": 152.726, "prerotation": 139.724}
    tf = {"gemm_tc": 647.136, "jacobi_df": 0.85686, "prerotation": 0.92389}
    prof = {k: (v, tf.get(k, 0.0) * 1e12 * v * 1e-3, 61) for k, v in ms.items()}
    out = bench.category_rooflines(prof, {"fp64": 1.2, "df": 6.45, "bf16": 1372.4}, mixed=True)
    c = out["categories"]["prerotation"]
    assert c["pipe"] == "df" and abs(c["frac"] - 0.92389 / 6.45) < 1e-9

    class PeakProbes:
        def df_peak_tflops(self, n):
            return 6.45

        def fp32_peak_tflops(self, n):
            return 75.0

        def fp64_peak_tflops(self, n):
            return 1.2

    r = bench._roofline(PeakProbes(), {"prerotation": prof["prerotation"], "vector": (52.6, 0.0, 61)}, 64)
    assert r["kernel"] == "prerotation" and r["peak"] == 6.45 and r["traffic"] is None
    assert abs(r["frac"] - 0.92389 / 6.45) < 1e-6


def test_category_rooflines_fp64_run_uses_the_fp64_pipe():
    prof = {"gemm_f64": (1370.0, 0.8465e12 * 1.370, 40), "cholesky": (102.0, 0.4e12 * 0.102, 13),
            "model": (27.0, 0.0, 30)}
    out = bench.category_rooflines(prof, {"fp64": 1.2}, mixed=False)
    assert out["categories"]["cholesky"]["pipe"] == "fp64"
    assert abs(out["categories"]["gemm_f64"]["frac"] - 0.8465 / 1.2) < 1e-9
    assert bench.category_rooflines(prof, {})["step"]["ideal_ms"] == 0.0  # no peaks measured


def test_oracle_pool_is_bounded_by_the_container():
    assert 1 <= bench.host_cores() <= len(os.sched_getaffinity(0))
    free = bench.host_free_bytes()
    assert free is None or free > 0


def test_cgroup_memory_limit_bounds_the_free_bytes(tmp_path):
    lim, use = tmp_path / "max", tmp_path / "current"
    lim.write_text("10000000000\n")
    use.write_text("4000000000\n")
    got = bench.host_free_bytes(((str(lim), str(use)),))
    assert got <= 6_000_000_000
    lim.write_text("max\n")  # no limit: only what the OS reports
    assert bench.host_free_bytes(((str(lim), str(use)),)) == bench.host_free_bytes(())
    assert bench.host_free_bytes(((str(tmp_path / "missing"), str(use)),)) == bench.host_free_bytes(())


def test_per_core_worker_runs_without_threadpoolctl(monkeypatch):
    # the GPU hosts may not have threadpoolctl: the worker then relies on the BLAS thread
    # variables its parent sets before spawning it
    monkeypatch.setitem(sys.modules, "threadpoolctl", None)
    rate, n, secs = bench._oracle_one_core((0.0, 1))
    assert n == 1 and rate > 0 and secs > 0


def test_per_core_leg_restores_the_blas_thread_variables(monkeypatch):
    monkeypatch.setenv("OMP_NUM_THREADS", "3")
    monkeypatch.delenv("OPENBLAS_NUM_THREADS", raising=False)
    bench.oracle_per_core(0.0, max_procs=1)
    assert os.environ["OMP_NUM_THREADS"] == "3"
    assert "OPENBLAS_NUM_THREADS" not in os.environ


def test_oracle_chain_is_algorithm_1():
    # ten leapfrogs of the timed chain make one Algorithm 1 iteration: the same proposal, test and
    # kept state as the oracle's sampler with the same seed
    import numpy as np
    from oracle.sampler import sample
    chain = bench.OracleChain(seed=3, n_inputs=12)
    for _ in range(bench.N_LEAPFROG):
        assert chain.leapfrog()
    assert chain.it == 1 and chain.accepted + chain.rejected == 1
    ref = sample(chain.model, np.zeros(chain.model.d), 1, 0, 3, 0, bench.EPS, bench.N_LEAPFROG, bench.N_FP)
    assert bool(ref["accept"][0]) == (chain.accepted == 1)
    assert np.array_equal(ref["q"][0], chain.q)
