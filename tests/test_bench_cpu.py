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
