"""Host-side pieces of the serving client (CPU only): the Poisson arrival trace and the trace
statistics (latency percentiles, makespan, throughput) computed from finished jobs."""
import numpy as np

from paper_2511_06407_b300 import rmhmc
from paper_2511_06407_b300.serve import Job, poisson_trace, trace_summary


def test_poisson_trace_has_the_requested_rate():
    t = np.array(poisson_trace([None] * 4000, rate_per_s=50.0, seed=3))
    assert np.all(np.diff(t) > 0) and t[0] > 0
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1 / 50.0) < 4 * (1 / 50.0) / np.sqrt(len(gaps))
    assert poisson_trace([None] * 5, 2.0, seed=1) == poisson_trace([None] * 5, 2.0, seed=1)


def test_trace_summary_from_finished_jobs():
    integ = rmhmc.Integrator(n_leapfrog=4, n_fp=6)
    jobs = []
    for i, (arr, fin) in enumerate([(0.5, 3.0), (1.0, 2.0), (1.5, 6.5), (2.0, 4.0)]):
        j = Job(problem={}, n_chains=16, n_iter=6, n_burn=2, integ=integ, arrival=arr, job_id=i)
        j.finished = fin
        jobs.append(j)
    out = trace_summary(jobs, max_active=3)
    lat = np.array([2.5, 1.0, 5.0, 2.0])
    assert out["jobs"] == 4 and out["makespan_s"] == 6.5 and out["max_concurrent_jobs"] == 3
    assert out["p50_latency_s"] == np.percentile(lat, 50) == 2.25
    assert abs(out["p99_latency_s"] - np.percentile(lat, 99)) < 1e-12
    # 4 jobs x 8 iterations x 16 chains x 4 leapfrogs x 13 substeps over 6.5 s
    assert abs(out["substeps_per_s"] - 4 * 8 * 16 * 4 * 13 / 6.5) < 1e-9
    empty = trace_summary([], max_active=0)
    assert empty["jobs"] == 0 and empty["p50_latency_s"] is None and empty["substeps_per_s"] is None
