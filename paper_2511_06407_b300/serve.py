"""Continuous-batching server for sampling jobs: the trace-driven client of the library's native
server (rmhmc_server_*, include/rmhmc.h).

A job is one problem (workload dict) sampled by n_chains chains, each with its own inverse
temperature, for n_burn + n_iter Algorithm-1 iterations. Admission, execution and completion run in
the library's scheduler thread: jobs are admitted in submission order as soon as their device
footprint (rmhmc_plan_bytes plus the server's per-job buffers) fits in what is left of the HBM
budget, every admitted job owns a model and a CUDA stream (so jobs of different sizes run
concurrently and their kernels overlap), `depth` iterations are kept in flight per job, and a
finished job's memory returns to the budget at once, so new jobs join while others run. This module
only submits each job at its arrival time, gives it device result buffers and collects the results.
Each job's computation touches only its own model, so its result is the same alone and in any mix.

Latency = finish time - arrival time (the server's clock); p50 / p99 over the jobs of a trace.
"""
import time
from dataclasses import dataclass, field

import numpy as np

from . import rmhmc
from . import workloads as wl


@dataclass
class Job:
    problem: dict
    n_chains: int
    n_iter: int
    n_burn: int = 0
    seed: int = 0
    tau: object = None
    integ: rmhmc.Integrator = field(default_factory=rmhmc.Integrator)
    arrival: float = 0.0          # seconds after the trace starts
    job_id: int = -1
    # filled in by the server
    admitted: float = None
    finished: float = None
    bytes: int = 0
    q_samples: object = None      # host (n_iter, n_chains, d)
    logp: object = None           # host (n_iter, n_chains)
    accept: object = None         # host (n_iter, n_chains)
    chain_status: object = None   # host (n_chains,)
    loglik: object = None         # host (n_iter, n_chains): untempered ln P(y | F) per sample

    @property
    def latency(self):
        return None if self.finished is None else self.finished - self.arrival


class Server:
    """Admission by HBM budget, device-resident chain state, concurrent jobs on their own streams."""

    def __init__(self, hbm_budget_bytes, depth=2, device=0):
        self.budget = int(hbm_budget_bytes)
        self.depth = depth
        self.device = device

    def run(self, jobs, realtime=True, log=None):
        """Serve a trace of jobs (arrival times in seconds from the start). Returns the jobs with
        their results and timings, and summary statistics."""
        import torch
        torch.cuda.set_device(self.device)
        pending = sorted(jobs, key=lambda j: j.arrival)
        for i, j in enumerate(pending):
            if j.job_id < 0:
                j.job_id = i
            j.bytes = rmhmc.plan_bytes(j.problem, j.n_chains)
            if j.bytes > self.budget:
                raise ValueError(f"job {j.job_id} needs {j.bytes} bytes, more than the whole budget")
        srv = rmhmc.NativeServer(self.budget, self.depth, self.device)
        running, done = {}, []
        try:
            while pending or running:
                now = srv.stats()["now"]
                while pending and (pending[0].arrival <= now or not realtime):
                    job = pending.pop(0)
                    d = wl.dims(job.problem)[2]
                    dev = f"cuda:{self.device}"
                    out = (torch.empty(job.n_iter, job.n_chains, d, dtype=torch.float64, device=dev),
                           torch.empty(job.n_iter, job.n_chains, dtype=torch.float64, device=dev),
                           torch.empty(job.n_iter, job.n_chains, dtype=torch.int32, device=dev),
                           torch.zeros(job.n_chains, dtype=torch.int32, device=dev),
                           torch.empty(job.n_iter, job.n_chains, dtype=torch.float64, device=dev))
                    jid = srv.submit(job.problem, job.n_chains, job.integ, job.n_iter, job.n_burn, job.seed,
                                     job.tau, None, *out)
                    running[jid] = (job, out)
                    if log:
                        log(f"t={now:.2f}s submit job {job.job_id} ({job.bytes / 2**20:.0f} MiB)")
                for jid in list(running):
                    state, err, times = srv.poll(jid)
                    if state in ("queued", "running"):
                        continue
                    job, out = running.pop(jid)
                    if state == "failed":
                        raise rmhmc.RmhmcError(f"job {job.job_id} failed: {rmhmc.lib().rmhmc_status_string(err).decode()}")
                    job.admitted, job.finished = times[1], times[2]
                    job.q_samples, job.logp, job.accept, job.chain_status, job.loglik = (x.cpu().numpy() for x in out)
                    done.append(job)
                    if log:
                        log(f"t={job.finished:.2f}s done job {job.job_id} latency {job.latency:.2f}s")
                if running or pending:
                    time.sleep(0.0005)
            stats = srv.stats()
        finally:
            srv.close()
        return sorted(done, key=lambda j: j.job_id), trace_summary(done, stats["max_active"])


def trace_summary(done, max_active):
    """Statistics of a served trace: p50 / p99 of the jobs' latencies (finish - arrival), the
    makespan (the last finish on the server's clock) and the leapfrog substeps of all jobs per
    second of makespan (n_fp fixed-point iterations for each implicit half plus the explicit one)."""
    makespan = max(j.finished for j in done) if done else 0.0
    lat = np.array([j.latency for j in done], dtype=np.float64)
    substeps = sum((j.n_iter + j.n_burn) * j.n_chains * j.integ.n_leapfrog * (2 * j.integ.n_fp + 1)
                   for j in done)
    return {"jobs": len(done), "makespan_s": makespan,
            "p50_latency_s": float(np.percentile(lat, 50)) if len(lat) else None,
            "p99_latency_s": float(np.percentile(lat, 99)) if len(lat) else None,
            "substeps_per_s": substeps / makespan if makespan > 0 else None,
            "max_concurrent_jobs": max_active}


def poisson_trace(problems, rate_per_s, seed=0):
    """Arrival times of a Poisson process of the given rate, one per problem."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_per_s, len(problems)))
    return [float(x) for x in t]
