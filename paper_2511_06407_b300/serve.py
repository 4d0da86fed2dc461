"""Continuous-batching server for sampling jobs.

A job is one problem (workload dict) sampled by n_chains chains, each with its own inverse
temperature, for n_burn + n_iter Algorithm-1 iterations. The server admits jobs in arrival order as
soon as (a) they have arrived and (b) their device footprint (rmhmc_plan_bytes) fits in what is left
of the HBM budget; every admitted job owns a model and a CUDA stream, so jobs of different sizes run
concurrently and their kernels overlap on the GPU. The host loop tops every active job up to
`depth` iterations in flight (one rmhmc_sample call of one iteration each, recorded in-place into
the job's device-resident result buffers), retires jobs whose last iteration has finished (CUDA
event query, no host synchronisation), frees their memory and admits the next jobs: new jobs join
while others are running. Each job's computation touches only its own model, so its result is the
same alone and in any mix.

Latency = finish time - arrival time; p50 / p99 over the jobs of a trace.
"""
import time
from dataclasses import dataclass, field

import numpy as np

from . import rmhmc


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

    @property
    def latency(self):
        return None if self.finished is None else self.finished - self.arrival


class _Active:
    def __init__(self, job, device):
        import torch
        self.job = job
        self.stream = torch.cuda.Stream(device=device)
        with torch.cuda.stream(self.stream):
            self.model = rmhmc.Model(job.problem, job.n_chains, job.tau, stream=self.stream)
            d = self.model.d
            f64 = dict(dtype=torch.float64, device=device)
            self.q = torch.empty(job.n_iter, job.n_chains, d, **f64)
            self.logp = torch.empty(job.n_iter, job.n_chains, **f64)
            self.acc = torch.empty(job.n_iter, job.n_chains, dtype=torch.int32, device=device)
            self.status = torch.zeros(job.n_chains, dtype=torch.int32, device=device)
            self.st_iter = torch.empty(job.n_chains, dtype=torch.int32, device=device)
            self.model.set_state(torch.zeros(job.n_chains, d, **f64), integ=job.integ)
        self.enqueued = 0           # iterations enqueued (burn-in included)
        self.events = []            # (iteration index, event) not yet known complete
        self.total = job.n_burn + job.n_iter

    def top_up(self, depth):
        """Enqueue iterations until `depth` are in flight."""
        import torch
        job = self.job
        while self.enqueued < self.total and len(self.events) < depth:
            it = self.enqueued
            with torch.cuda.stream(self.stream):
                if it < job.n_burn:
                    self.model.sample(0, 1, job.seed, chain_status=self.st_iter, integ=job.integ)
                else:
                    r = it - job.n_burn
                    self.model.sample(1, 0, job.seed, self.q[r:r + 1], self.logp[r:r + 1],
                                      self.acc[r:r + 1], chain_status=self.st_iter, integ=job.integ)
                self.status.bitwise_or_(self.st_iter)
                ev = torch.cuda.Event()
                ev.record(self.stream)
            self.events.append((it, ev))
            self.enqueued += 1

    def poll(self):
        """Drop completed events; True when the last iteration has completed."""
        while self.events and self.events[0][1].query():
            self.events.pop(0)
        return self.enqueued == self.total and not self.events

    def harvest(self):
        import torch
        job = self.job
        with torch.cuda.stream(self.stream):
            job.q_samples = self.q.cpu().numpy()
            job.logp = self.logp.cpu().numpy()
            job.accept = self.acc.cpu().numpy()
            job.chain_status = self.status.cpu().numpy()
        self.model.close()


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
        active, done, used = [], [], 0
        t0 = time.perf_counter()
        max_active = 0
        while pending or active:
            now = time.perf_counter() - t0
            if not realtime and not active and pending:
                now = max(now, pending[0].arrival)
            # admit in arrival order while the head of the queue has arrived and fits
            while pending and (pending[0].arrival <= now or not realtime) and used + pending[0].bytes <= self.budget:
                job = pending.pop(0)
                job.admitted = time.perf_counter() - t0
                active.append(_Active(job, self.device))
                used += job.bytes
                if log:
                    log(f"t={job.admitted:.2f}s admit job {job.job_id} ({job.bytes / 2**20:.0f} MiB, "
                        f"{len(active)} active)")
            max_active = max(max_active, len(active))
            for a in active:
                a.top_up(self.depth)
            still = []
            for a in active:
                if a.poll():
                    a.harvest()
                    a.job.finished = time.perf_counter() - t0
                    used -= a.job.bytes
                    done.append(a.job)
                    if log:
                        log(f"t={a.job.finished:.2f}s done job {a.job.job_id} latency {a.job.latency:.2f}s")
                else:
                    still.append(a)
            active = still
            if active:
                time.sleep(0.0005)
        makespan = time.perf_counter() - t0
        lat = np.array([j.latency for j in done])
        substeps = sum((j.n_iter + j.n_burn) * j.n_chains * j.integ.n_leapfrog * (2 * j.integ.n_fp + 1)
                       for j in done)
        stats = {"jobs": len(done), "makespan_s": makespan, "p50_latency_s": float(np.percentile(lat, 50)),
                 "p99_latency_s": float(np.percentile(lat, 99)), "substeps_per_s": substeps / makespan,
                 "max_concurrent_jobs": max_active}
        return sorted(done, key=lambda j: j.job_id), stats


def poisson_trace(problems, rate_per_s, seed=0):
    """Arrival times of a Poisson process of the given rate, one per problem."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_per_s, len(problems)))
    return [float(x) for x in t]
