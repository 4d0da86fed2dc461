#!/usr/bin/env python
"""Benchmark: SoftAbs-RMHMC generalized-leapfrog substeps per second on B300.

Workload (default): GP binary classification, N = 400 inputs x ~ U[-1, 1]^2, SE kernel with log
amplitude and log lengthscale (d = 402), 64 chains in one batch, plain FP64 path, soft-abs
alpha = 1e6, eps = 0.1, 6 fixed-point iterations. A step is one generalized leapfrog of every chain:
13 substeps per chain (6 implicit-momentum iterations, 6 implicit-position iterations, 1 explicit
half-step). value = chains x 13 x steps / seconds, whole job over all ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl b300|reference]

N > 1 runs under torch.distributed.run: every rank runs its own 64-chain replica (the chains are
independent; there is no collective on the data path) and the slowest rank's time is used.
--impl reference times the plain FP64 CPU oracle on the host cores instead (bounded samples).
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2511_06407_b300 import workloads as wl  # noqa: E402

N_INPUTS, N_CHAINS, EPS, N_FP = 400, 64, 0.005, 6
# DRAM bytes per k_jacobi launch per chain, from the ncu capture summarised in
# profiles/k_jacobi_N400_8chains.md (8 chains: 22.27 MB read + 2.18 MB written on average per launch);
# traffic grows with the number of chains, so a 64-chain launch is scaled by 64 / 8.
JACOBI_DRAM_BYTES_PER_CHAIN = (22.27e6 + 0.5 * (2.40e6 + 1.95e6)) / 8
SUBSTEPS_PER_LEAPFROG = 2 * N_FP + 1
METRIC = "RMHMC leapfrog substeps/s"
UNIT = "substeps/s"
WORKLOAD = (f"GP classification N={N_INPUTS} (d={N_INPUTS + 2}), SE kernel, {N_CHAINS} chains batched, "
            f"plain FP64, alpha=1e6, eps={EPS}, n_fp={N_FP}")


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows if len(r) >= 9 for i in range(4)
                          if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm)}


def cpu_cores_used():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads", 1) for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return int(max(n))
    except Exception:
        pass
    return os.cpu_count() or 1


def oracle_leapfrogs(seconds, max_leapfrogs=None):
    """Time the plain FP64 oracle on one chain of the benchmark workload for about `seconds`
    (at least one leapfrog). Returns (substeps/s, leapfrogs done, seconds)."""
    from oracle.geometry import Geometry
    from oracle.integrator import leapfrog
    from oracle.model import from_problem
    prob = wl.gp_classification(N_INPUTS, seed=0)
    m = from_problem(prob)
    rng = np.random.default_rng(0)
    geo0 = Geometry(m, np.zeros(m.d), 1.0)
    q, geo = np.zeros(m.d), geo0
    p = geo.sqrtG_z(rng.standard_normal(m.d))
    n, t0 = 0, time.perf_counter()
    while True:
        try:
            with np.errstate(all="ignore"):
                q, p, geo = leapfrog(m, q, p, EPS, N_FP, geo=geo)
            n += 1
        except np.linalg.LinAlgError:
            # the trajectory left the region where K is positive definite: restart from f = 0,
            # u = 0 with a fresh momentum (only completed leapfrogs are counted)
            q, geo = np.zeros(m.d), geo0
            p = geo.sqrtG_z(rng.standard_normal(m.d))
        el = time.perf_counter() - t0
        if (el >= seconds and n > 0) or (max_leapfrogs and n >= max_leapfrogs):
            break
    return SUBSTEPS_PER_LEAPFROG * n / el, n, el


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    # warm-up and timed steps: each step is a bounded sample (one oracle leapfrog of one chain)
    for _ in range(args.warmup):
        oracle_leapfrogs(0.0, max_leapfrogs=1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_leapfrogs(0.0, max_leapfrogs=1)
    el = time.perf_counter() - t0
    value = SUBSTEPS_PER_LEAPFROG * args.steps / el
    cores = cpu_cores_used()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": N_INPUTS, "d": N_INPUTS + 2, "chains": N_CHAINS},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "one chain of the workload, one leapfrog per step (numpy/LAPACK FP64, "
                                       "full third-derivative tensor)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_b300(args):
    import torch
    import torch.distributed as dist
    from paper_2511_06407_b300 import build, rmhmc
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0 or ws == 1:
        build.build()
    if ws > 1:
        dist.barrier()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    prob = wl.gp_classification(N_INPUTS, seed=0)
    C = args.chains
    model = rmhmc.Model(prob, C, stream=stream)
    d = model.d
    integ = rmhmc.Integrator(eps=EPS, n_fp=N_FP, n_leapfrog=1)
    q0 = torch.zeros(C, d, dtype=torch.float64, device=dev)
    model.set_state(q0, integ=integ)
    qo = torch.empty(C, d, dtype=torch.float64, device=dev)
    po = torch.empty_like(qo)
    Ho = torch.empty(C, dtype=torch.float64, device=dev)
    st = torch.empty(C, dtype=torch.int32, device=dev)

    # ---- warm-up: one Algorithm 1 iteration (momenta p ~ N(0, G) drawn by the library, one
    # leapfrog, Metropolis-Hastings), then plain leapfrogs
    model.sample(1, 0, 1234 + rank, integ=integ)
    if args.warmup > 1:
        model.leapfrog(args.warmup - 1, integ=integ)
    model.leapfrog(0, qo, po, integ=integ)
    p0 = po.clone()
    torch.cuda.synchronize()
    # ---- timed region: device-resident inputs
    clocks = ClockSampler(local)
    clocks.start()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    model.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        model.leapfrog(1, integ=integ)
    e1.record(stream)
    torch.cuda.synchronize()
    prof = model.profile_read()
    model.profile(False)
    if ws > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    if ws > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t.item())

    # ---- end to end: per step, momenta uploaded from pinned host memory, one leapfrog through the
    # C ABI, position / momentum / Hamiltonian read back into pinned host memory
    p_host = p0.cpu().pin_memory()
    p_dev = torch.empty_like(p0)
    q_host = torch.empty(C, d, dtype=torch.float64).pin_memory()
    pout_host = torch.empty_like(q_host).pin_memory()
    H_host = torch.empty(C, dtype=torch.float64).pin_memory()
    e_steps = max(1, min(args.steps, 3))
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e_steps):
        p_dev.copy_(p_host, non_blocking=True)
        model.leapfrog(1, qo, po, Ho, st, integ=integ, p_in=p_dev)
        q_host.copy_(qo, non_blocking=True)
        pout_host.copy_(po, non_blocking=True)
        H_host.copy_(Ho, non_blocking=True)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    te = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
    if ws > 1:
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
    e2e_s = float(te.item())
    status = st.cpu().numpy()

    if rank != 0:
        if ws > 1:
            dist.barrier()
            dist.destroy_process_group()
        return 0

    total_chains = C * ws
    value = total_chains * SUBSTEPS_PER_LEAPFROG * args.steps / (ms * 1e-3)
    e2e_value = total_chains * SUBSTEPS_PER_LEAPFROG * e_steps / e2e_s
    # roofline of the dominant kernel category (FP64 ALU bound), peak measured live on this GPU
    dom = max(prof, key=lambda k: prof[k][0])
    dom_ms, dom_flops, dom_launches = prof[dom]
    peak = rmhmc.fp64_peak_tflops(300)
    achieved = (dom_flops / dom_launches) / ((dom_ms / dom_launches) * 1e-3) / 1e12 if dom_launches else 0.0
    gpu_launches = int(sum(v[2] for v in prof.values()))
    # CPU baseline: the oracle on this host's cores, bounded sample
    cpu_baseline = None
    if not args.no_cpu_baseline:
        cb_value, cb_n, cb_s = oracle_leapfrogs(args.cpu_seconds)
        cpu_baseline = {"value": cb_value, "unit": UNIT, "cores": cpu_cores_used(), "kind": "oracle",
                        "sample": f"{cb_n} oracle leapfrog(s) of one chain of the workload in {cb_s:.1f} s "
                                  "(numpy/LAPACK FP64, full third-derivative tensor)"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD if C == N_CHAINS else WORKLOAD.replace(f"{N_CHAINS} chains", f"{C} chains"),
                   "N": N_INPUTS, "d": d, "chains_per_gpu": C,
                   "substeps_per_leapfrog": SUBSTEPS_PER_LEAPFROG,
                   "l2": "inputs larger than L2 (per-chain state ~16 MB, 64 chains ~1 GB > 126 MB)",
                   "parallelism": f"replicas x{ws}"},
        "leapfrogs_per_s": total_chains * args.steps / (ms * 1e-3),
        "roofline": {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak if peak else None,
                     "traffic": (JACOBI_DRAM_BYTES_PER_CHAIN * C) if dom == "jacobi_f64" else None,
                     "traffic_note": "bytes per k_jacobi launch, ncu capture at 8 chains scaled to the chain count",
                     "peak_note": "FP64 FMA throughput measured live on this GPU (rmhmc_fp64_peak)"},
        "profile_ms": {k: round(v[0], 3) for k, v in prof.items()},
        "profile_tflops": {k: (v[1] / (v[0] * 1e-3) / 1e12 if v[0] > 0 else 0.0) for k, v in prof.items()},
        "cpu_baseline": cpu_baseline,
        "e2e": {"value": e2e_value, "unit": UNIT,
                "h2d_bytes_per_step": int(p_host.numel() * 8),
                "d2h_bytes_per_step": int((q_host.numel() + pout_host.numel() + H_host.numel()) * 8)},
        "gpu_launches": gpu_launches,
        "chain_status_nonzero": int((status != 0).sum()),
        "valid": bool((status == 0).all()),
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="b300", choices=["b300", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--chains", type=int, default=N_CHAINS,
                    help="chains per GPU (the workload is 64; smaller values are for profiling)")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle timing leg")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_b300(args)


if __name__ == "__main__":
    sys.exit(main())
