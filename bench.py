#!/usr/bin/env python
"""Benchmark: SoftAbs-RMHMC generalized-leapfrog substeps per second on B300.

Workload (default): GP binary classification, N = 400 inputs x ~ U[-1, 1]^2, SE kernel with log
amplitude and log lengthscale (d = 402), 64 chains in one batch, soft-abs alpha = 1e6, eps = 0.001,
6 fixed-point iterations. A step is one Algorithm 1 iteration of every chain: a momentum draw
p ~ N(0, G), L = 10 generalized leapfrogs of 13 substeps each (6 implicit-momentum iterations, 6
implicit-position iterations, 1 explicit half-step), the Metropolis-Hastings test and the return of
rejected chains. value = chains x 10 x 13 x steps / seconds, whole job over all ranks. The
mixed-precision form is the headline; the plain FP64 path is timed after it on the same workload
(fewer iterations), with the error of one 10-leapfrog trajectory between the two.

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

# eps = 0.001 is the paper's step size for its simulated-data runs (Sec. 2.5); at N = 400 larger
# steps lose the chains within a few Algorithm 1 iterations (0.005: acceptance below 0.15 and most
# chains with a non-finite or non-positive-definite proposal after the first iteration; 0.002:
# failures from the tenth), while 0.001 keeps every proposal finite and accepted over the run.
N_INPUTS, N_CHAINS, EPS, N_FP, N_LEAPFROG = 400, 64, 0.001, 6, 10
# DRAM bytes per launch per chain of the dominant kernels, as ncu's dram__bytes_read.sum +
# dram__bytes_write.sum of single-kernel captures at 8 chains of this workload (traffic grows
# with the number of chains, so a 64-chain launch is scaled by 64 / 8). A kernel enters here only
# with counters taken from its current code.
DRAM_BYTES_PER_CHAIN = {}  # (k_jacobi_t<ElemDF>'s last capture predates its current criterion reads)
SUBSTEPS_PER_LEAPFROG = 2 * N_FP + 1
# The paper's settings for its simulated primal-model runs (Sec. 2.5): step size, and kappa of the
# map g(lambda) = sqrt(kappa^2 + lambda^2) (passed as alpha = 1 / kappa).
SOLIN_EPS, SOLIN_KAPPA = 0.001, 1.0
METRIC = "RMHMC leapfrog substeps/s"
UNIT = "substeps/s"
WORKLOAD = (f"GP classification N={N_INPUTS} (d={N_INPUTS + 2}), SE kernel, {N_CHAINS} chains batched, "
            f"plain FP64, Algorithm 1 iterations of L={N_LEAPFROG} generalized leapfrogs (momentum "
            f"refresh + Metropolis-Hastings), alpha=1e6, eps={EPS}, n_fp={N_FP}")


MIXED_NOTE = ("mixed precision: Jacobi rotations in double-float (FP32 pairs, ~48-bit); the K^-1 algebra "
              "(K^-1, K^-1 dK and products) and the d x d products Psi^T H Psi, Psi C Psi^T on the tcgen05 "
              "tensor cores by exact bf16 slicing (9 / 7 slices = 63 / 49 bits, FP32 accumulation in "
              "TMEM, combined in FP64); Cholesky, L^-1, log|G|, H and the Hamiltonian in FP64")
DTYPE_MIXED = "f64 + f32x2 (double-float) + bf16 slices on tensor cores (FP64-accurate GEMM)"


def aux_precision(args):
    """Precision of the auxiliary workloads: mixed unless --precision fp64."""
    return "fp64" if args.precision == "fp64" else "mixed"


def dtype_of(prec):
    return "f64" if prec == "fp64" else DTYPE_MIXED


def arm_config(C, ws, head):
    """The workload description both arms print (the GPU arm and the oracle reference arm)."""
    workload = WORKLOAD if C == N_CHAINS else WORKLOAD.replace(f"{N_CHAINS} chains", f"{C} chains")
    names = {"fp64": "plain FP64", "mixed": "mixed precision", "oracle": "plain FP64 oracle (CPU)"}
    workload = workload.replace("plain FP64", names[head])
    precision = {"fp64": "plain FP64", "mixed": MIXED_NOTE,
                 "oracle": "plain FP64 oracle: numpy/LAPACK on the host cores, one chain"}[head]
    return {"workload": workload, "N": N_INPUTS, "d": N_INPUTS + 2, "chains_per_gpu": C,
            "precision": precision,
            "step": (f"one Algorithm 1 iteration of every chain: L={N_LEAPFROG} leapfrogs x "
                     f"{SUBSTEPS_PER_LEAPFROG} substeps" if head != "oracle" else
                     "one leapfrog of one chain's Algorithm 1 run (bounded sample)"),
            "substeps_per_leapfrog": SUBSTEPS_PER_LEAPFROG, "n_leapfrog": N_LEAPFROG,
            "l2": "inputs larger than L2 (per-chain state ~16 MB, 64 chains ~1 GB > 126 MB)",
            "parallelism": f"replicas x{ws}"}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, ws, device):
    """The largest of the ranks' values of x, returned on every rank (x itself when ws == 1): the
    job's time is its slowest rank's."""
    if ws == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank, ws, steps, seconds):
    """Whole-job throughput: the units every rank processed in `steps` steps over the job's time."""
    return units_per_rank * ws * steps / seconds


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


class OracleChain:
    """One chain of the benchmark workload run by the plain FP64 oracle through Algorithm 1, one
    leapfrog at a time: every N_LEAPFROG leapfrogs the Metropolis-Hastings test of the trajectory
    and a fresh momentum p = G^{1/2} z (the oracle's Philox draws, key (seed, 0)). The model and the
    first geometry are built in the constructor, outside any timed region. A trajectory that leaves
    the region where K is positive definite is a rejected proposal (as in the oracle's sampler)."""

    def __init__(self, seed=0, n_inputs=None):
        from oracle.geometry import Geometry
        from oracle.model import from_problem
        self.model = from_problem(wl.gp_classification(n_inputs or N_INPUTS, seed=0))
        self.seed, self.it = seed, 0
        self.q = np.zeros(self.model.d)
        self.geo = Geometry(self.model, self.q, 1.0)
        self.accepted = self.rejected = 0
        self._refresh()

    def _refresh(self):
        from oracle.philox import normals
        self.p = self.geo.sqrtG_z(normals(self.seed, 0, self.it, self.model.d))
        self.H0 = self.geo.hamiltonian(self.p)
        self.traj = (self.q, self.p, self.geo)
        self.k = 0

    def _finish(self, H1, new):
        from oracle.philox import mh_uniform
        with np.errstate(divide="ignore"):
            logr = np.log(mh_uniform(self.seed, 0, self.it))
        if new is not None and np.isfinite(H1) and logr < self.H0 - H1:
            self.q, _, self.geo = new
            self.accepted += 1
        else:
            self.rejected += 1
        self.it += 1
        self._refresh()

    def leapfrog(self):
        """One generalized leapfrog (and, after the trajectory's last, the MH test and momentum
        refresh). Returns False when the trajectory failed numerically (proposal rejected; the
        leapfrog is not counted)."""
        from oracle.integrator import leapfrog
        q, p, geo = self.traj
        try:
            with np.errstate(all="ignore"):
                self.traj = leapfrog(self.model, q, p, EPS, N_FP, geo=geo)
        except np.linalg.LinAlgError:
            self._finish(np.inf, None)
            return False
        self.k += 1
        if self.k == N_LEAPFROG:
            self._finish(self.traj[2].hamiltonian(self.traj[1]), self.traj)
        return True


def oracle_leapfrogs(seconds, max_leapfrogs=None, seed=0):
    """Time the plain FP64 oracle on one chain of the benchmark workload (Algorithm 1, continued
    leapfrog by leapfrog) for about `seconds` (at least one leapfrog); the set-up (model, first
    geometry) is outside the timed region. Returns (substeps/s, leapfrogs done, seconds)."""
    chain = OracleChain(seed)
    n, t0 = 0, time.perf_counter()
    while True:
        n += 1 if chain.leapfrog() else 0
        el = time.perf_counter() - t0
        if (el >= seconds and n > 0) or (max_leapfrogs and n >= max_leapfrogs):
            break
    return SUBSTEPS_PER_LEAPFROG * n / el, n, el


# Peak resident memory of one oracle process on the benchmark workload (d = 402: the full d^3
# third-derivative tensor and its temporaries; 1.58 GB measured), with margin.
ORACLE_PROCESS_BYTES = 2.0e9

# Environment variables that fix the thread count of the BLAS libraries numpy may be linked with;
# a `spawn` child reads them when it first imports numpy.
BLAS_THREAD_VARS = ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS",
                    "VECLIB_MAXIMUM_THREADS", "NUMEXPR_NUM_THREADS")


def _oracle_one_core(job):
    """Worker of oracle_per_core: one chain with single-threaded BLAS. The parent sets
    BLAS_THREAD_VARS to 1 before it spawns the pool; threadpoolctl, where installed, also limits
    any BLAS pool already running."""
    seconds, seed = job
    try:
        from threadpoolctl import threadpool_limits
    except ImportError:
        return oracle_leapfrogs(seconds, seed=seed)
    with threadpool_limits(limits=1):
        return oracle_leapfrogs(seconds, seed=seed)


# At most this many oracle processes at once, whatever the host reports.
ORACLE_MAX_PROCS = 32


def host_cores():
    """Cores this process may run on: its CPU affinity set, bounded by the BLAS thread count the
    single-chain leg uses (both follow the container's cpuset, unlike os.cpu_count())."""
    try:
        n = len(os.sched_getaffinity(0))
    except AttributeError:
        n = os.cpu_count() or 1
    return max(1, min(n, cpu_cores_used()))


# cgroup memory limit and usage files (v2, then v1)
CGROUP_MEMORY_FILES = (("/sys/fs/cgroup/memory.max", "/sys/fs/cgroup/memory.current"),
                       ("/sys/fs/cgroup/memory/memory.limit_in_bytes",
                        "/sys/fs/cgroup/memory/memory.usage_in_bytes"))


def host_free_bytes(cgroup_files=CGROUP_MEMORY_FILES):
    """Host memory this process may still use: the smaller of what the OS reports available and the
    room left under each cgroup memory limit found, or None if neither is known."""
    free = None
    try:
        import psutil
        free = psutil.virtual_memory().available
    except ImportError:
        pass
    for lim_path, use_path in cgroup_files:
        try:
            with open(lim_path) as f:
                lim = f.read().strip()
            if lim == "max":
                continue
            with open(use_path) as f:
                room = int(lim) - int(f.read().strip())
        except (OSError, ValueError):
            continue
        free = room if free is None else min(free, room)
    return free


def oracle_per_core(seconds, max_procs=None):
    """The many-chain CPU baseline: one chain per host core, each process with single-threaded
    BLAS, all running at once for about `seconds`. The pool is started with `spawn` (never forked
    from a process that holds a CUDA context); its size is the usable core count, bounded by the
    host memory this process may still use (ORACLE_PROCESS_BYTES per process) and by
    ORACLE_MAX_PROCS. Returns (aggregate substeps/s, processes, total leapfrogs, longest worker
    time)."""
    import multiprocessing as mp
    n = min(host_cores(), ORACLE_MAX_PROCS)
    free = host_free_bytes()
    if free is not None:
        n = min(n, int(0.8 * free // ORACLE_PROCESS_BYTES))
    if max_procs:
        n = min(n, max_procs)
    n = max(1, n)
    saved = {k: os.environ.get(k) for k in BLAS_THREAD_VARS}
    os.environ.update({k: "1" for k in BLAS_THREAD_VARS})
    try:
        with mp.get_context("spawn").Pool(n) as pool:
            res = pool.map(_oracle_one_core, [(seconds, 1 + i) for i in range(n)])
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return sum(r[0] for r in res), n, sum(r[1] for r in res), max(r[2] for r in res)


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    # one chain of the workload, set up outside the timed region; each warm-up and timed step is a
    # bounded sample: one leapfrog of that chain's Algorithm 1 run (momentum refresh and the
    # Metropolis-Hastings test after every N_LEAPFROG-th), the trajectory continued across steps
    chain = OracleChain(seed=0)
    for _ in range(args.warmup):
        chain.leapfrog()
    t0, done = time.perf_counter(), 0
    for _ in range(args.steps):
        done += 1 if chain.leapfrog() else 0
    el = time.perf_counter() - t0
    value = SUBSTEPS_PER_LEAPFROG * done / el
    cores = cpu_cores_used()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": arm_config(args.chains, args.gpus, "oracle"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"one chain of the workload, one leapfrog of its Algorithm 1 run per step "
                                       f"({done} of {args.steps} completed; numpy/LAPACK FP64, full "
                                       "third-derivative tensor; set-up outside the timed region)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _time_iterations(model, integ, steps, seed, stream, local, ws, dev):
    """K timed Algorithm 1 iterations of every chain (device-resident state) in one rmhmc_sample
    call, CUDA events on the model's stream, library profiling off, clocks sampled meanwhile.
    Returns (ms as the max over ranks, accept (K x C), chain status (C), clocks)."""
    import torch
    import torch.distributed as dist
    C = model.n_chains
    acc = torch.zeros(steps, C, dtype=torch.int32, device=dev)
    cs = torch.zeros(C, dtype=torch.int32, device=dev)
    clocks = ClockSampler(local)
    clocks.start()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")  # (lets a profiler select the timed region: ncu --nvtx-include timed/)
    e0.record(stream)
    model.sample(steps, 0, seed, accept=acc, chain_status=cs, integ=integ)
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clk = clocks.stop()
    return max_over_ranks(e0.elapsed_time(e1), ws, dev), acc.cpu().numpy(), cs.cpu().numpy(), clk


def _profile_iteration(model, integ, seed):
    """One more Algorithm 1 iteration, outside the timed region, with the library's per-launch-site
    events on (per-category time, counted FLOPs) and, where torch's profiler (CUPTI) works, the
    kernels the device actually ran. Returns (category profile, {kernel: launches} or None)."""
    import torch
    kernels = None
    model.profile(True)
    try:
        from torch.profiler import ProfilerActivity, profile
        with profile(activities=[ProfilerActivity.CUDA]) as tp:
            model.sample(1, 0, seed, integ=integ)
            torch.cuda.synchronize()
        kernels = {}
        for ev in tp.events():
            if getattr(ev, "device_type", None) is not None and "CUDA" in str(ev.device_type):
                name = ev.name.split("(")[0].split("<")[0].replace("void ", "").strip()
                if name.startswith("Memcpy") or name.startswith("Memset") or name.startswith("["):
                    continue
                kernels[name] = kernels.get(name, 0) + 1
        if not kernels:
            kernels = None
    except Exception:
        model.sample(1, 0, seed, integ=integ)
        kernels = None
    prof = model.profile_read()
    model.profile(False)
    return prof, kernels


def _measured_bf16_peak():
    """(sustained, burst) dense bf16 TFLOP/s of the B300s (cuBLAS), from MEASURED_PEAKS.json."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            mp = json.load(f)
        return float(mp["bf16_tflops_sustained"]), float(mp["bf16_tflops"])
    except (OSError, KeyError, ValueError):
        return 1400.0, 1800.0  # the recipe's fallback figures


def _tensor_roofline(prof):
    """The tensor-core GEMM category against the measured bf16 peak: executed bf16 FLOPs (all slice
    products of all 128 x 64 tiles) / CUDA-event time, inside the step, so the sustained figure."""
    if "gemm_tc" not in prof or not prof["gemm_tc"][2]:
        return None
    ms, flops, launches = prof["gemm_tc"]
    sus, burst = _measured_bf16_peak()
    achieved = flops / (ms * 1e-3) / 1e12
    return {"bound": "tensor", "kernel": "gemm_tc (k_tc_split + k_gemm_tc)", "achieved": achieved, "peak": sus,
            "unit": "TFLOP/s", "frac": achieved / sus, "traffic": None,
            "peak_note": f"cuBLAS bf16 measured, sustained ({sus}; burst {burst}), MEASURED_PEAKS.json",
            "achieved_note": "bf16 tensor FLOPs executed (slice products incl. tile padding); time includes "
                             "the slicing kernels"}


# The pipe whose measured peak bounds each timed category's counted FLOPs: FP64 FMA
# (rmhmc_fp64_peak), the double-float multiply-add (rmhmc_df_peak), the bf16 tensor rate.
CATEGORY_PIPE = {"gemm_f64": "fp64", "jacobi_f64": "fp64", "cholesky": "fp64", "trinv": "fp64",
                 "jacobi_df": "df", "gemm_tc": "bf16", "prerotation": "df"}


def category_rooflines(prof, peaks, mixed=False):
    """Per timed category ({name: (ms, flops, launches)}): its share of the step and, where the
    library counts its FLOPs, the achieved TFLOP/s against the measured peak of its pipe; and the
    step's flop-weighted total: the time every counted category would take at its pipe's peak over
    the measured time (`frac`: of all categories, whose O(N^2) / O(d^2) memory-bound phases count
    no FLOPs and only add time; `frac_counted`: of the counted ones). In the mixed form the
    Cholesky and L^-1 count FP64-equivalent FLOPs of which most run on the tensor cores: they get
    that rate but no single pipe."""
    total = sum(v[0] for v in prof.values())
    cats, ideal, counted = {}, 0.0, 0.0
    for name, (ms, flops, launches) in sorted(prof.items(), key=lambda kv: -kv[1][0]):
        if not launches:
            continue
        e = {"ms": round(ms, 3), "share": ms / total if total else None}
        pipe = CATEGORY_PIPE.get(name)
        if mixed and name in ("cholesky", "trinv"):
            pipe = None
            if flops > 0 and ms > 0:
                e["achieved_fp64_equivalent"] = flops / (ms * 1e-3) / 1e12
        if pipe and flops > 0 and ms > 0 and peaks.get(pipe):
            achieved = flops / (ms * 1e-3) / 1e12
            e.update(pipe=pipe, achieved=achieved, peak=peaks[pipe], frac=achieved / peaks[pipe])
            ideal += flops / (peaks[pipe] * 1e12) * 1e3
            counted += ms
        cats[name] = e
    return {"unit": "TFLOP/s", "categories": cats,
            "step": {"ideal_ms": ideal, "measured_ms": total, "frac": ideal / total if total else None,
                     "frac_counted": ideal / counted if counted else None}}


def _measured_pipe_peaks(rmhmc):
    """{pipe: TFLOP/s} measured on this GPU (FP64 and double-float live, bf16 from the measured
    sustained cuBLAS figure); {} if a probe fails."""
    try:
        return {"fp64": rmhmc.fp64_peak_tflops(300), "df": rmhmc.df_peak_tflops(300),
                "bf16": _measured_bf16_peak()[0]}
    except Exception:
        return {}


def _roofline(rmhmc, prof, C):
    """Roofline of the dominant kernel category (ALU bound; peaks measured live on this GPU)."""
    dom = max(prof, key=lambda k: prof[k][0])
    dom_ms, dom_flops, dom_launches = prof[dom]
    if dom == "gemm_tc":
        return _tensor_roofline(prof)
    if dom in ("jacobi_df", "prerotation"):
        # the double-float multiply-add (Dot2 step: 12 FP32 instructions) measured on this GPU
        peak = rmhmc.df_peak_tflops(300)
        fp32 = rmhmc.fp32_peak_tflops(300)
        peak_note = (f"double-float multiply-add throughput measured live (rmhmc_df_peak, Dot2 chains); "
                     f"for reference the FP32 FMA rate is {fp32:.1f} TFLOP/s, /12 = {fp32 / 12:.2f}")
    else:
        peak = rmhmc.fp64_peak_tflops(300)
        peak_note = "FP64 FMA throughput measured live on this GPU (rmhmc_fp64_peak)"
    achieved = (dom_flops / dom_launches) / ((dom_ms / dom_launches) * 1e-3) / 1e12 if dom_launches else 0.0
    out = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
           "frac": achieved / peak if peak else None, "traffic": None, "peak_note": peak_note}
    if dom.startswith("jacobi"):
        out["achieved_note"] = ("executed work: 16x16x16 rotation-tile products x 8192 flops (skipped identity "
                                "tiles not counted) + inner rotation rounds x 1952 flops; rotation angles, "
                                "stopping tests and conversions not counted")
    elif dom == "prerotation":
        out["achieved_note"] = ("double-float multiply-adds of the first- and second-order sparse products "
                                "(2 flops each, 24 dp per pre-rotated pair); the FP32 higher-order products, "
                                "the coupling test and the element-wise passes not counted")
    if dom in DRAM_BYTES_PER_CHAIN:
        out["traffic"] = DRAM_BYTES_PER_CHAIN[dom] * C
        out["traffic_note"] = "bytes per launch, ncu capture at 8 chains scaled to the chain count"
    return out


def _trajectory_error(rmhmc, prob, q0, seed=7):
    """One 10-leapfrog trajectory of the same chains from the same (q, p) in both precisions, p
    drawn from N(0, G(q)) with G of the FP64 geometry: max over chains of
    ||x_mixed - x_fp64|| / ||x_fp64|| for x = q and p."""
    import torch
    C, d = q0.shape
    f64 = dict(dtype=torch.float64, device=q0.device)
    m = rmhmc.Model(prob, C)
    m.set_state(q0, integ=rmhmc.Integrator(eps=EPS, n_fp=N_FP, n_leapfrog=1, precision="fp64"))
    G = torch.empty(C, d, d, **f64)
    m.geometry(G=G)
    torch.cuda.synchronize()
    m.close()
    gen = torch.Generator(device=q0.device).manual_seed(seed)
    z = torch.randn(C, d, 1, generator=gen, **f64)
    p0 = (torch.linalg.cholesky(G) @ z).squeeze(-1).contiguous()
    out = {}
    for prec in ("fp64", "mixed"):
        integ = rmhmc.Integrator(eps=EPS, n_fp=N_FP, n_leapfrog=1, precision=prec)
        m = rmhmc.Model(prob, C)
        m.set_state(q0, p0, integ=integ)
        m.leapfrog(10, integ=integ)
        q, p = torch.empty_like(q0), torch.empty_like(q0)
        st = torch.empty(C, dtype=torch.int32, device=q0.device)
        m.leapfrog(0, q, p, status_out=st, integ=integ)
        torch.cuda.synchronize()
        out[prec] = (q.cpu().numpy(), p.cpu().numpy(), st.cpu().numpy())
        m.close()
    ok = (out["fp64"][2] == 0) & (out["mixed"][2] == 0)
    rel = {}
    for k, name in enumerate(("q", "p")):
        a, b = out["fp64"][k][ok], out["mixed"][k][ok]
        rel[name] = float(np.max(np.linalg.norm(b - a, axis=1) / np.linalg.norm(a, axis=1))) if ok.any() else None
    return {"chains": int(C), "chains_finite": int(ok.sum()), "leapfrogs": 10,
            "max_rel_q": rel["q"], "max_rel_p": rel["p"]}


def _e2e(rmhmc, prob, C, integ, steps, seed, stream, dev, ws, jacobi=None):
    """End to end through the public API, as a user runs the sampler from host data: the model is
    created from the host arrays (X, y copied in), the chains' start q0 is copied from pinned host
    memory, and every step is one Algorithm 1 iteration (rmhmc_sample) whose draws (q, log P,
    accept, chain status) are copied back to pinned host memory. Returns (seconds as the max over
    ranks, h2d bytes per step, d2h bytes per step, chain status)."""
    import torch
    import torch.distributed as dist
    d = wl.dims(prob)[2]
    q0_host = torch.zeros(C, d, dtype=torch.float64).pin_memory()
    qs_host = torch.empty(1, C, d, dtype=torch.float64).pin_memory()
    lp_host = torch.empty(1, C, dtype=torch.float64).pin_memory()
    acc_host = torch.empty(1, C, dtype=torch.int32).pin_memory()
    cs_host = torch.empty(C, dtype=torch.int32).pin_memory()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    model = rmhmc.Model(prob, C, stream=stream)
    if jacobi:  # the autotuned settings of the device-timed arm
        model.set_jacobi(jacobi["cluster"], jacobi["schedule"])
        model.set_gemm_tile(jacobi["gemm_tile"])
        model.set_prerotation(jacobi["prerotation"])
    q0 = torch.empty(C, d, dtype=torch.float64, device=dev)
    q0.copy_(q0_host, non_blocking=True)
    model.set_state(q0, integ=integ)
    qs = torch.empty(1, C, d, dtype=torch.float64, device=dev)
    lp = torch.empty(1, C, dtype=torch.float64, device=dev)
    acc = torch.empty(1, C, dtype=torch.int32, device=dev)
    cs = torch.empty(C, dtype=torch.int32, device=dev)
    status = np.zeros(C, dtype=np.int32)
    for _ in range(steps):
        model.sample(1, 0, seed, qs, lp, acc, chain_status=cs, integ=integ)
        qs_host.copy_(qs, non_blocking=True)
        lp_host.copy_(lp, non_blocking=True)
        acc_host.copy_(acc, non_blocking=True)
        cs_host.copy_(cs, non_blocking=True)
        torch.cuda.current_stream().synchronize()
        status |= cs_host.numpy()
    torch.cuda.synchronize()
    el = max_over_ranks(time.perf_counter() - t0, ws, dev)
    model.close()
    X = np.asarray(prob["X"])
    h2d = (X.size + np.asarray(prob["y"]).size + q0_host.numel()) * 8 / steps
    d2h = (qs_host.numel() + lp_host.numel()) * 8 + (acc_host.numel() + cs_host.numel()) * 4
    return el, int(h2d), int(d2h), status


def _run_arm(rmhmc, prob, C, prec, warmup, steps, seed, stream, local, ws, dev):
    """Warm-up and timed Algorithm 1 iterations of one precision, then one profiled iteration."""
    import torch
    model = rmhmc.Model(prob, C, stream=stream)
    integ = rmhmc.Integrator(eps=EPS, n_fp=N_FP, n_leapfrog=N_LEAPFROG, precision=prec)
    model.set_state(torch.zeros(C, model.d, dtype=torch.float64, device=dev), integ=integ)
    # the library's autotuner picks the Jacobi cluster size and rotation order for this model by
    # timing one leapfrog of each combination (untimed set-up; the state is restored)
    jacobi = dict(zip(("cluster", "schedule", "gemm_tile", "prerotation"), model.autotune(integ)))
    warm_cs = torch.zeros(C, dtype=torch.int32, device=dev)
    model.sample(warmup, 0, seed, chain_status=warm_cs, integ=integ)
    ms, acc, cs, clk = _time_iterations(model, integ, steps, seed, stream, local, ws, dev)
    prof, kernels = _profile_iteration(model, integ, seed)
    q = torch.empty(C, model.d, dtype=torch.float64, device=dev)
    model.leapfrog(0, q, integ=integ)
    torch.cuda.synchronize()
    model.close()
    return {"ms": ms, "acc": acc, "status": cs, "warm_status": warm_cs.cpu().numpy(), "clk": clk,
            "prof": prof, "kernels": kernels, "q": q, "jacobi": jacobi}


def _status_summary(status):
    """Chains whose proposals failed numerically during the timed iterations, by failure kind."""
    bits = (("not_pd", 1), ("jacobi_not_converged", 2), ("non_finite", 4), ("wait_timeout", 8))
    return {"chains_with_failed_proposal": int((status != 0).sum()),
            **{name: int(((status & bit) != 0).sum()) for name, bit in bits}}


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
    seed = 1234 + rank
    precisions = ["mixed", "fp64"] if args.precision == "both" else [args.precision]
    runs = {}
    for prec in precisions:
        steps = args.steps if prec == precisions[0] else max(1, min(args.steps, args.fp64_steps))
        warm = args.warmup if prec == precisions[0] else max(1, min(args.warmup, 2))
        runs[prec] = _run_arm(rmhmc, prob, C, prec, warm, steps, seed, stream, local, ws, dev)
        runs[prec]["steps"] = steps
    head = precisions[0]
    h = runs[head]
    ms = h["ms"]
    integ = rmhmc.Integrator(eps=EPS, n_fp=N_FP, n_leapfrog=N_LEAPFROG, precision=head)
    e_steps = max(1, min(args.steps, args.e2e_steps))
    e2e_s, h2d, d2h, e2e_status = _e2e(rmhmc, prob, C, integ, e_steps, seed + 1, stream, dev, ws, jacobi=h["jacobi"])

    if rank != 0:
        if ws > 1:
            dist.barrier()
            dist.destroy_process_group()
        return 0

    units = C * N_LEAPFROG * SUBSTEPS_PER_LEAPFROG  # substeps per step on one rank
    value = job_value(units, ws, args.steps, ms * 1e-3)
    e2e_value = job_value(units, ws, e_steps, e2e_s)
    roof = _roofline(rmhmc, h["prof"], C)
    pipe_peaks = _measured_pipe_peaks(rmhmc)
    per_iter_launches = (sum(h["kernels"].values()) if h["kernels"]
                         else int(sum(v[2] for v in h["prof"].values())))
    traj = None
    if args.precision == "both":
        k = min(4, C)
        traj = _trajectory_error(rmhmc, prob, runs["fp64"]["q"][:k].clone())
    # CPU baselines: the oracle on this host's cores, bounded samples (single-GPU runs only: with
    # N > 1 ranks the host's cores are shared with the other ranks' processes)
    cpu_baseline = cpu_baseline_per_core = None
    if not args.no_cpu_baseline and ws == 1:
        cb_value, cb_n, cb_s = oracle_leapfrogs(args.cpu_seconds)
        cpu_baseline = {"value": cb_value, "unit": UNIT, "cores": cpu_cores_used(), "kind": "oracle",
                        "sample": f"{cb_n} oracle leapfrog(s) of one chain's Algorithm 1 run in {cb_s:.1f} s "
                                  "(numpy/LAPACK FP64, full third-derivative tensor; set-up untimed)"}
        pc_value, pc_n, pc_l, pc_s = oracle_per_core(args.cpu_seconds)
        cpu_baseline_per_core = {"value": pc_value, "unit": UNIT, "cores": pc_n, "kind": "oracle",
                                 "sample": f"{pc_n} processes at once, one chain each with single-threaded "
                                           f"BLAS, {pc_l} oracle leapfrogs in at most {pc_s:.1f} s; value = "
                                           "sum of the processes' rates"}

    def prof_summary(prof):
        return ({k: round(v[0], 3) for k, v in prof.items() if v[2]},
                {k: (v[1] / (v[0] * 1e-3) / 1e12 if v[0] > 0 else 0.0) for k, v in prof.items() if v[2]})

    pms, ptf = prof_summary(h["prof"])
    failed = _status_summary(h["status"])
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if head == "fp64" else DTYPE_MIXED,
        "data": "synthetic",
        "config": arm_config(C, ws, head),
        "leapfrogs_per_s": C * ws * N_LEAPFROG * args.steps / (ms * 1e-3),
        "acceptance": float(h["acc"].mean()),
        "jacobi_autotuned": h["jacobi"],
        "timed_region_failures": failed,
        "valid": failed["chains_with_failed_proposal"] == 0,
        "roofline": roof,
        "roofline_tensor_gemm": _tensor_roofline(h["prof"]),
        "profile_note": "per-category times and FLOPs from one further profiled iteration (library "
                        "events around each launch site), outside the timed region",
        "profile_ms": pms, "profile_tflops": ptf,
        "roofline_by_category": category_rooflines(h["prof"], pipe_peaks, mixed=head == "mixed"),
        "cpu_baseline": cpu_baseline,
        "cpu_baseline_per_core": cpu_baseline_per_core,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "steps": e_steps,
                "note": "model created from host X, y and q0 (pinned) inside the timed region, then one "
                        "rmhmc_sample iteration per step with its draws copied to pinned host memory",
                "chains_with_failed_proposal": int((e2e_status != 0).sum())},
        "gpu_launches": per_iter_launches * args.steps,
        "gpu_launches_note": ("kernels per iteration counted by torch's CUDA profiler (CUPTI) in the "
                              "profiled iteration, times the timed iterations" if h["kernels"] else
                              "launch sites counted by the library's profiler, times the timed iterations"),
        "clocks": h["clk"],
    }
    if "fp64" in runs and head != "fp64":
        r = runs["fp64"]
        f_ms, f_tf = prof_summary(r["prof"])
        f_value = job_value(units, ws, r["steps"], r["ms"] * 1e-3)
        line["fp64"] = {"value": f_value, "steps": r["steps"], "ms_per_step": r["ms"] / r["steps"],
                        "acceptance": float(r["acc"].mean()), "roofline": _roofline(rmhmc, r["prof"], C),
                        "jacobi_autotuned": r["jacobi"],
                        "profile_ms": f_ms, "profile_tflops": f_tf,
                        "roofline_by_category": category_rooflines(r["prof"], pipe_peaks),
                        "timed_region_failures": _status_summary(r["status"]), "clocks": r["clk"]}
        line["speedup_vs_fp64"] = value / f_value
        line["trajectory_error_vs_fp64"] = traj
    print(json.dumps(line), flush=True)
    if not line["valid"]:
        print(f"bench: {failed['chains_with_failed_proposal']} chain(s) had a numerically failed proposal "
              "in the timed region; the value is not a valid measurement", file=sys.stderr)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def _clock_and_time(fn, local):
    import torch
    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    fn()
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    return el, clocks.stop()


def run_propensity(args):
    """Additive 3-kernel propensity model, N = 500 (d = 1506), 32 chains."""
    import torch
    from paper_2511_06407_b300 import build, rmhmc
    build.build()
    prob = wl.propensity(500, seed=0, n_kernels=3)
    C = 32
    model = rmhmc.Model(prob, C)
    prec = aux_precision(args)
    integ = rmhmc.Integrator(eps=args.eps or EPS, n_fp=N_FP, n_leapfrog=1, precision=prec)
    model.set_state(torch.zeros(C, model.d, dtype=torch.float64, device="cuda"), integ=integ)
    tuned = model.autotune(integ)
    model.sample(1, 0, 99, integ=integ)
    model.leapfrog(max(args.warmup - 1, 0), integ=integ)
    st = torch.empty(C, dtype=torch.int32, device="cuda")
    el, clk = _clock_and_time(lambda: model.leapfrog(args.steps, status_out=st, integ=integ), 0)
    status = st.cpu().numpy()
    model.profile(True)  # one more leapfrog with the per-launch events, outside the timed region
    model.leapfrog(1, integ=integ)
    prof = model.profile_read()
    model.profile(False)
    value = C * SUBSTEPS_PER_LEAPFROG * args.steps / el
    print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
                      "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
                      "dtype": dtype_of(prec), "data": "synthetic",
                      "config": {"workload": "propensity model N=500, SE+linear+overlap (d=1506), 32 chains, "
                                             f"{prec}, eps={integ.eps}", "d": model.d, "chains": C,
                                 "autotuned_cluster_schedule_tile": tuned},
                      "profile_ms": {k: round(v[0], 1) for k, v in prof.items()},
                      "profile_tflops": {k: (v[1] / (v[0] * 1e-3) / 1e12 if v[0] > 0 else 0.0) for k, v in prof.items()},
                      "chain_status_nonzero": int((status != 0).sum()), "clocks": clk}), flush=True)
    return 0


def run_ess(args):
    """Effective samples per second of Algorithm 1 (L = 10, n_fp = 6), plain FP64 and mixed
    precision, independent seeds, plus the matched-error check: posterior means and variances of
    (log P, hyperparameters, mean F) of the mixed run within 3 Monte-Carlo standard errors of the
    FP64 run's. --ess-model dual: the GP-classification problem (N = --ess-n, SoftAbs coth);
    primal (default): the simulated data of Sec. 2.5 with D = --ess-d Gaussian kernels
    (d = 30 D + 4, g = sqrt(1 + l^2)), the paper's own experimental model."""
    import torch
    from paper_2511_06407_b300 import build, rmhmc
    from paper_2511_06407_b300 import diagnostics as dg
    build.build()
    C = args.chains
    if args.ess_model == "dual":
        N = args.ess_n
        prob = wl.gp_classification(N, seed=0)
        eps = args.eps or (EPS if N == N_INPUTS else 0.01)
        geom = {}
        names = ["log P", "log c", "log l", "mean f"]
        label = f"GP classification N={N} (d={N + 2})"
        hyper = slice(-2, None)
    else:
        N = 500
        prob = wl.solin_logistic(args.ess_d, N=N, seed=0)
        eps = args.eps or 0.05
        geom = dict(g_kind="sqrt", alpha=1.0)
        names = ["log P", "log c_g", "log s_g", "b"]
        label = f"primal model of Sec. 2.5, D={args.ess_d} (d={wl.dims(prob)[2]}), N=500, g=sqrt(1+l^2)"
        hyper = slice(-3, -1)
    runs = {}
    for k, prec in enumerate(("fp64", "mixed")):
        integ = rmhmc.Integrator(eps=eps, n_leapfrog=10, n_fp=N_FP, precision=prec, **geom)
        model = rmhmc.Model(prob, C)
        d = model.d
        model.set_state(torch.zeros(C, d, dtype=torch.float64, device="cuda"), integ=integ)
        cs = torch.zeros(C, dtype=torch.int32, device="cuda")
        seed = 11 + (0 if args.ess_same_seed else 1000 * k)
        model.sample(0, args.burn, seed, chain_status=cs, integ=integ)
        qs = torch.empty(args.iters, C, d, dtype=torch.float64, device="cuda")
        lp = torch.empty(args.iters, C, dtype=torch.float64, device="cuda")
        acc = torch.empty(args.iters, C, dtype=torch.int32, device="cuda")
        cs2 = torch.zeros(C, dtype=torch.int32, device="cuda")
        el, clk = _clock_and_time(lambda: model.sample(args.iters, 0, seed, qs, lp, acc, chain_status=cs2,
                                                       integ=integ), 0)
        Q, LP = qs.cpu().numpy(), lp.cpu().numpy()
        # the fourth quantity: the mean latent value (dual) or the bias b (primal)
        last = Q[:, :, :N].mean(axis=2, keepdims=True) if args.ess_model == "dual" else Q[:, :, -4:-3]
        draws = np.concatenate([LP[:, :, None], Q[:, :, hyper], last], axis=2)
        summ = dg.summary(draws, names)
        x = draws.transpose(1, 0, 2)  # chains x iterations x quantities
        mean = x.reshape(-1, 4).mean(axis=0)
        var = x.reshape(-1, 4).var(axis=0)
        se_mean = np.array([dg.mcse_mean(x[:, :, j]) for j in range(4)])
        se_var = np.array([dg.mcse_mean((x[:, :, j] - mean[j]) ** 2) for j in range(4)])
        runs[prec] = {"seconds": el, "min_ess": summ["min_ess"], "ess_per_s": summ["min_ess"] / el,
                      "_draws": draws, "_accept": acc.cpu().numpy(),
                      "max_rhat": summ["max_rhat"], "acceptance": float(acc.cpu().numpy().mean()),
                      "substeps_per_s": C * args.iters * 10 * SUBSTEPS_PER_LEAPFROG / el,
                      "chain_status_nonzero": int(((cs | cs2).cpu().numpy() != 0).sum()),
                      "chain_status_bits": {name: int((((cs | cs2).cpu().numpy() & bit) != 0).sum())
                                            for name, bit in (("not_pd", 1), ("jacobi_not_converged", 2),
                                                              ("non_finite", 4))},
                      "ess": {r["name"]: round(min(r["ess_bulk"], r["ess_tail"]), 1) for r in summ["rows"]},
                      "mean": mean, "var": var, "se_mean": se_mean, "se_var": se_var, "clocks": clk}
        model.close()
    a, b = runs["fp64"], runs["mixed"]
    paths = None
    if args.ess_same_seed:
        # the same Philox draws in both precisions: the mixed chains follow the FP64 chains
        da, db = a["_draws"], b["_draws"]
        paths = {"same_decisions_fraction": float((a["_accept"] == b["_accept"]).mean()),
                 "max_rel_diff_per_quantity": [float(np.max(np.abs(db[..., j] - da[..., j])) /
                                                     max(float(np.max(np.abs(da[..., j]))), 1e-300))
                                               for j in range(da.shape[2])]}
    oracle = None
    if args.ess_model == "dual" and N == N_INPUTS and eps == EPS and not args.no_cpu_baseline:
        # the oracle runs the same dynamics (FP64, same L, n_fp and step): its ESS per substep is
        # the FP64 run's, so its ESS/s on this host's cores is that times its measured substeps/s
        pc_value, pc_n, pc_l, pc_s = oracle_per_core(args.cpu_seconds)
        ess_per_substep = a["min_ess"] / (C * args.iters * 10 * SUBSTEPS_PER_LEAPFROG)
        oracle = {"substeps_per_s": pc_value, "cores": pc_n, "ess_per_s": ess_per_substep * pc_value,
                  "sample": f"{pc_n} processes, one oracle chain each (single-threaded BLAS), {pc_l} leapfrogs "
                            f"in {pc_s:.1f} s; ESS per substep taken from the FP64 GPU run"}
    for r in runs.values():
        r.pop("_draws")
        r.pop("_accept")
    z_mean = np.abs(a["mean"] - b["mean"]) / np.sqrt(a["se_mean"] ** 2 + b["se_mean"] ** 2)
    z_var = np.abs(a["var"] - b["var"]) / np.sqrt(a["se_var"] ** 2 + b["se_var"] ** 2)
    matched = bool((z_mean <= 3).all() and (z_var <= 3).all())
    for r in runs.values():
        for key in ("mean", "var", "se_mean", "se_var"):
            r[key] = [round(float(v), 6) for v in r[key]]
    print(json.dumps({"metric": "effective samples/s (min over log P, hyperparameters and a mean coordinate; bulk and tail ESS)",
                      "value": b["ess_per_s"], "unit": "ESS/s", "n_gpus": 1, "higher_is_better": True,
                      "dtype": "f64; mixed: " + DTYPE_MIXED, "data": "synthetic",
                      "config": {"workload": f"{label}, {C} chains, eps={eps}, L=10, "
                                             f"n_fp=6, {args.burn} burn-in + {args.iters} kept iterations",
                                 "quantities": names},
                      "fp64": runs["fp64"], "mixed": runs["mixed"],
                      "speedup_ess_per_s": b["ess_per_s"] / a["ess_per_s"] if a["ess_per_s"] > 0 else None,
                      "same_seed_paths": paths, "oracle_host": oracle,
                      "matched_error": {"z_mean": [round(float(v), 2) for v in z_mean],
                                        "z_var": [round(float(v), 2) for v in z_var], "within_3_se": matched}}),
          flush=True)
    return 0


def run_solin(args):
    """The primal (reduced-rank) model of the paper's own experiments (Sec. 2.5): simulated
    logistic data, N = 500, D Gaussian kernels x M = 30 sinusoidal features (d = 30 D + 4), g =
    sqrt(1 + lambda^2), eps = 0.001, n_fp = 6; both precisions, one after the other."""
    import torch
    from paper_2511_06407_b300 import build, rmhmc
    build.build()
    D = args.solin_d
    prob = wl.solin_logistic(D, N=500, seed=0)
    C = args.chains
    out = {}
    for prec in ("mixed", "fp64"):
        model = rmhmc.Model(prob, C)
        integ = rmhmc.Integrator(eps=args.eps or SOLIN_EPS, n_fp=N_FP, n_leapfrog=1, g_kind="sqrt",
                                 alpha=1.0 / SOLIN_KAPPA,
                                 precision=prec)
        model.set_state(torch.zeros(C, model.d, dtype=torch.float64, device="cuda"), integ=integ)
        tuned = model.autotune(integ)
        model.sample(1, 0, 5, integ=integ)
        model.leapfrog(max(args.warmup - 1, 0), integ=integ)
        st = torch.empty(C, dtype=torch.int32, device="cuda")
        el, clk = _clock_and_time(lambda: model.leapfrog(args.steps, status_out=st, integ=integ), 0)
        model.profile(True)  # one more leapfrog with the per-launch events, outside the timed region
        model.leapfrog(1, integ=integ)
        prof = model.profile_read()
        model.profile(False)
        out[prec] = {"value": C * SUBSTEPS_PER_LEAPFROG * args.steps / el,
                     "leapfrogs_per_s_per_chain": args.steps / el, "ms_per_step": 1e3 * el / args.steps,
                     "profile_ms": {k: round(v[0], 1) for k, v in prof.items() if v[2]},
                     "roofline": _roofline(rmhmc, prof, C), "autotuned_cluster_schedule_tile": tuned,
                     "chain_status_nonzero": int((st.cpu().numpy() != 0).sum()), "clocks": clk}
        d = model.d
        model.close()
    head = out[aux_precision(args)]
    print(json.dumps({"metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
                      "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
                      "dtype": dtype_of(aux_precision(args)), "data": "synthetic",
                      "config": {"workload": f"primal reduced-rank model (Sec. 2.5): simulated logistic data N=500, "
                                             f"D={D} Gaussian kernels x 30 features (d={d}), {C} chains, "
                                             f"g=sqrt(1+l^2), eps={args.eps or 0.001}", "d": d, "chains": C},
                      "mixed": out["mixed"], "fp64": out["fp64"],
                      "speedup_vs_fp64": out["mixed"]["value"] / out["fp64"]["value"]}), flush=True)
    return 0


def run_fig1c(args):
    """Fig. 1C's comparison: eigen-update work per Hessian, static (cold start from Psi = I at every
    eigen-update) against dynamic (warm start from the previous Psi, Sec. 2.4), across the primal
    model's dimension (the simulated data of Sec. 2.5, D = 1, 2, 4, 8, 16 Gaussian kernels: d = 34 ..
    484), under both stopping rules (METRIC, the sampler's default, and RELATIVE, every eigenpair
    resolved), with both rotation orders. Per configuration: args.chains chains, one Algorithm 1
    iteration (L = 10, eps = 0.001, n_fp = 6, g = sqrt(1 + l^2)) after one untimed iteration; reported
    per eigen-update: sweeps (cyclic-sweep equivalents), rounds, 16 x 16 sub-problems solved and
    rotated, rotation-tile products, and the iteration's time."""
    import torch
    from paper_2511_06407_b300 import build, rmhmc
    build.build()
    C = args.chains
    rows = []
    for D in (1, 2, 4, 8, 16):
        prob = wl.solin_logistic(D, N=500, seed=0)
        for rule in ("metric", "relative"):
            for start in ("warm", "cold"):
                for sched in ("cyclic", "dynamic"):
                    integ = rmhmc.Integrator(eps=args.eps or SOLIN_EPS, n_fp=N_FP, n_leapfrog=N_LEAPFROG,
                                             g_kind="sqrt", alpha=1.0 / SOLIN_KAPPA, precision=aux_precision(args),
                                             jacobi_rule=rule, eigen_start=start)
                    model = rmhmc.Model(prob, C)
                    model.set_jacobi(0, sched)
                    model.set_state(torch.zeros(C, model.d, dtype=torch.float64, device="cuda"), integ=integ)
                    model.sample(1, 0, 5, integ=integ)
                    model.profile(True)
                    model.profile(False)  # resets the counters
                    sw = torch.zeros(1, C, dtype=torch.int32, device="cuda")
                    cs = torch.zeros(C, dtype=torch.int32, device="cuda")
                    el, _ = _clock_and_time(lambda: model.sample(1, 0, 5, sweeps=sw, chain_status=cs, integ=integ), 0)
                    cnt = model.jacobi_counters()
                    u = max(cnt["updates"], 1)
                    rows.append({"D": D, "d": model.d, "rule": rule, "start": start, "schedule": sched,
                                 "sweeps_per_update": float(sw.cpu().numpy().sum()) / u,
                                 "rounds_per_update": cnt["rounds"] / u, "solves_per_update": cnt["solves"] / u,
                                 "rotated_per_update": cnt["rotated"] / u,
                                 "tile_products_per_update": cnt["tile_products"] / u,
                                 "updates": cnt["updates"], "iteration_ms": 1e3 * el,
                                 "chain_status_nonzero": int((cs.cpu().numpy() != 0).sum())})
                    print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
                    model.close()
    print(json.dumps({"metric": "Jacobi work per eigen-update, static vs dynamic (Fig. 1C)", "unit": "per update",
                      "n_gpus": 1, "dtype": dtype_of(aux_precision(args)), "data": "synthetic",
                      "config": {"workload": f"primal model of Sec. 2.5 (N=500, D=1..16, d=34..484), {C} chains, "
                                             f"one Algorithm 1 iteration (L={N_LEAPFROG}, eps={args.eps or SOLIN_EPS}, "
                                             f"n_fp={N_FP}) after one untimed"},
                      "rows": rows}), flush=True)
    return 0


def run_uneven(args):
    """The uneven-batch configuration: args.problems problems (default 128, seeds 0..127),
    N ~ U{32..512}, 1-3 additive kernels (SE, linear, overlap), 8 chains each (1024 chains,
    d from 34 to 1542), advanced together by one captured CUDA graph per leapfrog over the
    problems' streams. Each problem's Jacobi cluster size and rotation schedule come from the
    autotuner, run once per size class (d in steps of 128, same number of kernels) and shared
    within the class. A step is one generalized leapfrog of every chain (13 substeps)."""
    import torch
    from paper_2511_06407_b300 import build, rmhmc
    build.build()
    n_max = args.uneven_nmax
    probs = wl.uneven_batch(args.problems, seed=0, n_min=32, n_max=n_max)
    C = 8
    prec = aux_precision(args)
    integ = rmhmc.Integrator(eps=args.eps or EPS, n_fp=N_FP, n_leapfrog=1, precision=prec)
    plan = sum(rmhmc.plan_bytes(p, C) for p in probs)
    models, tuned, choice = [], {}, []
    t_setup = time.perf_counter()
    streams = []
    for i, prob in enumerate(probs):
        s = rmhmc.new_stream()  # one distinct stream per problem (torch's pool has 32)
        streams.append(s)
        with torch.cuda.stream(s):
            m = rmhmc.Model(prob, C, stream=s)
            m.set_state(torch.zeros(C, m.d, dtype=torch.float64, device="cuda"), integ=integ)
            key = (m.d // 128, len(prob["kernels"]))
            if key not in tuned:
                tuned[key] = m.autotune(integ)
            else:
                m.set_jacobi(*tuned[key][:2])
                m.set_gemm_tile(tuned[key][2])
                m.set_prerotation(tuned[key][3])
            choice.append(tuned[key])
            m.sample(1, 0, 7 + i, integ=integ)
        models.append(m)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t_setup
    batch = rmhmc.Batch(models)
    t0 = time.perf_counter()
    batch.leapfrog(1, integ)  # captures the graph
    torch.cuda.synchronize()
    t_capture = time.perf_counter() - t0
    if args.warmup > 1:
        batch.leapfrog(args.warmup - 1, integ)
    el, clk = _clock_and_time(lambda: batch.leapfrog(args.steps, integ), 0)
    st = []
    for m in models:
        x = torch.empty(C, dtype=torch.int32, device="cuda")
        with torch.cuda.stream(m.stream):
            m.leapfrog(0, status_out=x, integ=integ)
        st.append(x)
    torch.cuda.synchronize()
    bad = int(sum((x.cpu().numpy() != 0).sum() for x in st))
    chains = C * len(models)
    ds = [m.d for m in models]
    scheds = {}
    for c, sc, nt, pr in choice:
        key = f"{sc}/{c}/{nt}/{'pre' if pr else 'nopre'}"
        scheds[key] = scheds.get(key, 0) + 1
    print(json.dumps({"metric": METRIC, "value": chains * SUBSTEPS_PER_LEAPFROG * args.steps / el, "unit": UNIT,
                      "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
                      "dtype": dtype_of(prec), "data": "synthetic",
                      "config": {"workload": f"uneven batch: {len(models)} problems (seeds 0..{len(models) - 1}), "
                                             f"N~U{{32..{n_max}}}, 1-3 kernels (SE, linear, overlap), 8 chains "
                                             f"each, one captured CUDA graph per leapfrog over the problems' "
                                             f"streams, eps={integ.eps}, n_fp={N_FP}",
                                 "step": "one generalized leapfrog of every chain (13 substeps)",
                                 "d_min": min(ds), "d_max": max(ds), "d_mean": float(np.mean(ds)),
                                 "chains": chains, "device_bytes_planned": plan,
                                 "autotuned_schedule_cluster_tile": scheds, "autotuned_classes": len(tuned)},
                      "setup_s": t_setup, "graph_capture_s": t_capture,
                      "chain_status_nonzero": bad, "valid": bad == 0, "clocks": clk}), flush=True)
    batch.close()
    for m in models:
        m.close()
    torch.cuda.synchronize()
    for s in streams:
        rmhmc.release_stream(s)
    return 0


def run_serve(args):
    """The served-stream configuration: a Poisson trace of args.jobs arrivals at args.rate per second
    (default 64 at 50/s) of sampling jobs with N ~ U{args.serve_nmin..args.serve_nmax} (default
    50..800), 1-3 additive kernels, 16 inverse temperatures tau_s = (s/15)^5 x 4 chains (64 chains
    per job), served with continuous batching by the library's scheduler under an HBM budget. The
    configuration asks for 500 iterations per job; one B300 needs hours for that trace (a job is
    ~1e15-1e17 FP operations), so the iterations (args.serve_burn + args.serve_iters of
    args.serve_leapfrogs leapfrogs) are scaled down and printed. Each finished job's tempered chains
    give a ln BME estimate by thermodynamic integration over its 16 temperatures (the BME appendix)."""
    from paper_2511_06407_b300 import bme, build, rmhmc
    from paper_2511_06407_b300.serve import Job, Server, poisson_trace
    build.build()
    probs = wl.uneven_batch(args.jobs, seed=100, n_min=args.serve_nmin, n_max=args.serve_nmax)
    prec = aux_precision(args)
    integ = rmhmc.Integrator(eps=args.eps or EPS, n_fp=N_FP, n_leapfrog=args.serve_leapfrogs, precision=prec)
    temps = bme.power_schedule(args.serve_temps)
    taus = np.repeat(temps, args.serve_chains_per_temp)
    C = len(taus)
    arrivals = poisson_trace(probs, args.rate, seed=1)
    jobs = [Job(p, C, n_iter=args.serve_iters, n_burn=args.serve_burn, seed=i, tau=taus, integ=integ,
                arrival=a, job_id=i) for i, (p, a) in enumerate(zip(probs, arrivals))]
    done, stats = Server(hbm_budget_bytes=int(args.hbm_gb * 2**30)).run(jobs)
    bad = int(sum((j.chain_status != 0).sum() for j in done))
    lnz = []
    for j in done:
        ok = j.chain_status == 0
        if ok.all() and np.all(np.isfinite(j.loglik)):
            est, se, _ = bme.evidence(taus, j.loglik)
            lnz.append((j.job_id, wl.dims(j.problem)[2], est, se))
    ds = [wl.dims(p)[2] for p in probs]
    print(json.dumps({"metric": "served RMHMC substeps/s; job latency p50/p99", "value": stats["substeps_per_s"],
                      "unit": UNIT, "n_gpus": 1, "higher_is_better": True, "dtype": dtype_of(prec),
                      "data": "synthetic",
                      "p50_latency_s": stats["p50_latency_s"], "p99_latency_s": stats["p99_latency_s"],
                      "makespan_s": stats["makespan_s"], "jobs": stats["jobs"],
                      "max_concurrent_jobs": stats["max_concurrent_jobs"],
                      "config": {"workload": f"Poisson trace, {args.jobs} jobs at {args.rate}/s, "
                                             f"N~U{{{args.serve_nmin}..{args.serve_nmax}}}, 1-3 kernels, "
                                             f"{args.serve_temps} temperatures (s/{args.serve_temps - 1})^5 x "
                                             f"{args.serve_chains_per_temp} chains, {args.serve_burn} burn-in + "
                                             f"{args.serve_iters} recorded iterations x {args.serve_leapfrogs} "
                                             f"leapfrogs (the configuration's 500 iterations scaled down), "
                                             f"HBM budget {args.hbm_gb} GiB, native scheduler (rmhmc_server_*)",
                                 "eps": integ.eps, "d_min": min(ds), "d_max": max(ds),
                                 "d_mean": float(np.mean(ds)), "chains_per_job": C},
                      "bme_jobs": len(lnz), "bme_examples": lnz[:4],
                      "chain_status_nonzero": bad}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="b300", choices=["b300", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--fp64-steps", type=int, default=3,
                    help="timed iterations of the plain FP64 comparison leg (at most --steps)")
    ap.add_argument("--e2e-steps", type=int, default=5,
                    help="iterations of the end-to-end leg (at most --steps)")
    ap.add_argument("--chains", type=int, default=N_CHAINS,
                    help="chains per GPU (the workload is 64; smaller values are for profiling)")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle timing leg")
    ap.add_argument("--workload", default="gp400",
                    choices=["gp400", "propensity", "uneven", "serve", "ess", "solin", "fig1c"],
                    help="gp400 is the benchmark; the others are extra measurements")
    ap.add_argument("--eps", type=float, default=None)
    ap.add_argument("--precision", default="both", choices=["both", "fp64", "mixed"],
                    help="both (default): the mixed form is the headline, timed beside the plain FP64 path "
                         "on the same workload, with the trajectory error between them")
    ap.add_argument("--problems", type=int, default=128)
    ap.add_argument("--uneven-nmax", type=int, default=512, help="largest N of the uneven batch")
    ap.add_argument("--ess-n", type=int, default=100, help="inputs N of the dual ESS workload")
    ap.add_argument("--ess-model", default="primal", choices=["primal", "dual"])
    ap.add_argument("--ess-same-seed", action="store_true",
                    help="both precisions use the same seed (their chains then follow each other)")
    ap.add_argument("--ess-d", type=int, default=4, help="Gaussian kernels D of the primal ESS workload")
    ap.add_argument("--solin-d", type=int, default=16, help="Gaussian kernels D of the solin workload (d = 30 D + 4)")
    ap.add_argument("--iters", type=int, default=200, help="kept iterations of the ESS workload")
    ap.add_argument("--burn", type=int, default=100, help="burn-in iterations of the ESS workload")
    ap.add_argument("--jobs", type=int, default=64)
    ap.add_argument("--rate", type=float, default=50.0)
    ap.add_argument("--hbm-gb", type=float, default=200.0)
    ap.add_argument("--serve-nmin", type=int, default=50)
    ap.add_argument("--serve-nmax", type=int, default=800)
    ap.add_argument("--serve-temps", type=int, default=16)
    ap.add_argument("--serve-chains-per-temp", type=int, default=4)
    ap.add_argument("--serve-iters", type=int, default=2, help="recorded iterations per served job")
    ap.add_argument("--serve-burn", type=int, default=0)
    ap.add_argument("--serve-leapfrogs", type=int, default=2, help="leapfrogs per served iteration")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "propensity":
        return run_propensity(args)
    if args.workload == "uneven":
        return run_uneven(args)
    if args.workload == "ess":
        return run_ess(args)
    if args.workload == "solin":
        return run_solin(args)
    if args.workload == "fig1c":
        return run_fig1c(args)
    if args.workload == "serve":
        return run_serve(args)
    return run_b300(args)


if __name__ == "__main__":
    sys.exit(main())
