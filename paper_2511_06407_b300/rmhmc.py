"""Thin ctypes binding of librmhmc (include/rmhmc.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts workload dicts and torch CUDA
tensors into the C structs and device pointers the ABI takes, and raises on a non-OK status.
There is no fallback: if librmhmc.so is missing or fails to load, every call raises.
"""
import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int, c_uint64, c_void_p
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librmhmc.so")

MAX_COLS = 16
KINDS = {"se": 0, "linear": 1, "overlap": 2}
LIKS = {"bernoulli": 0, "gaussian": 1, "meanvar": 2}
GKINDS = {"coth": 0, "sqrt": 1}
PRECISIONS = {"fp64": 0, "mixed": 1}
JACOBI_RULES = {"metric": 0, "relative": 1}
EIGEN_STARTS = {"warm": 0, "cold": 1}
CHAIN_NOTPD, CHAIN_NOTCONV, CHAIN_NONFINITE, CHAIN_TIMEOUT = 1, 2, 4, 8
JACOBI_SCHEDULES = ["cyclic", "dynamic"]  # rmhmc_jacobi_schedule
PROF_NCAT = 11


class KernelDesc(ctypes.Structure):
    _fields_ = [("kind", c_int), ("n_cols", c_int), ("cols", c_int * MAX_COLS), ("jitter", c_double),
                ("prior_a", c_double * 2), ("prior_b", c_double * 2)]


class ModelDesc(ctypes.Structure):
    _fields_ = [("N", c_int), ("n_cov", c_int), ("X", POINTER(c_double)), ("y", POINTER(c_double)),
                ("lik", c_int), ("noise_var", c_double), ("n_kernels", c_int),
                ("kernels", POINTER(KernelDesc)), ("sample_hypers", c_int),
                ("u_fixed", POINTER(c_double))]


class PrimalDesc(ctypes.Structure):
    _fields_ = [("N", c_int), ("n_gauss", c_int), ("n_linear", c_int), ("Xg", POINTER(c_double)),
                ("Xl", POINTER(c_double)), ("y", POINTER(c_double)), ("lik", c_int),
                ("noise_var", c_double), ("M", c_int), ("L", c_double), ("bias_var", c_double),
                ("prior_a", c_double * 3), ("prior_b", c_double * 3), ("J", c_int), ("delta", c_double)]


class IntegratorC(ctypes.Structure):
    _fields_ = [("eps", c_double), ("n_leapfrog", c_int), ("n_fp", c_int), ("g_kind", c_int),
                ("alpha", c_double), ("jacobi_tol", c_double), ("max_sweeps", c_int),
                ("reorth_every", c_int), ("precision", c_int), ("jacobi_rule", c_int),
                ("eigen_start", c_int)]


class JobDesc(ctypes.Structure):
    _fields_ = [("model", POINTER(ModelDesc)), ("primal", POINTER(PrimalDesc)), ("n_chains", c_int),
                ("tau_host", POINTER(c_double)), ("q0_host", POINTER(c_double)), ("integ", IntegratorC),
                ("n_iter", c_int), ("n_burn", c_int), ("seed", ctypes.c_uint64), ("q_samples_dev", c_void_p),
                ("logp_dev", c_void_p), ("accept_dev", c_void_p), ("chain_status_dev", c_void_p),
                ("loglik_dev", c_void_p)]


@dataclass
class Integrator:
    """Leapfrog and geometry settings (rmhmc_integrator)."""
    eps: float = 0.1
    n_leapfrog: int = 10
    n_fp: int = 6
    g_kind: str = "coth"
    alpha: float = 1e6
    jacobi_tol: float = 1e-13
    max_sweeps: int = 30
    reorth_every: int = 10
    precision: str = "fp64"
    jacobi_rule: str = "metric"
    eigen_start: str = "warm"

    def c(self):
        return IntegratorC(self.eps, self.n_leapfrog, self.n_fp, GKINDS[self.g_kind], self.alpha,
                           self.jacobi_tol, self.max_sweeps, self.reorth_every,
                           PRECISIONS[self.precision], JACOBI_RULES[self.jacobi_rule],
                           EIGEN_STARTS[self.eigen_start])


class RmhmcError(RuntimeError):
    pass


_lib_handle = None


def lib():
    """Load librmhmc.so (raises if it is missing: there is no CPU fallback)."""
    global _lib_handle
    if _lib_handle is not None:
        return _lib_handle
    if not os.path.exists(LIB_PATH):
        raise RmhmcError(f"{LIB_PATH} is missing: build it with `python -m paper_2511_06407_b300.build`")
    L = ctypes.CDLL(LIB_PATH)
    L.rmhmc_init_model.argtypes = [POINTER(ModelDesc), c_int, POINTER(c_double), c_void_p,
                                   POINTER(c_void_p)]
    L.rmhmc_set_state.argtypes = [c_void_p, POINTER(IntegratorC), c_void_p, c_void_p]
    L.rmhmc_leapfrog.argtypes = [c_void_p, POINTER(IntegratorC), c_int, c_void_p, c_void_p,
                                 c_void_p, c_void_p, c_void_p]
    L.rmhmc_sample.argtypes = [c_void_p, POINTER(IntegratorC), c_int, c_int, c_uint64, c_void_p,
                               c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]
    L.rmhmc_geometry.argtypes = [c_void_p] + [c_void_p] * 6
    L.rmhmc_hamiltonian_grad.argtypes = [c_void_p] + [c_void_p] * 4
    L.rmhmc_dim.argtypes = [c_void_p]
    L.rmhmc_dim.restype = c_int
    L.rmhmc_n_chains.argtypes = [c_void_p]
    L.rmhmc_n_chains.restype = c_int
    L.rmhmc_free_model.argtypes = [c_void_p]
    L.rmhmc_free_model.restype = None
    L.rmhmc_profile.argtypes = [c_void_p, c_int]
    L.rmhmc_profile.restype = c_int
    L.rmhmc_profile_read.argtypes = [c_void_p, POINTER(c_double), POINTER(c_double),
                                     POINTER(ctypes.c_longlong)]
    L.rmhmc_profile_read.restype = c_int
    L.rmhmc_profile_category.argtypes = [c_int]
    L.rmhmc_profile_category.restype = c_char_p
    L.rmhmc_fp64_peak.argtypes = [c_void_p, c_int, POINTER(c_double)]
    L.rmhmc_fp64_peak.restype = c_int
    L.rmhmc_fp32_peak.argtypes = [c_void_p, c_int, POINTER(c_double)]
    L.rmhmc_fp32_peak.restype = c_int
    L.rmhmc_df_peak.argtypes = [c_void_p, c_int, POINTER(c_double)]
    L.rmhmc_df_peak.restype = c_int
    L.rmhmc_eigh_noalloc.argtypes = [c_void_p, c_int, c_int, c_void_p, c_void_p, c_void_p,
                                     c_double, c_int, c_void_p, c_void_p]
    L.rmhmc_eigh_noalloc.restype = c_int
    L.rmhmc_gemm_tc.argtypes = [c_void_p, c_int, c_int, c_int, c_int, c_int, c_double, c_void_p,
                                c_int, ctypes.c_longlong, c_void_p, c_int, ctypes.c_longlong,
                                c_double, c_void_p, c_int, ctypes.c_longlong, c_int, c_int, c_int,
                                c_void_p]
    L.rmhmc_gemm_tc.restype = c_int
    L.rmhmc_test_gemm_stall.argtypes = [c_int, c_double]
    L.rmhmc_test_gemm_stall.restype = c_int
    L.rmhmc_server_create.argtypes = [c_int, ctypes.c_size_t, c_int, POINTER(c_void_p)]
    L.rmhmc_server_create.restype = c_int
    L.rmhmc_server_submit.argtypes = [c_void_p, POINTER(JobDesc), POINTER(c_int)]
    L.rmhmc_server_submit.restype = c_int
    L.rmhmc_server_poll.argtypes = [c_void_p, c_int, POINTER(c_int), POINTER(c_int), POINTER(c_double)]
    L.rmhmc_server_poll.restype = c_int
    L.rmhmc_server_wait.argtypes = [c_void_p, c_int, c_double]
    L.rmhmc_server_wait.restype = c_int
    L.rmhmc_server_stats.argtypes = [c_void_p, POINTER(c_double), POINTER(c_int), POINTER(c_int),
                                     POINTER(c_int), POINTER(ctypes.c_size_t)]
    L.rmhmc_server_stats.restype = c_int
    L.rmhmc_server_destroy.argtypes = [c_void_p]
    L.rmhmc_server_destroy.restype = None
    L.rmhmc_batch_create.argtypes = [POINTER(c_void_p), c_int, c_void_p, POINTER(c_void_p)]
    L.rmhmc_batch_create.restype = c_int
    L.rmhmc_batch_leapfrog.argtypes = [c_void_p, POINTER(IntegratorC), c_int]
    L.rmhmc_batch_leapfrog.restype = c_int
    L.rmhmc_batch_free.argtypes = [c_void_p]
    L.rmhmc_batch_free.restype = None
    L.rmhmc_autotune.argtypes = [c_void_p, POINTER(IntegratorC), POINTER(c_int), POINTER(c_int), POINTER(c_int),
                                 POINTER(c_int)]
    L.rmhmc_set_gemm_tile.argtypes = [c_void_p, c_int]
    L.rmhmc_set_gemm_tile.restype = c_int
    L.rmhmc_autotune.restype = c_int
    L.rmhmc_set_jacobi.argtypes = [c_void_p, c_int, c_int]
    L.rmhmc_set_jacobi.restype = c_int
    L.rmhmc_set_prerotation.argtypes = [c_void_p, c_int]
    L.rmhmc_set_prerotation.restype = c_int
    L.rmhmc_stream_create.argtypes = [POINTER(c_void_p)]
    L.rmhmc_stream_create.restype = c_int
    L.rmhmc_stream_destroy.argtypes = [c_void_p]
    L.rmhmc_stream_destroy.restype = c_int
    L.rmhmc_jacobi_counters.argtypes = [c_void_p, POINTER(ctypes.c_longlong)]
    L.rmhmc_jacobi_counters.restype = c_int
    L.rmhmc_plan_bytes.argtypes = [POINTER(ModelDesc), c_int, POINTER(ctypes.c_size_t)]
    L.rmhmc_plan_bytes.restype = c_int
    L.rmhmc_init_primal.argtypes = [POINTER(PrimalDesc), c_int, POINTER(c_double), c_void_p,
                                    POINTER(c_void_p)]
    L.rmhmc_init_primal.restype = c_int
    L.rmhmc_plan_bytes_primal.argtypes = [POINTER(PrimalDesc), c_int, POINTER(ctypes.c_size_t)]
    L.rmhmc_plan_bytes_primal.restype = c_int
    L.rmhmc_version.argtypes = []
    L.rmhmc_status_string.argtypes = [c_int]
    L.rmhmc_status_string.restype = c_char_p
    L.rmhmc_version.restype = c_char_p
    for name in ("rmhmc_init_model", "rmhmc_set_state", "rmhmc_leapfrog", "rmhmc_sample",
                 "rmhmc_geometry", "rmhmc_hamiltonian_grad"):
        getattr(L, name).restype = c_int
    _lib_handle = L
    return L


def _check(rc):
    if rc != 0:
        raise RmhmcError(f"rmhmc status {rc}: {lib().rmhmc_status_string(rc).decode()}")


def _ptr(t, shape=None, dtype=None):
    """Device pointer of a contiguous CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
        raise RmhmcError("expected a contiguous CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise RmhmcError(f"expected dtype {dtype}, got {t.dtype}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise RmhmcError(f"expected shape {tuple(shape)}, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


def _desc(problem):
    """(ModelDesc, keep-alive list) for a workload dict."""
    X = np.ascontiguousarray(problem["X"], dtype=np.float64)
    y = np.ascontiguousarray(problem["y"], dtype=np.float64)
    ks = (KernelDesc * len(problem["kernels"]))()
    for i, k in enumerate(problem["kernels"]):
        cols = list(k["cols"])
        if not 1 <= len(cols) <= MAX_COLS:
            raise RmhmcError(f"kernel {i}: {len(cols)} covariate columns (1..{MAX_COLS} supported)")
        ks[i].kind = KINDS[k["kind"]]
        ks[i].n_cols = len(cols)
        for j, cidx in enumerate(cols):
            ks[i].cols[j] = int(cidx)
        ks[i].jitter = float(k["jitter"])
        ks[i].prior_a[0], ks[i].prior_a[1] = (float(v) for v in k["prior_a"])
        ks[i].prior_b[0], ks[i].prior_b[1] = (float(v) for v in k["prior_b"])
    uf = None
    if not problem["sample_hypers"]:
        uf = np.ascontiguousarray(problem["u_fixed"], dtype=np.float64)
    desc = ModelDesc(X.shape[0], X.shape[1], X.ctypes.data_as(POINTER(c_double)),
                     y.ctypes.data_as(POINTER(c_double)), LIKS[problem["lik"]],
                     float(problem["noise_var"]), len(problem["kernels"]), ks,
                     1 if problem["sample_hypers"] else 0,
                     uf.ctypes.data_as(POINTER(c_double)) if uf is not None else None)
    return desc, [X, y, ks, uf]


def _primal_desc(problem):
    """(PrimalDesc, keep-alive list) for a primal-model workload dict."""
    y = np.ascontiguousarray(problem["y"], dtype=np.float64)
    N = y.shape[0]
    Xg = np.ascontiguousarray(problem["Xg"], dtype=np.float64).reshape(N, -1)
    Xl = np.ascontiguousarray(problem["Xl"], dtype=np.float64).reshape(N, -1)
    desc = PrimalDesc(N, Xg.shape[1], Xl.shape[1],
                      Xg.ctypes.data_as(POINTER(c_double)) if Xg.shape[1] else None,
                      Xl.ctypes.data_as(POINTER(c_double)) if Xl.shape[1] else None,
                      y.ctypes.data_as(POINTER(c_double)), LIKS[problem["lik"]], float(problem["noise_var"]),
                      int(problem["M"]), float(problem["L"]), float(problem["bias_var"]),
                      (c_double * 3)(*[float(v) for v in problem["prior_a"]]),
                      (c_double * 3)(*[float(v) for v in problem["prior_b"]]),
                      int(problem.get("J", 1)), float(problem.get("delta", 0.0)))
    return desc, [y, Xg, Xl]


def is_primal(problem):
    return problem.get("model") == "primal"


def plan_bytes(problem, n_chains):
    """Device bytes a Model for this problem and chain count would allocate (rmhmc_plan_bytes)."""
    out = ctypes.c_size_t()
    if is_primal(problem):
        desc, keep = _primal_desc(problem)
        _check(lib().rmhmc_plan_bytes_primal(ctypes.byref(desc), int(n_chains), ctypes.byref(out)))
    else:
        desc, keep = _desc(problem)
        _check(lib().rmhmc_plan_bytes(ctypes.byref(desc), int(n_chains), ctypes.byref(out)))
    return out.value


class Model:
    """One problem (a workload dict) with n_chains chains on the current CUDA device/stream."""

    def __init__(self, problem, n_chains, tau=None, stream=None):
        import torch
        L = lib()
        primal = is_primal(problem)
        desc, keep = _primal_desc(problem) if primal else _desc(problem)
        tau_arr = None
        if tau is not None:
            tau_arr = np.ascontiguousarray(np.broadcast_to(np.asarray(tau, dtype=np.float64), (n_chains,)))
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        handle = c_void_p()
        init = L.rmhmc_init_primal if primal else L.rmhmc_init_model
        _check(init(ctypes.byref(desc), int(n_chains),
                    tau_arr.ctypes.data_as(POINTER(c_double)) if tau_arr is not None else None,
                    c_void_p(stream.cuda_stream), ctypes.byref(handle)))
        self._h = handle
        self.d = L.rmhmc_dim(self._h)
        self.n_chains = L.rmhmc_n_chains(self._h)
        self.integ = None

    def close(self):
        if getattr(self, "_h", None):
            lib().rmhmc_free_model(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _integ(self, integ):
        integ = integ or self.integ or Integrator()
        return integ, integ.c()

    def set_state(self, q, p=None, integ=None):
        import torch
        integ, ic = self._integ(integ)
        self.integ = integ
        sh = (self.n_chains, self.d)
        _check(lib().rmhmc_set_state(self._h, ctypes.byref(ic), _ptr(q, sh, torch.float64),
                                     _ptr(p, sh, torch.float64)))

    def leapfrog(self, n_steps, q_out=None, p_out=None, H_out=None, status_out=None, integ=None,
                 p_in=None):
        import torch
        integ, ic = self._integ(integ)
        sh = (self.n_chains, self.d)
        _check(lib().rmhmc_leapfrog(self._h, ctypes.byref(ic), int(n_steps),
                                    _ptr(p_in, sh, torch.float64),
                                    _ptr(q_out, sh, torch.float64), _ptr(p_out, sh, torch.float64),
                                    _ptr(H_out, (self.n_chains,), torch.float64),
                                    _ptr(status_out, (self.n_chains,), torch.int32)))

    def sample(self, n_iter, n_burn, seed, q_samples=None, logp=None, accept=None, sweeps=None,
               chain_status=None, integ=None, loglik=None):
        import torch
        integ, ic = self._integ(integ)
        C, d = self.n_chains, self.d
        _check(lib().rmhmc_sample(self._h, ctypes.byref(ic), int(n_iter), int(n_burn), int(seed),
                                  _ptr(q_samples, (n_iter, C, d), torch.float64),
                                  _ptr(logp, (n_iter, C), torch.float64),
                                  _ptr(loglik, (n_iter, C), torch.float64),
                                  _ptr(accept, (n_iter, C), torch.int32),
                                  _ptr(sweeps, (n_iter, C), torch.int32),
                                  _ptr(chain_status, (C,), torch.int32)))

    def geometry(self, U=None, dU=None, hess=None, lam=None, G=None, sweeps=None):
        import torch
        C, d = self.n_chains, self.d
        f64 = torch.float64
        _check(lib().rmhmc_geometry(self._h, _ptr(U, (C,), f64), _ptr(dU, (C, d), f64),
                                    _ptr(hess, (C, d, d), f64), _ptr(lam, (C, d), f64),
                                    _ptr(G, (C, d, d), f64), _ptr(sweeps, (C,), torch.int32)))

    def hamiltonian_grad(self, p, dHdq=None, Ginv_p=None, H=None):
        import torch
        C, d = self.n_chains, self.d
        f64 = torch.float64
        _check(lib().rmhmc_hamiltonian_grad(self._h, _ptr(p, (C, d), f64), _ptr(dHdq, (C, d), f64),
                                            _ptr(Ginv_p, (C, d), f64), _ptr(H, (C,), f64)))


    def autotune(self, integ=None):
        """Pick this model's Jacobi cluster size, rotation schedule and (mixed form) GEMM tile width
        and pre-rotation by timing leapfrogs (rmhmc_autotune); returns (cluster, schedule name, tile,
        pre-rotation on)."""
        integ = integ or self.integ or Integrator()
        cl, sc, nt, pr = c_int(), c_int(), c_int(), c_int()
        _check(lib().rmhmc_autotune(self._h, ctypes.byref(integ.c()), ctypes.byref(cl), ctypes.byref(sc),
                                    ctypes.byref(nt), ctypes.byref(pr)))
        return cl.value, JACOBI_SCHEDULES[sc.value], nt.value, bool(pr.value)

    def set_gemm_tile(self, nt=64):
        """Output tile width of the model's tensor-core GEMMs, 64 or 32 (rmhmc_set_gemm_tile)."""
        _check(lib().rmhmc_set_gemm_tile(self._h, int(nt)))

    def set_prerotation(self, enable=True):
        """Turn the mixed form's first-order pre-rotation of warm eigen-updates on or off
        (rmhmc_set_prerotation)."""
        _check(lib().rmhmc_set_prerotation(self._h, 1 if enable else 0))

    def jacobi_counters(self):
        """Eigen-update work since the last profile reset (rmhmc_jacobi_counters), as a dict."""
        out = (ctypes.c_longlong * 8)()
        _check(lib().rmhmc_jacobi_counters(self._h, out))
        keys = ("tile_products", "inner_rounds", "rounds", "solves", "rotated", "updates",
                "prerotated_updates", "prerotated_pairs")
        return dict(zip(keys, [int(v) for v in out]))

    def set_jacobi(self, cluster=0, schedule="cyclic"):
        """Set the Jacobi cluster size (0 = default) and rotation schedule ("cyclic"/"dynamic")."""
        _check(lib().rmhmc_set_jacobi(self._h, int(cluster), JACOBI_SCHEDULES.index(schedule)))

    def profile(self, enable=True):
        _check(lib().rmhmc_profile(self._h, 1 if enable else 0))

    def profile_read(self):
        """{category: (ms, flops, launches)} since profile(True); synchronises the stream."""
        n = PROF_NCAT
        ms, fl, ln = (c_double * n)(), (c_double * n)(), (ctypes.c_longlong * n)()
        _check(lib().rmhmc_profile_read(self._h, ms, fl, ln))
        return {lib().rmhmc_profile_category(i).decode(): (ms[i], fl[i], int(ln[i])) for i in range(n)}


class Batch:
    """Models of different sizes advanced together by one CUDA graph per leapfrog
    (rmhmc_batch_*). Each model must have been created with its own torch.cuda.Stream."""

    def __init__(self, models, stream=None):
        import torch
        self.models = list(models)
        self.stream = stream or torch.cuda.Stream()  # a created stream: the default one cannot be captured
        arr = (c_void_p * len(self.models))(*[m._h for m in self.models])
        h = c_void_p()
        _check(lib().rmhmc_batch_create(arr, len(self.models), c_void_p(self.stream.cuda_stream),
                                        ctypes.byref(h)))
        self._h = h

    def leapfrog(self, n_steps, integ):
        _check(lib().rmhmc_batch_leapfrog(self._h, ctypes.byref(integ.c()), int(n_steps)))

    def close(self):
        if getattr(self, "_h", None):
            lib().rmhmc_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fp64_peak_tflops(ms_target=200, stream=None):
    """Measured FP64 FMA throughput of the current GPU (TFLOP/s)."""
    import torch
    stream = stream or torch.cuda.current_stream()
    out = c_double()
    _check(lib().rmhmc_fp64_peak(c_void_p(stream.cuda_stream), int(ms_target), ctypes.byref(out)))
    return out.value


def fp32_peak_tflops(ms_target=200, stream=None):
    """Measured FP32 FMA throughput of the current GPU (TFLOP/s)."""
    import torch
    stream = stream or torch.cuda.current_stream()
    out = c_double()
    _check(lib().rmhmc_fp32_peak(c_void_p(stream.cuda_stream), int(ms_target), ctypes.byref(out)))
    return out.value


def df_peak_tflops(ms_target=200, stream=None):
    """Measured double-float (Dot2) multiply-add throughput of the current GPU (TFLOP/s, 2 per step)."""
    import torch
    stream = stream or torch.cuda.current_stream()
    out = c_double()
    _check(lib().rmhmc_df_peak(c_void_p(stream.cuda_stream), int(ms_target), ctypes.byref(out)))
    return out.value


def new_stream():
    """A fresh non-blocking CUDA stream (rmhmc_stream_create) as a torch ExternalStream: unlike
    torch.cuda.Stream(), which takes streams from a pool of 32 in turn, every call gives a distinct
    stream, as a batch of many models needs. Release it with release_stream once its work is done."""
    import torch
    h = c_void_p()
    _check(lib().rmhmc_stream_create(ctypes.byref(h)))
    return torch.cuda.ExternalStream(h.value)


def release_stream(stream):
    """Destroy a stream made by new_stream (its queued work completes first)."""
    _check(lib().rmhmc_stream_destroy(c_void_p(stream.cuda_stream)))


def eigh_noalloc(A, lam=None, Q=None, tol=1e-13, max_sweeps=30, sweeps=None, status=None,
                 stream=None):
    """Batched symmetric eigendecomposition through rmhmc_eigh_noalloc (no device allocation;
    fixed 8 MiB workspace shared by all calls on a device). A: (n, d, d) CUDA float64."""
    import torch
    n, d, _ = A.shape
    stream = stream or torch.cuda.current_stream()
    _check(lib().rmhmc_eigh_noalloc(c_void_p(stream.cuda_stream), int(n), int(d),
                                    _ptr(A, (n, d, d), torch.float64),
                                    _ptr(lam, (n, d), torch.float64), _ptr(Q, (n, d, d), torch.float64),
                                    float(tol), int(max_sweeps), _ptr(sweeps, (n,), torch.int32),
                                    _ptr(status, (n,), torch.int32)))


def gemm_tc(A, B, C=None, ta=False, tb=False, alpha=1.0, beta=0.0, slices=9, sym=False,
            status=None, stream=None):
    """C = alpha op(A) op(B) + beta C through rmhmc_gemm_tc (FP64-accurate GEMM on the tensor
    cores by bf16 slicing). A, B, C: contiguous CUDA float64, (batch, rows, cols) or 2-D; op() is
    the transpose when ta / tb. Returns C (allocated when None)."""
    import torch
    two_d = A.dim() == 2
    A3 = A.unsqueeze(0) if two_d else A
    B3 = B.unsqueeze(0) if B.dim() == 2 else B
    batch = A3.shape[0]
    m, k = (A3.shape[2], A3.shape[1]) if ta else (A3.shape[1], A3.shape[2])
    kb, n = (B3.shape[2], B3.shape[1]) if tb else (B3.shape[1], B3.shape[2])
    if kb != k or B3.shape[0] != batch:
        raise RmhmcError("gemm_tc: shapes do not conform")
    if C is None:
        C = torch.zeros((batch, m, n) if not two_d else (m, n), dtype=torch.float64, device=A.device)
        beta = 0.0
    C3 = C.unsqueeze(0) if C.dim() == 2 else C
    stream = stream or torch.cuda.current_stream()
    _check(lib().rmhmc_gemm_tc(c_void_p(stream.cuda_stream), int(bool(ta)), int(bool(tb)), m, n, k,
                               float(alpha), _ptr(A3, None, torch.float64), A3.shape[2],
                               A3.shape[1] * A3.shape[2], _ptr(B3, None, torch.float64), B3.shape[2],
                               B3.shape[1] * B3.shape[2], float(beta),
                               _ptr(C3, (batch, m, n), torch.float64), n, m * n, batch, int(slices),
                               int(bool(sym)), _ptr(status, (batch,), torch.int32)))
    return C


def test_gemm_stall(entry, wait_ms=20.0):
    """Test switch of the GEMM's bounded waits (rmhmc_test_gemm_stall): entry >= 0 makes later
    tensor-core GEMM launches issue no copy for that batch entry, with every wait limited to
    wait_ms; entry < 0 restores normal operation."""
    _check(lib().rmhmc_test_gemm_stall(int(entry), float(wait_ms)))


JOB_STATES = {0: "queued", 1: "running", 2: "done", 3: "failed"}


class NativeServer:
    """The library's continuous-batching server (rmhmc_server_*): a native scheduler thread admits
    jobs by the HBM budget and runs them concurrently, each on its own model and stream."""

    def __init__(self, hbm_budget_bytes, depth=2, device=0):
        h = c_void_p()
        _check(lib().rmhmc_server_create(int(device), int(hbm_budget_bytes), int(depth), ctypes.byref(h)))
        self._h = h
        self._keep = {}

    def submit(self, problem, n_chains, integ, n_iter, n_burn=0, seed=0, tau=None, q0=None,
               q_out=None, logp_out=None, accept_out=None, status_out=None, loglik_out=None):
        """Queue a job; the output tensors (CUDA, contiguous) must stay alive until it is done."""
        if is_primal(problem):
            desc, keep = _primal_desc(problem)
            model, primal = None, ctypes.pointer(desc)
        else:
            desc, keep = _desc(problem)
            model, primal = ctypes.pointer(desc), None
        t = None if tau is None else np.ascontiguousarray(tau, dtype=np.float64)
        q = None if q0 is None else np.ascontiguousarray(q0, dtype=np.float64)
        jd = JobDesc(model, primal, int(n_chains),
                     t.ctypes.data_as(POINTER(c_double)) if t is not None else None,
                     q.ctypes.data_as(POINTER(c_double)) if q is not None else None,
                     integ.c(), int(n_iter), int(n_burn), int(seed) & (2 ** 64 - 1),
                     _ptr(q_out), _ptr(logp_out), _ptr(accept_out), _ptr(status_out), _ptr(loglik_out))
        jid = c_int()
        _check(lib().rmhmc_server_submit(self._h, ctypes.byref(jd), ctypes.byref(jid)))
        self._keep[jid.value] = (q_out, logp_out, accept_out, status_out, loglik_out)
        return jid.value

    def poll(self, job_id):
        """(state name, job error code, (submitted, admitted, finished) seconds)."""
        st, err, times = c_int(), c_int(), (c_double * 3)()
        _check(lib().rmhmc_server_poll(self._h, int(job_id), ctypes.byref(st), ctypes.byref(err), times))
        return JOB_STATES[st.value], err.value, tuple(times)

    def wait(self, job_id=-1, timeout=-1.0):
        _check(lib().rmhmc_server_wait(self._h, int(job_id), float(timeout)))

    def stats(self):
        now, na, mx, nq, used = c_double(), c_int(), c_int(), c_int(), ctypes.c_size_t()
        _check(lib().rmhmc_server_stats(self._h, ctypes.byref(now), ctypes.byref(na), ctypes.byref(mx),
                                        ctypes.byref(nq), ctypes.byref(used)))
        return {"now": now.value, "active": na.value, "max_active": mx.value, "queued": nq.value,
                "bytes_in_use": used.value}

    def close(self):
        if self._h is not None:
            lib().rmhmc_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def version():
    return lib().rmhmc_version().decode()
