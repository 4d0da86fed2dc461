"""Oracle evaluations in spawned worker processes with single-threaded BLAS (test infrastructure).

On hosts with many cores, OpenBLAS's threaded kernels were seen to stall for tens of minutes on the
small matrices of the N = 50 problem (a sampler run that takes 20 s with one BLAS thread). The
workers here import numpy with one BLAS thread (the thread-count variables are set before the
pool starts and restored after), and independent oracle evaluations of a test run side by side.
The pool is started with `spawn`, never forked from a process that has used the GPU.
"""
import multiprocessing as mp
import os
from concurrent.futures import ProcessPoolExecutor

_THREAD_VARS = ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")


def run(fn, jobs, max_workers=8):
    """[fn(job) for job in jobs], computed in spawned single-BLAS-thread worker processes."""
    jobs = list(jobs)
    if not jobs:
        return []
    saved = {v: os.environ.get(v) for v in _THREAD_VARS}
    for v in _THREAD_VARS:
        os.environ[v] = "1"
    try:
        workers = max(1, min(len(jobs), max_workers, os.cpu_count() or 1))
        with ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
            return list(ex.map(fn, jobs))
    finally:
        for v, x in saved.items():
            if x is None:
                os.environ.pop(v, None)
            else:
                os.environ[v] = x


def _model(problem):
    if problem.get("model") == "primal":
        from oracle.primal import from_problem
    else:
        from oracle.model import from_problem
    return from_problem(problem)


def sample_job(job):
    """job = (problem, inverse method 'lu' / 'cholesky', keyword arguments of oracle.sampler.sample
    except the model and q0, which is f = 0, u = 0[, eigen driver 'evd' / 'ev'])."""
    import numpy as np
    from oracle import model as mdl
    from oracle.geometry import eigen_driver
    from oracle.sampler import sample
    problem, method, kw = job[:3]
    driver = job[3] if len(job) > 3 else "evd"
    m = _model(problem)
    with mdl.inverse_method(method), eigen_driver(driver):
        return sample(m, np.zeros(m.d), **kw)


def quantities_job(job):
    """job = (problem, q, tau, p or None, inverse method, eigen driver): the geometric quantities
    the parity tests compare (U, dU, H, lam, G; with p also dH/dq, G^-1 p and H(q, p))."""
    from oracle import model as mdl
    from oracle.geometry import Geometry, eigen_driver
    problem, q, tau, p, method, driver = job
    m = _model(problem)
    with mdl.inverse_method(method), eigen_driver(driver):
        geo = Geometry(m, q, tau, 1e6, "coth", with_third=p is not None)
        out = {"U": geo.U, "dU": geo.dU, "H": geo.H, "lam": geo.lam, "G": geo.G()}
        if p is not None:
            out.update(dHdq=geo.dHdq(p), Ginv_p=geo.Ginv_p(p), Ham=geo.hamiltonian(p))
    return out
