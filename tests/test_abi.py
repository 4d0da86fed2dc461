"""The C ABI library builds, loads and exports every function include/rmhmc.h declares
(no GPU needed: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "rmhmc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rmhmc_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("rmhmc_init_model", "rmhmc_set_state", "rmhmc_leapfrog", "rmhmc_sample",
              "rmhmc_free_model", "rmhmc_dim", "rmhmc_status_string"):
        assert n in names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2511_06407_b300 import build
    path = build.build()
    L = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing
    L.rmhmc_status_string.restype = ctypes.c_char_p
    assert L.rmhmc_status_string(0) == b"ok"
    L.rmhmc_version.restype = ctypes.c_char_p
    assert b"sm_103a" in L.rmhmc_version()


def _prototypes():
    """{name: number of parameters} for every function prototype in include/rmhmc.h."""
    src = open(os.path.join(ROOT, "include", "rmhmc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for name, params in re.findall(r"\b(rmhmc_[a-z_0-9]+)\s*\(([^;{]*?)\)\s*;", src, flags=re.S):
        params = params.strip()
        out[name] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_argtypes_match_header_prototypes():
    """Every function the binding calls declares exactly the header's parameter count (a stale
    binding would pass garbage for the missing arguments)."""
    from paper_2511_06407_b300 import rmhmc
    L = rmhmc.lib()
    protos = _prototypes()
    assert len(protos) >= 14
    for name, n in protos.items():
        fn = getattr(L, name)
        assert fn.argtypes is not None, f"binding does not declare argtypes for {name}"
        assert len(fn.argtypes) == n, (name, len(fn.argtypes), n)


def test_binding_structs_match_header_layout(tmp_path):
    """The ctypes mirrors have the C compiler's sizes and field offsets."""
    import subprocess
    from paper_2511_06407_b300 import rmhmc
    structs = {"rmhmc_kernel_desc": rmhmc.KernelDesc, "rmhmc_model_desc": rmhmc.ModelDesc,
               "rmhmc_integrator": rmhmc.IntegratorC, "rmhmc_primal_desc": rmhmc.PrimalDesc,
               "rmhmc_job_desc": rmhmc.JobDesc}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rmhmc.h"', "int main(void){"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    for line in filter(None, out):
        cname, field, val = line.split()
        py = structs[cname]
        got = ctypes.sizeof(py) if field == "size" else getattr(py, field).offset
        assert got == int(val), (cname, field, got, val)


def test_invalid_descriptions_are_rejected_without_a_gpu():
    from paper_2511_06407_b300 import rmhmc
    L = rmhmc.lib()
    out = ctypes.c_void_p()
    # N = 0 is rejected before any device call
    desc = rmhmc.ModelDesc()
    desc.N = 0
    assert L.rmhmc_init_model(ctypes.byref(desc), 1, None, None, ctypes.byref(out)) == 1
    assert L.rmhmc_init_model(None, 1, None, None, ctypes.byref(out)) == 1
    # the primal model: no covariates, then too many features (d > 4096), then a bad prior
    pd = rmhmc.PrimalDesc()
    pd.N = 10
    assert L.rmhmc_init_primal(ctypes.byref(pd), 1, None, None, ctypes.byref(out)) == 1
    y = (ctypes.c_double * 10)()
    xg = (ctypes.c_double * 10)()
    pd.y, pd.Xg, pd.n_gauss, pd.M, pd.L, pd.bias_var, pd.J = y, xg, 1, 5000, 8.0, 1.0, 1
    pd.prior_a[:] = [2.0, 2.0, 2.0]
    pd.prior_b[:] = [2.0, 2.0, 2.0]
    size = ctypes.c_size_t()
    assert L.rmhmc_plan_bytes_primal(ctypes.byref(pd), 1, ctypes.byref(size)) == 1
    pd.M = 30
    assert L.rmhmc_plan_bytes_primal(ctypes.byref(pd), 2, ctypes.byref(size)) == 0 and size.value > 0
    pd.J = 2  # the mean/variance model needs its own likelihood
    assert L.rmhmc_plan_bytes_primal(ctypes.byref(pd), 2, ctypes.byref(size)) == 1
    pd.lik, pd.delta = 2, 0.05
    assert L.rmhmc_plan_bytes_primal(ctypes.byref(pd), 2, ctypes.byref(size)) == 0
    pd.prior_b[1] = 0.0
    assert L.rmhmc_plan_bytes_primal(ctypes.byref(pd), 2, ctypes.byref(size)) == 1


def test_binding_rejects_kernels_with_too_many_columns():
    import pytest
    from paper_2511_06407_b300 import rmhmc, workloads as wl
    prob = wl.gp_classification(8, seed=0)
    prob["kernels"][0]["cols"] = list(range(rmhmc.MAX_COLS + 1))
    with pytest.raises(rmhmc.RmhmcError):
        rmhmc._desc(prob)
    prob["kernels"][0]["cols"] = []
    with pytest.raises(rmhmc.RmhmcError):
        rmhmc._desc(prob)


def test_server_is_refused_cleanly_without_a_gpu():
    """rmhmc_server_create validates the device before starting its scheduler thread: on a host
    without a CUDA device it returns EINVAL (raised by the binding), nothing is left running."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    from paper_2511_06407_b300 import build, rmhmc
    build.build()
    with pytest.raises(rmhmc.RmhmcError):
        rmhmc.NativeServer(2**20)
