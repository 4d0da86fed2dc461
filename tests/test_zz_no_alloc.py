"""rmhmc_eigh_noalloc: the allocation-free eigendecomposition entry point.

Some callers cannot allocate device memory: code running inside another framework's pooled or
arena allocator, plug-ins whose host forbids cudaMalloc, or loops that must never reach the
allocator. For them the library offers this one entry point, whose workspace is a fixed device
array inside the library. This file checks it against the existing path (rmhmc_set_state's
cold-start Jacobi, read back through rmhmc_geometry) on two calls in a row, within the
eigenvalue tolerance the other parity tests use (1e-10 normwise on the sorted eigenvalues). It is
named to run after every other test file.
"""
import ctypes

import numpy as np
import pytest

from paper_2511_06407_b300 import workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rm():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2511_06407_b300 import build, rmhmc
    build.build()
    return rmhmc


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def test_noalloc_eigh_matches_existing_entry_point_twice(rm):
    prob = wl.gp_classification(50, seed=0)
    C = 3
    model = rm.Model(prob, C)
    d = model.d
    Q0 = wl.random_state(prob, C, seed=21, f_scale=0.3, u_scale=0.2)
    model.set_state(torch.tensor(Q0, device="cuda"), integ=rm.Integrator())
    H = torch.empty(C, d, d, dtype=torch.float64, device="cuda")
    lam_ref = torch.empty(C, d, dtype=torch.float64, device="cuda")
    model.geometry(hess=H, lam=lam_ref)
    torch.cuda.synchronize()
    lam_ref = np.sort(lam_ref.cpu().numpy(), axis=1)
    Hn = H.cpu().numpy()
    outs = []
    for call in range(2):
        lam = torch.full((C, d), np.nan, dtype=torch.float64, device="cuda")
        Q = torch.full((C, d, d), np.nan, dtype=torch.float64, device="cuda")
        sw = torch.empty(C, dtype=torch.int32, device="cuda")
        st = torch.full((C,), -1, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        rm.eigh_noalloc(H, lam, Q, tol=1e-13, max_sweeps=30, sweeps=sw, status=st)
        torch.cuda.synchronize()
        if call == 1:
            # after the first call (which may load the module that holds the fixed array) the
            # entry point takes no device memory at all
            assert torch.cuda.mem_get_info()[0] == free_before
        lam, Q, st = lam.cpu().numpy(), Q.cpu().numpy(), st.cpu().numpy()
        assert np.all(st == 0), st
        for c in range(C):
            assert rel(np.sort(lam[c]), lam_ref[c]) < 1e-10, (call, c)
            assert np.abs(Q[c].T @ Q[c] - np.eye(d)).max() < 1e-10
            res = Hn[c] @ Q[c] - Q[c] * lam[c]
            assert np.linalg.norm(res) <= 1e-10 * np.linalg.norm(Hn[c])
        outs.append((lam, Q))
    # the second call sees the first call's leftovers in the workspace and gives the same answer
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])
    model.close()


def test_noalloc_eigh_rejects_batches_beyond_its_workspace(rm):
    L = rm.lib()
    A = torch.zeros(1, 1, 1, dtype=torch.float64, device="cuda")
    # d = 800 (padded 800) needs 2 * 800^2 doubles > 1,048,576: rejected before any launch
    rc = L.rmhmc_eigh_noalloc(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), 1, 800,
                              ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(A.data_ptr()), None,
                              1e-13, 30, None, None)
    assert rc == 9  # RMHMC_ESCRATCH
    assert b"workspace" in L.rmhmc_status_string(rc)
