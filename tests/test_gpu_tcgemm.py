"""rmhmc_gemm_tc (FP64-accurate GEMM on the tensor cores by bf16 slicing) against exact products.

The reference is the exact dot product, computed on the CPU by error-free transformations (each
a_il b_lj as the unevaluated sum of its rounded product and Dekker's exact error term, summed
with math.fsum, which is correctly rounded): a plain definition, independent of the slicing.

Bound (slices S, per output (i, j), with 2^eA_i >= max |row i of op(A)| and 2^eB_j likewise):
|C - C_exact| <= 2^-52 |C_exact| + 8 k 2^(eA_i + eB_j - 7S): the slice representation
(2^-7S per product), the dropped slice pairs ((S - 1) 2^(-7S - 2)) and the rounding of the shared
accumulator of the highest groups, with margin."""
import math

import numpy as np
import pytest

from paper_2511_06407_b300 import rmhmc

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _two_prod(a, b):
    """p + e == a * b exactly (Dekker / Veltkamp splitting; no overflow for these inputs)."""
    f = 134217729.0  # 2^27 + 1
    ca, cb = f * a, f * b
    ah = ca - (ca - a)
    al = a - ah
    bh = cb - (cb - b)
    bl = b - bh
    p = a * b
    e = ((ah * bh - p) + ah * bl + al * bh) + al * bl
    return p, e


def exact_matmul(A, B):
    """Correctly rounded (A @ B)_ij for 2-D float64 arrays."""
    m, k = A.shape
    n = B.shape[1]
    out = np.empty((m, n))
    for i in range(m):
        p, e = _two_prod(A[i][:, None], B)  # k x n
        for j in range(n):
            out[i, j] = math.fsum(np.concatenate([p[:, j], e[:, j]]))
    return out


def op(X, t):
    return np.swapaxes(X, -1, -2) if t else X


def exponents(X, axis):
    mx = np.abs(X).max(axis=axis)
    return np.where(mx > 0, np.frexp(mx)[1], 0)


def make(shape, rng, scale_axis=None, spread=20):
    X = rng.standard_normal(shape)
    if scale_axis is not None:
        sh = [1] * len(shape)
        sh[scale_axis] = shape[scale_axis]
        X *= 2.0 ** rng.integers(-spread, spread + 1, size=shape[scale_axis]).reshape(sh)
    return X


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("ta,tb", [(False, False), (False, True), (True, False), (True, True)])
def test_integer_products_are_exact(ta, tb):
    """Integer inputs whose products and sums are exact in FP64: the result must be bit-exact
    (2 tiles plus a ragged tail in every dimension, batch 3)."""
    rng = np.random.default_rng(1)
    b, m, n, k = 3, 200, 150, 300
    A = rng.integers(-1000, 1001, size=(b, m, k)).astype(np.float64)
    B = rng.integers(-1000, 1001, size=(b, k, n)).astype(np.float64)
    C = rmhmc.gemm_tc(cuda(op(A, ta)), cuda(op(B, tb)), ta=ta, tb=tb).cpu().numpy()
    want = np.einsum("bik,bkj->bij", A.astype(np.int64), B.astype(np.int64)).astype(np.float64)
    np.testing.assert_array_equal(C, want)


@pytest.mark.parametrize("slices", [7, 8, 9])
@pytest.mark.parametrize("ta,tb", [(False, False), (True, True)])
def test_random_products_within_the_slicing_bound(slices, ta, tb):
    """Rows of A and columns of B scaled by 2^U{-20..20}: wide dynamic range between rows, the
    case that row-wise exponents must handle."""
    rng = np.random.default_rng(2 + slices)
    m, n, k = 160, 100, 200
    A = make((m, k), rng, 0)
    B = make((k, n), rng, 1)
    C = rmhmc.gemm_tc(cuda(op(A, ta)), cuda(op(B, tb)), ta=ta, tb=tb, slices=slices).cpu().numpy()
    ref = exact_matmul(A, B)
    eA, eB = exponents(A, 1), exponents(B, 0)
    bound = 2.0 ** -52 * np.abs(ref) + 8 * k * np.ldexp(1.0, eA[:, None] + eB[None, :] - 7 * slices)
    err = np.abs(C - ref)
    assert np.all(err <= bound), float((err / bound).max())
    if slices == 9:  # at this width the slicing error is below FP64 GEMM rounding
        fp64 = np.abs(A @ B - ref)
        assert err.max() <= max(4 * fp64.max(), 2.0 ** -52 * np.abs(ref).max())


def test_long_k_runs_in_exact_chunks_and_honours_beta():
    """k = 700 needs two launches (at most 512 per launch for exact group sums); beta != 0."""
    rng = np.random.default_rng(5)
    b, m, n, k = 2, 130, 70, 700
    A = make((b, m, k), rng)
    B = make((b, k, n), rng)
    C0 = rng.standard_normal((b, m, n))
    C = rmhmc.gemm_tc(cuda(A), cuda(B), C=cuda(C0), alpha=0.75, beta=-0.5, slices=9).cpu().numpy()
    for i in range(b):
        ref = exact_matmul(A[i], B[i])
        want = 0.75 * ref - 0.5 * C0[i]
        tol = 2.0 ** -50 * (np.abs(0.75 * ref) + np.abs(0.5 * C0[i])) + \
            8 * k * np.ldexp(1.0, exponents(A[i], 1)[:, None] + exponents(B[i], 0)[None, :] - 63)
        assert np.all(np.abs(C[i] - want) <= tol)


def test_symmetric_product_is_exactly_symmetric():
    """sym: A A^T computed on the lower triangle and mirrored (tiles above the diagonal skipped)."""
    rng = np.random.default_rng(6)
    b, m, k = 2, 300, 180
    A = make((b, m, k), rng, 1, spread=6)
    At = cuda(A)
    C = rmhmc.gemm_tc(At, At, tb=True, sym=True).cpu().numpy()
    full = rmhmc.gemm_tc(At, At, tb=True).cpu().numpy()
    np.testing.assert_array_equal(C, np.swapaxes(C, 1, 2))
    lower = np.tril(np.ones((m, m), dtype=bool))
    np.testing.assert_array_equal(C[:, lower], full[:, lower])
    ref = exact_matmul(A[0], A[0].T)
    assert np.abs(C[0] - ref).max() <= 2.0 ** -50 * np.abs(ref).max() * k


def test_non_finite_rows_give_nan_rows_and_edge_sizes():
    rng = np.random.default_rng(7)
    m, n, k = 70, 90, 33
    A = make((m, k), rng)
    B = make((k, n), rng)
    A[3, 5] = np.inf
    B[7, 11] = np.nan
    C = rmhmc.gemm_tc(cuda(A), cuda(B)).cpu().numpy()
    assert np.isnan(C[3]).all() and np.isnan(C[:, 11]).all()
    keep = np.ones((m, n), dtype=bool)
    keep[3] = False
    keep[:, 11] = False
    Af, Bf = A.copy(), B.copy()
    Af[3] = 0
    Bf[:, 11] = 0
    ref = exact_matmul(Af, Bf)
    assert np.abs(C[keep] - ref[keep]).max() <= 2.0 ** -50 * np.abs(ref).max() * k
    # k = 0: C = beta C; one-element products
    C0 = torch.ones((4, 5), dtype=torch.float64, device="cuda")
    out = rmhmc.gemm_tc(torch.zeros((4, 0), dtype=torch.float64, device="cuda"),
                        torch.zeros((0, 5), dtype=torch.float64, device="cuda"), C=C0, beta=2.0)
    assert torch.all(out == 2.0)
    one = rmhmc.gemm_tc(cuda(np.array([[1.5]])), cuda(np.array([[-0.1]]))).item()
    assert abs(one - 1.5 * -0.1) <= np.spacing(0.15)


def test_status_clear_and_bad_arguments_rejected():
    rng = np.random.default_rng(8)
    A = cuda(make((2, 64, 48), rng))
    B = cuda(make((2, 48, 64), rng))
    st = torch.zeros(2, dtype=torch.int32, device="cuda")
    rmhmc.gemm_tc(A, B, status=st)
    torch.cuda.synchronize()
    assert st.tolist() == [0, 0]
    with pytest.raises(rmhmc.RmhmcError):
        rmhmc.gemm_tc(A, B, slices=5)
    with pytest.raises(rmhmc.RmhmcError):
        rmhmc.gemm_tc(A, cuda(make((2, 48, 40), rng)), sym=True)


def test_bounded_wait_runs_out_and_the_context_stays_usable():
    """Failure detection without a GPU fault. The test switch makes the GEMM issue no copy for
    batch entry 1, so that entry's first pipeline wait finds nothing to wait for and runs out
    after 20 ms: the call returns, entry 1 is marked RMHMC_CHAIN_TIMEOUT and filled with NaN, the
    other entries are exact, and the next normal call on the same context is correct."""
    rng = np.random.default_rng(12)
    A = cuda(make((3, 200, 96), rng))
    B = cuda(make((3, 96, 130), rng))
    ref = rmhmc.gemm_tc(A, B, slices=9)
    st = torch.zeros(3, dtype=torch.int32, device="cuda")
    rmhmc.test_gemm_stall(1, 20.0)
    try:
        out = rmhmc.gemm_tc(A, B, slices=9, status=st)
        torch.cuda.synchronize()
    finally:
        rmhmc.test_gemm_stall(-1)
    assert st.tolist() == [0, rmhmc.CHAIN_TIMEOUT, 0]
    assert torch.isnan(out[1]).all()
    assert torch.equal(out[0], ref[0]) and torch.equal(out[2], ref[2])
    st2 = torch.zeros(3, dtype=torch.int32, device="cuda")
    out2 = rmhmc.gemm_tc(A, B, slices=9, status=st2)
    torch.cuda.synchronize()
    assert st2.tolist() == [0, 0, 0]
    assert torch.equal(out2, ref)
    with pytest.raises(rmhmc.RmhmcError):
        rmhmc.test_gemm_stall(0, 0.0)  # a limit outside 1..2000 ms is refused
