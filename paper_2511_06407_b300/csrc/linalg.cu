// Batched FP64 dense linear algebra for the plain-FP64 path: GEMM, Cholesky, triangular inverse,
// GEMV. On B300 the FP64 pipe (about 1.1 TFLOP/s for the whole GPU, 1/64 of FP32) bounds all of
// these; the kernels keep every SM's FP64 units fed with many independent CTAs and modest tiles
// rather than chasing memory bandwidth.
#include <math.h>

#include "internal.cuh"

namespace rmhmc {

namespace {

constexpr int BM = 64, BN = 64, BK = 16, GT = 256;

// C = alpha op(A) op(B) + beta C for one 64 x 64 tile per CTA; thread (ty, tx) owns rows
// ty + 16 i and columns tx + 16 j (i, j < 4) so shared-memory reads are conflict-free.
template <bool TA, bool TB>
__global__ void __launch_bounds__(GT) k_gemm(int m, int n, int k, double alpha,
                                             const double* __restrict__ A, int lda, long long sA,
                                             const double* __restrict__ B, int ldb, long long sB,
                                             double beta, double* __restrict__ C, int ldc,
                                             long long sC, int sym, int tri) {
  const int tm = blockIdx.y, tn = blockIdx.x, b = blockIdx.z;
  if (sym && tn > tm) return;
  A += b * sA;
  B += b * sB;
  C += b * sC;
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
  const int row0 = tm * BM, col0 = tn * BN;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  int kbeg = 0;
  if (tri) kbeg = (max(row0, col0) / BK) * BK;
  for (int k0 = kbeg; k0 < k; k0 += BK) {
#pragma unroll
    for (int e = tid; e < BM * BK; e += GT) {
      int mm, kk;
      if (TA) { kk = e / BM; mm = e % BM; } else { mm = e / BK; kk = e % BK; }
      const int gr = row0 + mm, gk = k0 + kk;
      double v = 0.0;
      if (gr < m && gk < k) v = TA ? A[(long long)gk * lda + gr] : A[(long long)gr * lda + gk];
      As[kk][mm] = v;
    }
#pragma unroll
    for (int e = tid; e < BN * BK; e += GT) {
      int kk, nn;
      if (TB) { nn = e / BK; kk = e % BK; } else { kk = e / BN; nn = e % BN; }
      const int gk = k0 + kk, gc = col0 + nn;
      double v = 0.0;
      if (gk < k && gc < n) v = TB ? B[(long long)gc * ldb + gk] : B[(long long)gk * ldb + gc];
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = row0 + ty + 16 * i;
    if (r >= m) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = col0 + tx + 16 * j;
      if (c >= n) continue;
      if (sym) {
        // the lower element (r >= c) is read and written here, its mirror only written: C must
        // be symmetric on entry when beta != 0 (every lower element belongs to one CTA)
        if (tm == tn && c > r) continue;
        const long long o = (long long)r * ldc + c;
        const double v = alpha * acc[i][j] + (beta != 0.0 ? beta * C[o] : 0.0);
        C[o] = v;
        if (c != r) C[(long long)c * ldc + r] = v;
      } else {
        const long long o = (long long)r * ldc + c;
        C[o] = alpha * acc[i][j] + (beta != 0.0 ? beta * C[o] : 0.0);
      }
    }
  }
}

constexpr int CB = 32;  // Cholesky / triangular-inverse block

// In-place right-looking blocked Cholesky (lower) of one N x N matrix per CTA (small N); the strict
// upper triangle is zeroed. A pivot that is not positive marks the chain and is replaced by 1 so
// that the factor stays finite. Larger N: panel steps (k_chol_diag + k_chol_rows) with the
// trailing update A22 -= L21 L21^T between them as a batched symmetric GEMM over all matrices (so
// every SM takes part).
// The panel step split for parallelism. k_chol_diag: one CTA of 128 threads per matrix factors the
// kb x kb diagonal block at (k0, k0) in shared memory (right-looking; each column's trailing update
// spread over the four warps, so four FP64 pipes of the SM share it), writes it back with zeros
// above its diagonal, keeps the reciprocal pivots in rdiag (kb per matrix) and adds its share of
// log|A|. The pivot's reciprocal square root comes from the FP32 one refined by two FP64 Newton
// steps and the root from one more (FP64 square root and division are long multi-instruction
// sequences on this part); pivots outside [1e-30, 1e30] take the FP64 square root and division.
__global__ void __launch_bounds__(128) k_chol_diag(double* __restrict__ Ab, int N, int k0,
                                                  double* __restrict__ rdiag,
                                                  double* __restrict__ logdet, int lds,
                                                  int* __restrict__ status, int per_chain) {
  const int b = blockIdx.x, tid = threadIdx.x;
  double* A = Ab + (long long)b * N * N;
  const int kb = min(CB, N - k0);
  __shared__ double Dk[CB][CB + 1];
  __shared__ double sir;
  for (int e = tid; e < kb * kb; e += blockDim.x) Dk[e / kb][e % kb] = A[(long long)(k0 + e / kb) * N + k0 + e % kb];
  __syncthreads();
  bool bad = false;
  double pm = 1.0;  // product of the pivots' square roots as pm 2^pe (one log at the end)
  int pe = 0;
  for (int j = 0; j < kb; ++j) {
    if (tid == 0) {
      double piv = Dk[j][j];
      if (!(piv > 0.0) || !isfinite(piv)) { bad = true; piv = 1.0; }
      double r, y;
      if (piv > 1e-30 && piv < 1e30) {
        y = (double)rsqrtf((float)piv);
        y = y * fma(-0.5 * piv, y * y, 1.5);
        y = y * fma(-0.5 * piv, y * y, 1.5);
        r = piv * y;
        r = fma(0.5 * y, fma(-r, r, piv), r);
      } else {
        r = sqrt(piv);
        y = 1.0 / r;
      }
      Dk[j][j] = r;
      sir = y;
      rdiag[(long long)b * CB + j] = y;
      int ex;
      pm = frexp(pm * r, &ex);
      pe += ex;
    }
    __syncthreads();
    const double ir = sir;
    if (tid > j && tid < kb) Dk[tid][j] *= ir;
    __syncthreads();
    // trailing lower triangle (i, l), j < l <= i < kb, as a flat index over 128 threads
    const int m = kb - j - 1, cnt = m * (m + 1) / 2;
    for (int e = tid; e < cnt; e += blockDim.x) {
      int i = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
      while ((i + 1) * (i + 2) / 2 <= e) ++i;
      while (i * (i + 1) / 2 > e) --i;
      const int gi = j + 1 + i, gl = j + 1 + (e - i * (i + 1) / 2);
      Dk[gi][gl] -= Dk[gi][j] * Dk[gl][j];
    }
    __syncthreads();
  }
  for (int e = tid; e < kb * kb; e += blockDim.x) {
    const int i = e / kb, j = e % kb;
    A[(long long)(k0 + i) * N + k0 + j] = (j <= i) ? Dk[i][j] : 0.0;
  }
  if (tid == 0) {
    const double ldacc = log(pm) + pe * 0.69314718055994530942;  // log of the product of the roots
    double* ldp = logdet + (long long)b * lds;
    *ldp = (k0 == 0 ? 0.0 : *ldp) + 2.0 * ldacc;
    if (bad) atomicOr(&status[b / per_chain], RMHMC_CHAIN_NOTPD);
  }
}

// L21 = A21 L11^-T for the rows below the diagonal block: one thread per row, the substitution
// unrolled over the 32 columns with the row in registers; grid (row blocks of 128, matrices).
template <int KB>
__global__ void __launch_bounds__(128) k_chol_rows(double* __restrict__ Ab, int N, int k0,
                                                  const double* __restrict__ rdiag) {
  const int b = blockIdx.y;
  double* A = Ab + (long long)b * N * N;
  __shared__ double Lk[KB][KB + 1];
  __shared__ double rd[KB];
  for (int e = threadIdx.x; e < KB * KB; e += blockDim.x)
    Lk[e / KB][e % KB] = A[(long long)(k0 + e / KB) * N + k0 + e % KB];
  if (threadIdx.x < KB) rd[threadIdx.x] = rdiag[(long long)b * CB + threadIdx.x];
  __syncthreads();
  const int i = k0 + KB + blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double* row = A + (long long)i * N + k0;
  double x[KB];
#pragma unroll
  for (int j = 0; j < KB; ++j) x[j] = row[j];
#pragma unroll
  for (int j = 0; j < KB; ++j) {
    double v = x[j];
#pragma unroll
    for (int p = 0; p < j; ++p) v = fma(-x[p], Lk[j][p], v);
    x[j] = v * rd[j];
  }
#pragma unroll
  for (int j = 0; j < KB; ++j) row[j] = x[j];
}

__global__ void __launch_bounds__(256) k_chol(double* __restrict__ Ab, int N,
                                             double* __restrict__ logdet, int lds,
                                             int* __restrict__ status, int per_chain) {
  const int b = blockIdx.x;
  double* A = Ab + (long long)b * N * N;
  __shared__ double Dk[CB][CB + 1];
  __shared__ double Pi[CB][CB + 1];
  __shared__ double Pl[CB][CB + 1];
  __shared__ int bad;
  __shared__ double ldacc;
  const int tid = threadIdx.x;
  if (tid == 0) { bad = 0; ldacc = 0.0; }
  __syncthreads();
  for (int k0 = 0; k0 < N; k0 += CB) {
    const int kb = min(CB, N - k0);
    for (int e = tid; e < kb * kb; e += blockDim.x) {
      const int i = e / kb, j = e % kb;
      Dk[i][j] = A[(long long)(k0 + i) * N + k0 + j];
    }
    __syncthreads();
    for (int j = 0; j < kb; ++j) {
      if (tid == 0) {
        double piv = Dk[j][j];
        if (!(piv > 0.0) || !isfinite(piv)) { bad = 1; piv = 1.0; }
        const double r = sqrt(piv);
        Dk[j][j] = r;
        ldacc += log(r);
      }
      __syncthreads();
      for (int i = j + 1 + tid; i < kb; i += blockDim.x) Dk[i][j] /= Dk[j][j];
      __syncthreads();
      const int rem = kb - j - 1;
      for (int e = tid; e < rem * rem; e += blockDim.x) {
        const int i = j + 1 + e / rem, l = j + 1 + e % rem;
        if (l <= i) Dk[i][l] -= Dk[i][j] * Dk[l][j];
      }
      __syncthreads();
    }
    for (int e = tid; e < kb * kb; e += blockDim.x) {
      const int i = e / kb, j = e % kb;
      A[(long long)(k0 + i) * N + k0 + j] = (j <= i) ? Dk[i][j] : 0.0;
    }
    __syncthreads();
    // panel: L21 = A21 L11^-T, one row per thread
    for (int i = k0 + kb + tid; i < N; i += blockDim.x) {
      double x[CB];
      for (int j = 0; j < kb; ++j) {
        double v = A[(long long)i * N + k0 + j];
        for (int p = 0; p < j; ++p) v -= x[p] * Dk[j][p];
        x[j] = v / Dk[j][j];
      }
      for (int j = 0; j < kb; ++j) A[(long long)i * N + k0 + j] = x[j];
    }
    __syncthreads();
    // trailing update of the lower triangle: A22 -= L21 L21^T, in 32 x 32 tiles
    const int t0 = k0 + kb;
    const int nt = (N - t0 + CB - 1) / CB;
    for (int ti = 0; ti < nt; ++ti) {
      const int r0 = t0 + ti * CB;
      const int rn = min(CB, N - r0);
      for (int e = tid; e < CB * kb; e += blockDim.x) {
        const int i = e / kb, p = e % kb;
        Pi[i][p] = (i < rn) ? A[(long long)(r0 + i) * N + k0 + p] : 0.0;
      }
      for (int tl = 0; tl <= ti; ++tl) {
        const int c0 = t0 + tl * CB;
        const int cn = min(CB, N - c0);
        for (int e = tid; e < CB * kb; e += blockDim.x) {
          const int i = e / kb, p = e % kb;
          Pl[i][p] = (i < cn) ? A[(long long)(c0 + i) * N + k0 + p] : 0.0;
        }
        __syncthreads();
        for (int e = tid; e < CB * CB; e += blockDim.x) {
          const int i = e / CB, l = e % CB;
          if (i < rn && l < cn && (ti != tl || l <= i)) {
            double s = 0.0;
            for (int p = 0; p < kb; ++p) s = fma(Pi[i][p], Pl[l][p], s);
            A[(long long)(r0 + i) * N + c0 + l] -= s;
          }
        }
        __syncthreads();
      }
    }
    __syncthreads();
  }
  // zero the strict upper triangle (the factor is used as a plain lower-triangular matrix)
  for (long long e = tid; e < (long long)N * N; e += blockDim.x) {
    const int i = (int)(e / N), j = (int)(e % N);
    if (j > i) A[e] = 0.0;
  }
  if (tid == 0) {
    logdet[(long long)b * lds] = 2.0 * ldacc;
    if (bad) atomicOr(&status[b / per_chain], RMHMC_CHAIN_NOTPD);
  }
}

// X = L^-1 for the lower-triangular diagonal block L[o:o+N, o:o+N] of an ld x ld matrix (o = 0,
// N = ld: the whole matrix): one CTA per (32-column tile, matrix). Column tile c0 of X is zero above
// row c0; each 32-row block below is a small GEMM against the rows already solved followed by
// forward substitution with the diagonal block.
__global__ void __launch_bounds__(256) k_trinv(const double* __restrict__ Lb,
                                              double* __restrict__ Xb, int N, int ld, int o) {
  const int ct = blockIdx.x, b = blockIdx.y;
  const double* L = Lb + (long long)b * ld * ld + (long long)o * ld + o;
  double* X = Xb + (long long)b * ld * ld + (long long)o * ld + o;
  const int c0 = ct * CB;
  const int cn = min(CB, N - c0);
  __shared__ double Ls[CB][CB + 1];
  __shared__ double Xs[CB][CB + 1];
  __shared__ double R[CB][CB + 1];
  __shared__ double rdg[CB];
  const int tid = threadIdx.x;
  for (int r = tid; r < c0; r += blockDim.x)
    for (int j = 0; j < cn; ++j) X[(long long)r * ld + c0 + j] = 0.0;
  for (int r0 = c0; r0 < N; r0 += CB) {
    const int rn = min(CB, N - r0);
    for (int e = tid; e < CB * CB; e += blockDim.x) {
      const int i = e / CB, j = e % CB;
      R[i][j] = (i < rn && j < cn && r0 + i == c0 + j) ? 1.0 : 0.0;
    }
    for (int p0 = c0; p0 < r0; p0 += CB) {
      __syncthreads();
      for (int e = tid; e < CB * CB; e += blockDim.x) {
        const int i = e / CB, j = e % CB;
        Ls[i][j] = (i < rn) ? L[(long long)(r0 + i) * ld + p0 + j] : 0.0;
        Xs[i][j] = (j < cn) ? X[(long long)(p0 + i) * ld + c0 + j] : 0.0;
      }
      __syncthreads();
      for (int e = tid; e < CB * CB; e += blockDim.x) {
        const int i = e / CB, j = e % CB;
        double s = 0.0;
#pragma unroll 8
        for (int p = 0; p < CB; ++p) s = fma(Ls[i][p], Xs[p][j], s);
        R[i][j] -= s;
      }
    }
    __syncthreads();
    for (int e = tid; e < CB * CB; e += blockDim.x) {
      const int i = e / CB, j = e % CB;
      Ls[i][j] = (i < rn && j < rn) ? L[(long long)(r0 + i) * ld + r0 + j] : (i == j ? 1.0 : 0.0);
    }
    __syncthreads();
    if (tid < CB) rdg[tid] = 1.0 / Ls[tid][tid];  // the block's reciprocal pivots, in parallel
    __syncthreads();
    if (tid < CB) {
      const int j = tid;
      for (int i = 0; i < rn; ++i) {
        double v = R[i][j];
        for (int p = 0; p < i; ++p) v = fma(-Ls[i][p], R[p][j], v);
        R[i][j] = v * rdg[i];
      }
    }
    __syncthreads();
    for (int e = tid; e < rn * cn; e += blockDim.x) {
      const int i = e / cn, j = e % cn;
      X[(long long)(r0 + i) * ld + c0 + j] = R[i][j];
    }
    __syncthreads();
  }
}

// y = alpha A x + beta y (warp per row) and y = alpha A^T x + beta y (thread per column).
__global__ void k_gemv_n(int rows, int cols, const double* __restrict__ A, int lda, long long sA,
                         const double* __restrict__ x, long long sx, double* __restrict__ y,
                         long long sy, double alpha, double beta) {
  const int b = blockIdx.y;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= rows) return;
  const double* a = A + b * sA + (long long)warp * lda;
  const double* xv = x + b * sx;
  double s = 0.0;
  for (int j = lane; j < cols; j += 32) s = fma(a[j], xv[j], s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    double* o = y + b * sy + warp;
    *o = alpha * s + (beta != 0.0 ? beta * *o : 0.0);
  }
}

__global__ void k_gemv_t(int rows, int cols, const double* __restrict__ A, int lda, long long sA,
                         const double* __restrict__ x, long long sx, double* __restrict__ y,
                         long long sy, double alpha, double beta) {
  const int b = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= cols) return;
  const double* a = A + b * sA;
  const double* xv = x + b * sx;
  double s = 0.0;
  for (int i = 0; i < rows; ++i) s = fma(a[(long long)i * lda + j], xv[i], s);
  double* o = y + b * sy + j;
  *o = alpha * s + (beta != 0.0 ? beta * *o : 0.0);
}

// Solve L t = f then L^T a = t for one lower-triangular N x N factor per CTA (blocked substitution,
// backward stable, unlike multiplying by an explicit inverse). Per 32-row block: the already solved
// part is subtracted with coalesced dot products over all warps (forward: a warp per row, lanes
// along the row; backward: lanes along a row segment of L, warps over the rows below, combined in
// shared memory), then warp 0 finishes the 32 x 32 triangle column by column (lane = row: one
// shuffle and one FMA per step) with the reciprocal pivots computed once up front.
__global__ void __launch_bounds__(1024) k_cholsolve(const double* __restrict__ Lb,
                                                  const double* __restrict__ fb,
                                                  double* __restrict__ tb, double* __restrict__ ab,
                                                  int N) {
  const int b = blockIdx.x;
  const double* L = Lb + (long long)b * N * N;
  const double* f = fb + (long long)b * N;
  double* t = tb + (long long)b * N;
  double* a = ab + (long long)b * N;
  extern __shared__ double x[];  // N solution, then N reciprocal pivots
  double* rd = x + N;
  __shared__ double rhs[CB];
  __shared__ double part[32][CB];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int i = threadIdx.x; i < N; i += blockDim.x) rd[i] = 1.0 / L[(long long)i * N + i];
  __syncthreads();
  // forward: L t = f
  for (int r0 = 0; r0 < N; r0 += CB) {
    const int rn = min(CB, N - r0);
    for (int i = warp; i < rn; i += nw) {
      double s = 0.0;
      for (int j = lane; j < r0; j += 32) s = fma(L[(long long)(r0 + i) * N + j], x[j], s);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) rhs[i] = f[r0 + i] - s;
    }
    __syncthreads();
    if (warp == 0) {
      double v = lane < rn ? rhs[lane] : 0.0;  // lane = row r0 + lane
      for (int j = 0; j < rn; ++j) {
        const double xj = __shfl_sync(0xffffffffu, v * rd[r0 + j], j);
        if (lane == j) v = xj;
        else if (lane > j && lane < rn) v = fma(-L[(long long)(r0 + lane) * N + r0 + j], xj, v);
      }
      if (lane < rn) x[r0 + lane] = v;
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < N; i += blockDim.x) t[i] = x[i];
  __syncthreads();
  // backward: L^T a = t, row blocks from the bottom; (L^T)_{ij} = L_ji
  for (int r1 = N; r1 > 0; r1 -= CB) {
    const int r0 = max(0, r1 - CB), rn = r1 - r0;
    double s = 0.0;
    if (lane < rn)
      for (int j = r1 + warp; j < N; j += nw) s = fma(L[(long long)j * N + r0 + lane], x[j], s);
    part[warp][lane] = s;
    __syncthreads();
    if (warp == 0) {
      double v = 0.0;
      if (lane < rn) {
        v = t[r0 + lane];
        for (int w = 0; w < nw; ++w) v -= part[w][lane];
      }
      for (int j = rn - 1; j >= 0; --j) {  // column j of L^T's triangle = row j of L
        const double xj = __shfl_sync(0xffffffffu, v * rd[r0 + j], j);
        if (lane == j) v = xj;
        else if (lane < j) v = fma(-L[(long long)(r0 + j) * N + r0 + lane], xj, v);
      }
      if (lane < rn) x[r0 + lane] = v;
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < N; i += blockDim.x) a[i] = x[i];
}

}  // namespace

void cholsolve_f64(cudaStream_t s, const double* L, const double* f, double* t, double* a, int N,
                   int batch) {
  if (batch <= 0) return;
  k_cholsolve<<<batch, 1024, 2 * N * sizeof(double), s>>>(L, f, t, a, N);
}

void gemm_f64(cudaStream_t s, bool ta, bool tb, int m, int n, int k, double alpha, const double* A,
              int lda, long long sA, const double* B, int ldb, long long sB, double beta, double* C,
              int ldc, long long sC, int batch, bool sym, bool tri) {
  if (m <= 0 || n <= 0 || batch <= 0) return;
  dim3 grid((n + BN - 1) / BN, (m + BM - 1) / BM, batch);
  if (!ta && !tb)
    k_gemm<false, false><<<grid, GT, 0, s>>>(m, n, k, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, sym, tri);
  else if (!ta && tb)
    k_gemm<false, true><<<grid, GT, 0, s>>>(m, n, k, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, sym, tri);
  else if (ta && !tb)
    k_gemm<true, false><<<grid, GT, 0, s>>>(m, n, k, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, sym, tri);
  else
    k_gemm<true, true><<<grid, GT, 0, s>>>(m, n, k, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, sym, tri);
}

__global__ void k_zero_upper(double* __restrict__ Xb, int N);

// One panel step: the diagonal block, then the rows below it; the last step zeroes the strict
// upper triangle.
void chol_panel(cudaStream_t s, double* A, int N, int k0, int batch, double* rdiag, double* logdet,
                int lds, int* status, int per_chain) {
  k_chol_diag<<<batch, 128, 0, s>>>(A, N, k0, rdiag, logdet, lds, status, per_chain);
  const int kb = CB < N - k0 ? CB : N - k0, rows = N - k0 - kb;
  if (rows > 0) k_chol_rows<CB><<<dim3((rows + 127) / 128, batch), 128, 0, s>>>(A, N, k0, rdiag);
  else k_zero_upper<<<dim3((unsigned)(((long long)N * N + 255) / 256), batch), 256, 0, s>>>(A, N);
}

void cholesky_f64(cudaStream_t s, double* A, int N, int batch, double* logdet, int logdet_stride,
                  int* status, int per_chain, double* rdiag) {
  if (batch <= 0) return;
  if (N <= 2 * CB) {  // small: one CTA per matrix does it all
    k_chol<<<batch, 256, 0, s>>>(A, N, logdet, logdet_stride, status, per_chain);
    return;
  }
  const long long NN = (long long)N * N;
  for (int k0 = 0; k0 < N; k0 += CB) {
    chol_panel(s, A, N, k0, batch, rdiag, logdet, logdet_stride, status, per_chain);
    const int k1 = k0 + CB;
    if (k1 < N)
      gemm_f64(s, false, true, N - k1, N - k1, CB, -1.0, A + (long long)k1 * N + k0, N, NN,
               A + (long long)k1 * N + k0, N, NN, 1.0, A + (long long)k1 * N + k1, N, NN, batch, true, false);
  }
}

void cholesky_tc(cudaStream_t s, double* A, int N, int batch, double* logdet, int logdet_stride,
                 int* status, int per_chain, uint8_t* tcA, uint8_t* tcB, double* rdiag) {
  if (batch <= 0) return;
  if (N <= 2 * CB) {
    k_chol<<<batch, 256, 0, s>>>(A, N, logdet, logdet_stride, status, per_chain);
    return;
  }
  const long long NN = (long long)N * N;
  for (int k0 = 0; k0 < N; k0 += CB) {
    chol_panel(s, A, N, k0, batch, rdiag, logdet, logdet_stride, status, per_chain);
    const int k1 = k0 + CB;
    if (k1 < N) {  // A22 -= L21 L21^T, L21 = A[k1:, k0:k1] (rows of L21 on both sides)
      double* L21 = A + (long long)k1 * N + k0;
      const TcOperand a = tc_operand(tcA, N - k1, CB, 9, batch, false);
      const TcOperand b = tc_operand(tcB, N - k1, CB, 9, batch, true);
      tc_split(s, L21, N, NN, true, batch, a);
      tc_split(s, L21, N, NN, true, batch, b);
      gemm_tc(s, a, b, -1.0, 1.0, A + (long long)k1 * N + k1, N, NN, batch, true, status, per_chain);
    }
  }
}

void trinv_lower_f64(cudaStream_t s, const double* L, double* X, int N, int batch) {
  if (batch <= 0) return;
  dim3 grid((N + CB - 1) / CB, batch);
  k_trinv<<<grid, 256, 0, s>>>(L, X, N, N, 0);
}

// X[i][j] = 0 for j > i (the blocks above the diagonal that the recursion never writes).
__global__ void k_zero_upper(double* __restrict__ Xb, int N) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)N * N) return;
  if (e % N > e / N) Xb[(long long)blockIdx.y * N * N + e] = 0.0;
}

namespace {

// X[o:o+n, o:o+n] = L[o:o+n, o:o+n]^-1: leaves of at most 128 rows by k_trinv, otherwise
//   X11 = L11^-1, X22 = L22^-1, X21 = -X22 (L21 X11)
// with the two products on the tensor cores (FP64-accurate, 9 slices). T: batch x (N/2 + 16)^2.
void trinv_rec(cudaStream_t s, const double* L, double* X, int N, int o, int n, int batch,
               uint8_t* tcA, uint8_t* tcB, double* T, int* status, int sdiv) {
  if (n <= 128) {
    k_trinv<<<dim3((n + CB - 1) / CB, batch), 256, 0, s>>>(L, X, n, N, o);
    return;
  }
  const int n1 = ((n / 2 + 15) / 16) * 16, n2 = n - n1;
  trinv_rec(s, L, X, N, o, n1, batch, tcA, tcB, T, status, sdiv);
  trinv_rec(s, L, X, N, o + n1, n2, batch, tcA, tcB, T, status, sdiv);
  const long long NN = (long long)N * N;
  const double* L21 = L + (long long)(o + n1) * N + o;
  const double* X11 = X + (long long)o * N + o;
  const double* X22 = X + (long long)(o + n1) * N + o + n1;
  double* X21 = X + (long long)(o + n1) * N + o;
  constexpr int S = 9;
  // T = L21 X11 (n2 x n1): rows of L21, columns of X11
  TcOperand a = tc_operand(tcA, n2, n1, S, batch, false), b = tc_operand(tcB, n1, n1, S, batch, true);
  tc_split(s, L21, N, NN, true, batch, a);
  tc_split(s, X11, N, NN, false, batch, b);
  gemm_tc(s, a, b, 1.0, 0.0, T, n1, (long long)n2 * n1, batch, false, status, sdiv);
  // X21 = -X22 T (n2 x n1): rows of X22, columns of T
  a = tc_operand(tcA, n2, n2, S, batch, false);
  b = tc_operand(tcB, n1, n2, S, batch, true);
  tc_split(s, X22, N, NN, true, batch, a);
  tc_split(s, T, n1, (long long)n2 * n1, false, batch, b);
  gemm_tc(s, a, b, -1.0, 0.0, X21, N, NN, batch, false, status, sdiv);
}

}  // namespace

void trinv_lower_tc(cudaStream_t s, const double* L, double* X, int N, int batch, uint8_t* tcA,
                    uint8_t* tcB, double* T, int* status, int sdiv) {
  if (batch <= 0 || N <= 0) return;
  k_zero_upper<<<dim3((unsigned)(((long long)N * N + 255) / 256), batch), 256, 0, s>>>(X, N);
  trinv_rec(s, L, X, N, 0, N, batch, tcA, tcB, T, status, sdiv);
}

void gemv_f64(cudaStream_t s, bool ta, int rows, int cols, const double* A, int lda, long long sA,
              const double* x, long long sx, double* y, long long sy, int batch, double alpha,
              double beta) {
  if (batch <= 0) return;
  if (!ta) {
    dim3 grid((rows * 32 + 255) / 256, batch);
    k_gemv_n<<<grid, 256, 0, s>>>(rows, cols, A, lda, sA, x, sx, y, sy, alpha, beta);
  } else {
    dim3 grid((cols + 127) / 128, batch);
    k_gemv_t<<<grid, 128, 0, s>>>(rows, cols, A, lda, sA, x, sx, y, sy, alpha, beta);
  }
}

}  // namespace rmhmc
