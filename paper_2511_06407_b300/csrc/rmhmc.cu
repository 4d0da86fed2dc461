// librmhmc: C ABI, per-chain state and the generalized-leapfrog / Algorithm 1 orchestration of
// the plain-FP64 SoftAbs-RMHMC path (declared in include/rmhmc.h).
//
// Every step of the path runs in the CUDA kernels of this library, enqueued on the model's
// stream; the host only sequences launches. Internal vectors use the padded dimension dp (a
// multiple of 16 >= d, zero in the padding) so that the d x d matrices tile evenly for the
// Jacobi blocks.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "df.cuh"
#include "internal.cuh"
#include "model_kernels.cuh"
#include "primal.cuh"

using namespace rmhmc;

namespace {

// ------------------------------------------------------------------------------- device helpers

// Soft-absolute map (Sec. 2.2): g(l) = l coth(alpha l) or sqrt(1/alpha^2 + l^2), and g'(l).
// coth form, x = alpha l:  |x| < 1e-3 Laurent series of x coth x (and of its derivative);
// |x| > 20 saturated (g = |l|, g' = sign l); |x| <= 1 g' = (sinh 2x - 2x) / (2 sinh^2 x) with
// sinh y - y summed from its Taylor series (no cancellation); otherwise g = l / tanh x,
// g' = 1/tanh x - x / sinh^2 x.
__device__ __forceinline__ double sinh_minus_identity(double y) {
  const double y2 = y * y;
  double term = y * y2 / 6.0, sum = 0.0;
  for (int k = 1; k <= 12; ++k) {
    sum += term;
    term *= y2 / ((2.0 * k + 2.0) * (2.0 * k + 3.0));
  }
  return sum;
}

__device__ __forceinline__ void softabs(double lam, double alpha, int kind, double& g, double& gp) {
  if (kind == RMHMC_G_SQRT) {
    const double kap = 1.0 / alpha;
    const double r = sqrt(kap * kap + lam * lam);
    g = r;
    gp = lam / r;
    return;
  }
  const double x = alpha * lam, ax = fabs(x);
  if (ax < 1e-3) {
    const double x2 = x * x;
    g = (1.0 + x2 / 3.0 - x2 * x2 / 45.0 + 2.0 * x2 * x2 * x2 / 945.0) / alpha;
    gp = 2.0 * x / 3.0 - 4.0 * x * x2 / 45.0 + 4.0 * x * x2 * x2 / 315.0;
  } else if (ax > 20.0) {
    g = fabs(lam);
    gp = lam > 0.0 ? 1.0 : -1.0;
  } else {
    const double th = tanh(x), sh = sinh(x);
    g = lam / th;
    gp = (ax <= 1.0) ? sinh_minus_identity(2.0 * x) / (2.0 * sh * sh) : 1.0 / th - x / (sh * sh);
  }
}

__global__ void k_softabs(const double* __restrict__ lam, double* __restrict__ g,
                          double* __restrict__ gp, int dp, int d, int C, double alpha, int kind) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)C * dp) return;
  const int i = (int)(e % dp);
  double a = 1.0, b = 0.0;
  if (i < d) softabs(lam[e], alpha, kind, a, b);
  g[e] = a;
  gp[e] = b;
}

// 1 / x for |x| in [1e-30, 1e30]: the FP32 reciprocal refined by two Newton steps r <- r (2 - x r)
// in FP64 (relative error ~1e-7 -> ~1e-14 -> FP64 rounding); a plain division outside that range.
__device__ __forceinline__ double recip_newton(double x) {
  const double ax = fabs(x);
  if (!(ax >= 1e-30 && ax <= 1e30)) return 1.0 / x;
  double r = (double)__frcp_rn((float)x);
  r = fma(r, fma(-x, r, 1.0), r);
  return fma(r, fma(-x, r, 1.0), r);
}

// C = diag(g'/g) - (b b^T) o T on the first d indices (zero elsewhere), b = t / g, with T the
// divided differences of Eq. d3_transform (near-equal eigenvalues take g' at the midpoint):
// Psi C Psi^T = W2 - W1 (Eq. Betancourt_formula). Grid (32 x 32 tiles of the lower triangle, C):
// the tile's b and g'/g are formed once (64 divisions instead of two per element), T_jl's division
// goes through recip_newton, and since every term is exactly symmetric in (j, l) (recip_newton is
// odd, the products commute) each tile below the diagonal is written twice, the mirror through a
// shared-memory transpose.
__global__ void __launch_bounds__(256) k_build_c(const double* __restrict__ t, const double* __restrict__ lam,
                                                 const double* __restrict__ g, const double* __restrict__ gp,
                                                 double* __restrict__ Cm, int dp, int d, double alpha,
                                                 int kind) {
  const int c = blockIdx.y, tile = blockIdx.x;
  int tj = (int)((sqrt(8.0 * tile + 1.0) - 1.0) * 0.5);  // tile (tj, tl), tl <= tj
  while (tj * (tj + 1) / 2 > tile) --tj;
  while ((tj + 1) * (tj + 2) / 2 <= tile) ++tj;
  const int tl = tile - tj * (tj + 1) / 2;
  const int j0 = tj * 32, l0 = tl * 32;
  const long long o = (long long)c * dp;
  __shared__ double sb[2][32], sl[2][32], sg[2][32], sgp[2][32];
  __shared__ double tileC[32][33];
  if (threadIdx.x < 64) {
    const int side = threadIdx.x >> 5, idx = (side == 0 ? j0 : l0) + (threadIdx.x & 31);
    const bool in = idx < d;
    const double gi = in ? g[o + idx] : 1.0;
    sg[side][threadIdx.x & 31] = gi;
    sb[side][threadIdx.x & 31] = in ? t[o + idx] / gi : 0.0;
    sl[side][threadIdx.x & 31] = in ? lam[o + idx] : 0.0;
    sgp[side][threadIdx.x & 31] = in ? gp[o + idx] : 0.0;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
  const int l = l0 + lane;
  double* Cc = Cm + (long long)c * dp * dp;
  for (int r = wy; r < 32; r += 8) {
    const int j = j0 + r;
    double v = 0.0;
    if (j < d && l < d && l <= j) {
      double T;
      if (j == l) {
        T = sgp[0][r];
      } else {
        const double lj = sl[0][r], ll = sl[1][lane];
        const double sc = fmax(1.0, fmax(fabs(lj), fabs(ll)));
        if (fabs(lj - ll) <= 1e-7 * sc) {  // near-equal eigenvalues: g' at the midpoint
          double gm, gpm;
          softabs(0.5 * (lj + ll), alpha, kind, gm, gpm);
          T = gpm;
        } else {
          T = (sg[0][r] - sg[1][lane]) * recip_newton(lj - ll);
        }
      }
      v = -sb[0][r] * sb[1][lane] * T;
      if (j == l) v += sgp[0][r] / sg[0][r];
    }
    tileC[r][lane] = v;
    if (j < dp && l < dp && (tj != tl || l <= j)) Cc[(long long)j * dp + l] = v;
  }
  __syncthreads();
  for (int r = wy; r < 32; r += 8) {  // (l, j) = mirror of the tile's (j, l), strictly above the diagonal
    const int lr = l0 + r, jc = j0 + lane;
    if (lr < dp && jc < dp && jc > lr) Cc[(long long)lr * dp + jc] = tileC[lane][r];
  }
}

// t_i <- t_i * s(g_i) on the first d entries (s = 1/g or sqrt(g)), zero in the padding.
__global__ void k_scale_g(double* __restrict__ t, const double* __restrict__ g, int dp, int d, int C,
                          int mode) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)C * dp) return;
  const int i = (int)(e % dp);
  t[e] = (i < d) ? (mode == 0 ? t[e] / g[e] : t[e] * sqrt(g[e])) : 0.0;
}

// out = a + s * b (vectors of C x dp)
__global__ void k_axpy(double* __restrict__ out, const double* __restrict__ a,
                       const double* __restrict__ b, double s, long long n) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) out[e] = a[e] + s * b[e];
}

// out = a + s * (b + c)
__global__ void k_axpy2(double* __restrict__ out, const double* __restrict__ a,
                        const double* __restrict__ b, const double* __restrict__ cc, double s,
                        long long n) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) out[e] = a[e] + s * (b[e] + cc[e]);
}

// Strided copy between the caller's d-stride layout and the internal dp-stride layout.
__global__ void k_restride(double* __restrict__ dst, int dst_ld, const double* __restrict__ src,
                           int src_ld, int d, int C) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)C * dst_ld) return;
  const int c = (int)(e / dst_ld), i = (int)(e % dst_ld);
  dst[e] = (i < d && src) ? src[(long long)c * src_ld + i] : 0.0;
}

__global__ void k_set_identity(double* __restrict__ A, int dp, int C) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)C * dp * dp) return;
  const long long r = e % ((long long)dp * dp);
  A[e] = (r / dp == r % dp) ? 1.0 : 0.0;
}

// H(q, p) of Eq. Hamiltonian per chain: U + (d log 2pi + sum log g) / 2 + p . (G^-1 p) / 2.
__global__ void __launch_bounds__(256) k_hamiltonian(const double* __restrict__ U,
                                                     const double* __restrict__ g,
                                                     const double* __restrict__ p,
                                                     const double* __restrict__ ginvp, int dp, int d,
                                                     double* __restrict__ Ham) {
  const int c = blockIdx.x;
  __shared__ double sh[32];
  double lg = 0.0, quad = 0.0;
  for (int i = threadIdx.x; i < d; i += blockDim.x) {
    const long long o = (long long)c * dp + i;
    lg += log(g[o]);
    quad = fma(p[o], ginvp[o], quad);
  }
  const double a = dev::block_sum(lg, sh);
  const double b = dev::block_sum(quad, sh);
  if (threadIdx.x == 0) Ham[c] = U[c] + 0.5 * (d * dev::LOG2PI + a) + 0.5 * b;
}

// Philox4x64-10 (Salmon et al., SC'11) with the published multipliers and Weyl increments.
__device__ __forceinline__ void philox(uint64_t x[4], uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t lo0 = M0 * x[0], hi0 = __umul64hi(M0, x[0]);
    const uint64_t lo1 = M1 * x[2], hi1 = __umul64hi(M1, x[2]);
    const uint64_t n0 = hi1 ^ x[1] ^ k0, n2 = hi0 ^ x[3] ^ k1;
    x[0] = n0;
    x[1] = lo1;
    x[2] = n2;
    x[3] = lo0;
    k0 += W0;
    k1 += W1;
  }
}

// Momentum normals: block b of (seed, chain, iteration) gives z[4b..4b+3] by Box-Muller.
__global__ void k_normals(double* __restrict__ z, int dp, int d, int C, uint64_t seed, uint64_t iter) {
  const int c = blockIdx.y;
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (4 * b >= dp) return;
  uint64_t x[4] = {(uint64_t)b, iter, 0ull, 0ull};
  philox(x, seed, (uint64_t)c);
  for (int pr = 0; pr < 2; ++pr) {
    const double u1 = (double)((x[2 * pr] >> 11) + 1) * 0x1.0p-53;
    const double u2 = (double)(x[2 * pr + 1] >> 11) * 0x1.0p-53;
    const double r = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    const int i0 = 4 * b + 2 * pr;
    if (i0 < dp) z[(long long)c * dp + i0] = (i0 < d) ? r * cs : 0.0;
    if (i0 + 1 < dp) z[(long long)c * dp + i0 + 1] = (i0 + 1 < d) ? r * sn : 0.0;
  }
}

// Metropolis-Hastings decision per chain (Algorithm 1): r from counter (0, iteration, 1, 0).
__global__ void k_accept(const double* __restrict__ H0, const double* __restrict__ H1,
                         int* __restrict__ status, int* __restrict__ acc, int C, uint64_t seed,
                         uint64_t iter, int* __restrict__ acc_out, int* __restrict__ sweeps_out,
                         const int* __restrict__ sweeps_acc, int* __restrict__ chain_status) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  uint64_t x[4] = {0ull, iter, 1ull, 0ull};
  philox(x, seed, (uint64_t)c);
  const double r = (double)(x[0] >> 11) * 0x1.0p-53;
  int st = status[c];
  if (!isfinite(H1[c])) st |= RMHMC_CHAIN_NONFINITE;
  const int a = (st == 0) && (log(r) < H0[c] - H1[c]);
  acc[c] = a;
  if (acc_out) acc_out[c] = a;
  if (sweeps_out) sweeps_out[c] = sweeps_acc[c];
  if (chain_status) chain_status[c] |= st;
  status[c] = 0;
}

// After rmhmc_leapfrog: a chain whose position, momentum, potential U or (when computed) Hamiltonian
// is not finite gets RMHMC_CHAIN_NONFINITE in the model's status (so that a later Metropolis-Hastings
// step rejects it) and in the caller's copy (out, may be null). Finiteness from the exponent bits.
__global__ void __launch_bounds__(128) k_flag_nonfinite(int* __restrict__ status, int* __restrict__ out,
                                                        const double* __restrict__ q,
                                                        const double* __restrict__ p,
                                                        const double* __restrict__ U,
                                                        const double* __restrict__ H, int dp, int d) {
  const int c = blockIdx.x;
  const long long o = (long long)c * dp;
  auto inf_or_nan = [](double x) { return (__double2hiint(x) & 0x7ff00000) == 0x7ff00000; };
  bool bad = false;
  for (int j = threadIdx.x; j < d; j += blockDim.x) bad |= inf_or_nan(q[o + j]) || inf_or_nan(p[o + j]);
  bad = __syncthreads_or(bad);
  if (threadIdx.x == 0) {
    bad = bad || inf_or_nan(U[c]) || (H != nullptr && inf_or_nan(H[c]));
    int st = status[c];
    if (bad) {
      st |= RMHMC_CHAIN_NONFINITE;
      status[c] = st;
    }
    if (out) out[c] = st;
  }
}

// Rejected chains return to the saved position and eigenvectors.
__global__ void k_restore(const int* __restrict__ acc, double* __restrict__ q,
                          const double* __restrict__ q_save, double* __restrict__ PsiT,
                          const double* __restrict__ PsiT_save, int* __restrict__ eig_count,
                          const int* __restrict__ eig_save, int dp) {
  const int c = blockIdx.y;
  if (acc[c]) return;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long o = (long long)c * dp * dp;
  if (e < (long long)dp * dp) PsiT[o + e] = PsiT_save[o + e];
  if (e < dp) q[(long long)c * dp + e] = q_save[(long long)c * dp + e];
  if (e == 0) eig_count[c] = eig_save[c];
}

// mask[c] = 1 where eig_count[c] is a positive multiple of every (re-orthonormalisation due)
__global__ void k_reorth_mask(const int* __restrict__ eig_count, int every, int C, int* __restrict__ mask) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < C) mask[c] = (eig_count[c] > 0 && eig_count[c] % every == 0) ? 1 : 0;
}

// eig_count += 1 per chain; sweeps_total += sweeps of the eigen-update just done
__global__ void k_inc(int* __restrict__ v, int C, int* __restrict__ tot, const int* __restrict__ last) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < C) {
    v[c] += 1;
    tot[c] += last[c];
  }
}

__global__ void k_record(const double* __restrict__ q, const double* __restrict__ U,
                         const double* __restrict__ LL, int dp, int d, int C,
                         double* __restrict__ qs, double* __restrict__ logp,
                         double* __restrict__ loglik) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)C * d) return;
  const int c = (int)(e / d), i = (int)(e % d);
  if (qs) qs[e] = q[(long long)c * dp + i];
  if (logp && i == 0) logp[c] = -U[c];
  if (loglik && i == 0) loglik[c] = LL[c];
}

// dst (C x d x d) <- the leading d x d block of src (C x dp x dp)
__global__ void k_compact(double* __restrict__ dst, const double* __restrict__ src, int dp, int d, int C) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)C * d * d) return;
  const long long c = e / ((long long)d * d), r = e % ((long long)d * d);
  dst[e] = src[c * dp * dp + (r / d) * dp + r % d];
}

// Y = diag(g) PsiT on the first d rows (zero below)
__global__ void k_scale_rows(double* __restrict__ Y, const double* __restrict__ PsiT,
                             const double* __restrict__ g, int dp, int d) {
  const int c = blockIdx.y;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)dp * dp) return;
  const int r = (int)(e / dp);
  const long long o = (long long)c * dp * dp + e;
  Y[o] = r < d ? g[(long long)c * dp + r] * PsiT[o] : 0.0;
}

// Eight independent FMA chains per thread: enough instruction-level parallelism to keep the FP64
// pipe busy; the result is kept live through a data-dependent store that never happens.
template <typename T>
__global__ void k_fma_peak(T* __restrict__ sink, int iters, T b, T c) {
  T a0 = (T)(threadIdx.x * 1e-3), a1 = a0 + (T)1, a2 = a0 + (T)2, a3 = a0 + (T)3;
  T a4 = a0 + (T)4, a5 = a0 + (T)5, a6 = a0 + (T)6, a7 = a0 + (T)7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      a0 = fma(a0, b, c); a1 = fma(a1, b, c); a2 = fma(a2, b, c); a3 = fma(a3, b, c);
      a4 = fma(a4, b, c); a5 = fma(a5, b, c); a6 = fma(a6, b, c); a7 = fma(a7, b, c);
    }
  }
  const T s = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
  if (s == (T)12345.678) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// ---- first-order pre-rotation of a warm eigen-update (mixed form)
// After a warm start M = Psi^T H Psi differs from a diagonal matrix by small couplings. Every pair
// (j, l) whose coupling fails the Jacobi stopping rule gets the rotation angle that zeroes it to
// first order, theta_jl = atan(2 m_jl / (m_ll - m_jj)) / 2 (antisymmetric in j, l); with the skew
// matrix A of these angles, X = I + A + A^2 / 2 + A^3 / 6 + A^4 / 24 (exp(A) to fourth order) is
// orthogonal up to A^6 / 72 (X^T X = I + A^6 / 72 + A^8 / 576: the odd orders cancel for skew A),
// and X^T M X has every such coupling reduced to second order. The Jacobi that follows checks the
// stopping rule as usual and rotates whatever is left. A chain takes the pre-rotation only when
// ||A||_F <= 1e-3 (then ||A^6|| / 72 is below 1e-19), i.e. after a warm start; a cold start
// (Psi = I) is left to the Jacobi. A pair whose first-order angle exceeds kPrerotMaxTheta (nearly
// equal diagonal entries: the first-order step would be poor) is left out of A for the Jacobi.
constexpr double kPrerotMaxA = 1e-3;
constexpr double kPrerotMaxTheta = 1e-5;
// |theta| <= 1e-5 <=> |x| <= tan(2e-5) for x = 2 m_jl / (m_ll - m_jj); the cut is taken at 2e-5 (the
// two differ by 3e-15 relative). On |x| <= 2e-5, atan(x) = x (1 - x^2 / 3 + ...) with x^2 / 3 below
// FP32 rounding, so the FP32 angle is x / 2.
constexpr double kPrerotMaxX = 2.0 * kPrerotMaxTheta;
constexpr int kPrerotParts = 16;  // CTAs per chain of k_prerot_norms

// Per chain, in kPrerotParts CTAs: partial sums of ||M||_F^2 and partial minima of |m_ii| (i < d),
// part[(c * kPrerotParts + b) * 2 + {0, 1}]; CTA 0 also clears the chain's sums of theta^2 and of
// the entries of A (acc[4 c + 2], acc[4 c + 3]) for k_prerot_rows. Grid (kPrerotParts, chains).
__global__ void __launch_bounds__(256) k_prerot_norms(const double* __restrict__ Mb, int dp, int d,
                                                      double* __restrict__ acc, double* __restrict__ part) {
  const int c = blockIdx.y, b = blockIdx.x;
  const long long DD = (long long)dp * dp;
  const double* M = Mb + c * DD;
  double tot = 0.0, dmin = 1e308;
  const long long e0 = DD * b / kPrerotParts, e1 = DD * (b + 1) / kPrerotParts;
  for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const double v = M[e];
    tot = fma(v, v, tot);
  }
  const int i0 = (int)((long long)d * b / kPrerotParts), i1 = (int)((long long)d * (b + 1) / kPrerotParts);
  for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) dmin = fmin(dmin, fabs(M[(long long)i * dp + i]));
  __shared__ double r0[8], r1[8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    tot += __shfl_xor_sync(0xffffffffu, tot, o);
    dmin = fmin(dmin, __shfl_xor_sync(0xffffffffu, dmin, o));
  }
  if ((threadIdx.x & 31) == 0) {
    r0[threadIdx.x >> 5] = tot;
    r1[threadIdx.x >> 5] = dmin;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0, m = 1e308;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      t += r0[w];
      m = fmin(m, r1[w]);
    }
    part[((long long)c * kPrerotParts + b) * 2] = t;
    part[((long long)c * kPrerotParts + b) * 2 + 1] = m;
    if (b == 0) {
      acc[4 * c + 2] = 0.0;  // sum of theta^2
      acc[4 * c + 3] = 0.0;  // entries of A
    }
  }
}

// x as a double-float pair (hi, lo) by integer operations on its bits (B300's FP64 pipe, which also
// runs the FP64 <-> FP32 conversions, is 1/64 of its FP32 rate): hi = x rounded to 24 significant
// bits, lo = x - hi rounded to 24 (both ties away from zero), so |x - hi - lo| <= 2^-25 |lo| <=
// 2^-49 |x|. Zero, subnormal doubles and magnitudes below FP32's normal range give (+-0, 0), and lo
// is 0 where it would fall below that range (|x| < ~1e-30); beyond the range hi is +-inf, and a NaN
// stays a NaN.
__device__ __forceinline__ float2 df_split_bits(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const unsigned long long mag = b & 0x7fffffffffffffffull;
  const int E = (int)(mag >> 52);
  if (E == 0x7ff)
    return make_float2(__uint_as_float(sign | 0x7f800000u | ((mag & 0xfffffffffffffull) ? 0x400000u : 0u)), 0.f);
  if (E < 1023 - 126) return make_float2(__uint_as_float(sign), 0.f);
  const unsigned low = (unsigned)(mag & 0x1fffffffull);                 // the 29 bits below hi
  const unsigned up = (low >> 28) & 1u;                                   // round half away from zero
  const unsigned long long hmag = (mag & ~0x1fffffffull) + ((unsigned long long)up << 29);  // (carries into E)
  const int Eh = (int)(hmag >> 52);
  if (Eh > 1023 + 127) return make_float2(__uint_as_float(sign | 0x7f800000u), 0.f);
  const float hi = __uint_as_float(sign | ((unsigned)(Eh - 1023 + 127) << 23) | (unsigned)((hmag >> 29) & 0x7fffffu));
  const int R = (int)low - (int)(up << 29);  // x - hi in units of 2^(E - 1075), |R| <= 2^28
  if (R == 0) return make_float2(hi, 0.f);
  const unsigned r = (unsigned)(R < 0 ? -R : R);
  const int nb = 32 - __clz(r);
  const int el = E - 1075 + (nb - 1) + 127;
  if (el <= 0) return make_float2(hi, 0.f);
  unsigned m = nb > 24 ? ((r >> (nb - 25)) + 1u) >> 1 : (r << (24 - nb));  // (rounded half up)
  int ef = el;
  if (m >> 24) {  // (the rounding carried into a 25th bit)
    m >>= 1;
    ++ef;
  }
  return make_float2(hi, __uint_as_float((sign ^ (R < 0 ? 0x80000000u : 0u)) | ((unsigned)ef << 23) | (m & 0x7fffffu)));
}

__device__ __forceinline__ bool finite_bits(double x) {
  return ((unsigned long long)__double_as_longlong(x) & 0x7ff0000000000000ull) != 0x7ff0000000000000ull;
}

// The rows of A (skew) as lists: for row j, the columns l and angles theta_jl of the pairs that
// fail the Jacobi's coupling test (METRIC or RELATIVE, with the double-float rounding floor
// 4 * 2^-48 ||M||_F). One warp per row (grid: row groups of 8, chains); the warp compacts its row
// with ballots. Per chain, entry e of row j is ent[e * dp + j] = (l, theta_jl as FP32 bits), entry-
// major so that the warps that walk 32 rows at once read one line per entry, and cnt[j] is the
// row's length (0 for the padding rows j >= d). The sums of theta^2 and of the entries are reduced
// per CTA before one atomic each.
// The angles are FP32: X (exp(A) to fourth order, below) is orthogonal to rounding for any small
// skew A, and M and Psi are rotated by the same X, so the angles' rounding only leaves a coupling of
// ~2^-24 of its size for the Jacobi. theta_lj = -theta_jl exactly (M is symmetric, the FP32
// conversions are sign-symmetric and the FP32 quotient is correctly rounded).
__global__ void __launch_bounds__(256) k_prerot_rows(const double* __restrict__ Mb, const double* __restrict__ part,
                                                     int dp, int d, int rule, double tol,
                                                     const int* __restrict__ status, int2* __restrict__ entb,
                                                     int* __restrict__ cntb, double* __restrict__ acc) {
  const int c = blockIdx.y, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long DD = (long long)dp * dp;
  const int j = blockIdx.x * 8 + warp;
  const double* M = Mb + c * DD;
  int2* ent = entb + c * DD;
  int* cnt = cntb + (long long)c * dp;
  // the test's constants, once per CTA: log2 of the floor, of tol^2 and of min |m_ii|^2 (the
  // partial results of k_prerot_norms in a fixed order)
  __shared__ float sfl[3];
  if (threadIdx.x == 0) {
    double nrm2 = 0.0, dmin = 1e308;
    for (int b = 0; b < kPrerotParts; ++b) {
      nrm2 += part[((long long)c * kPrerotParts + b) * 2];
      dmin = fmin(dmin, part[((long long)c * kPrerotParts + b) * 2 + 1]);
    }
    sfl[0] = log2_abs(16.0 * 1.2621774483536189e-29 * nrm2);
    sfl[1] = 2.f * log2_abs(tol);
    sfl[2] = 2.f * log2_abs(dmin);
  }
  __syncthreads();
  float t2 = 0.f;
  int n = 0;
  if (j < dp) {
    const bool live = j < d && status[c] == 0;
    // the stopping rule's test in the log domain (exponent fields and FP32 logarithms), the angle in
    // FP32 for the pairs that fail it
    const float lfloor2 = sfl[0], ltol2 = sfl[1], ldmin2 = sfl[2];
    const double djj = M[(long long)j * dp + j];
    const float lj = log2_abs(djj);
    const float fjj = df_split_bits(djj).x;
    for (int kb = 0; kb < dp; kb += 32) {
      const int l = kb + lane;
      float th = 0.f;
      if (live && l < d && l != j) {
        const double v = M[(long long)j * dp + l];
        const double dll = M[(long long)l * dp + l];
        const float lv = log2_abs(v), ll = log2_abs(dll);
        float lthr, lfl;
        if (rule == RMHMC_JACOBI_RELATIVE) {
          lthr = ltol2 + lj + ll;
          lfl = fminf(lfloor2, fmaxf(-86.37013f + 2.f * fmaxf(lj, ll), -996.578f));
        } else {
          lthr = ltol2 + 2.f * (lj + ll) - fmaxf(ldmin2, -996.578f);
          lfl = lfloor2;
        }
        const bool fin = finite_bits(v);
        if (!fin || 2.f * lv > fmaxf(lthr, lfl)) {
          // theta = atan(x) / 2 ~ x / 2 (x^2 / 3 < 2^-24 here); x = +-inf (equal diagonal entries,
          // or an entry beyond the FP32 range) and |x| > 2e-5 are left to the Jacobi; a non-finite
          // coupling or a NaN marks the chain (theta = 1: ||A||_F too large)
          const float x = 2.f * df_split_bits(v).x / (df_split_bits(dll).x - fjj);
          if (!fin || isnan(x)) th = 1.f;
          else if (fabsf(x) <= (float)kPrerotMaxX) th = 0.5f * x;
        }
      }
      const unsigned bal = __ballot_sync(0xffffffffu, th != 0.f);
      if (th != 0.f) {
        const int pos = n + __popc(bal & ((1u << lane) - 1u));
        ent[(long long)pos * dp + j] = make_int2(l, __float_as_int(th));
      }
      n += __popc(bal);
      t2 = fmaf(th, th, t2);
    }
    if (lane == 0) cnt[j] = n;
  }
  // (in FP32: the sum only decides the ||A||_F <= 1e-3 test, and the count is an integer)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t2 += __shfl_xor_sync(0xffffffffu, t2, o);
  __shared__ float r0[8];
  __shared__ int r1[8];
  if (lane == 0) {
    r0[warp] = t2;
    r1[warp] = n;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float a = 0.f;
    int b = 0;
    for (int w = 0; w < 8; ++w) {
      a += r0[w];
      b += r1[w];
    }
    if (b != 0) {
      atomicAdd(&acc[4 * c + 2], (double)a);
      atomicAdd(&acc[4 * c + 3], (double)b);
    }
  }
}

// (sh, sl) += t * (ah + al) for a double-float pair (ah, al) and an FP32 t: the product t * ah
// exactly (FMA residual), the running high sum by two-sum, t * al and the residuals into the low
// word (Dekker / Knuth error-free transformations; the low word is not renormalised: it stays
// below n 2^-24 |sh| for n terms)
__device__ __forceinline__ void df_madd(float& sh, float& sl, float t, float ah, float al) {
  const float p = t * ah;
  const float e = fmaf(t, ah, -p);
  const float s = sh + p;
  const float bp = s - sh;
  const float err = (sh - (s - bp)) + (p - bp);
  sh = s;
  sl += fmaf(t, al, err + e);
}

constexpr int kPrerotLines = 8;   // lines of the matrix per CTA of k_prerot_apply
constexpr int kPrerotLight = 32;  // rows with more entries go to a whole warp

// out(j) for every row j < dp of the 8 lines at once: -sum_k theta_jk in(k) over row j's list
// (in = ih + il, double-float pairs, [dp][8] in shared memory, read four lines at a time; the result
// as pairs (sh, sl) handed to sink(j, sh, sl)). Rows of at most 32 entries one per thread (the next
// entry loaded ahead; the entry-major lists give the 32 rows of a warp one line per entry), longer
// ones one per warp (lane-strided entries, then a tree over the lanes: lane 0's sum, in an order
// fixed by the lane numbers). The few rows of the smallest eigenvalues fail the test against nearly
// every partner: one thread each would serialise their warps.
template <class Sink>
__device__ __forceinline__ void prerot_product_df(const int2* __restrict__ ent, const int* scnt, const int* heavy,
                                                  int nh, int dp, const float* ih, const float* il, Sink sink) {
  constexpr int TL = kPrerotLines;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  auto madd = [&](float* sh, float* sl, int2 en) {
    const float t = -__int_as_float(en.y);
    const float4* h4 = reinterpret_cast<const float4*>(ih + en.x * TL);
    const float4* l4 = reinterpret_cast<const float4*>(il + en.x * TL);
#pragma unroll
    for (int q = 0; q < TL / 4; ++q) {
      const float4 h = h4[q], lo = l4[q];
      df_madd(sh[4 * q], sl[4 * q], t, h.x, lo.x);
      df_madd(sh[4 * q + 1], sl[4 * q + 1], t, h.y, lo.y);
      df_madd(sh[4 * q + 2], sl[4 * q + 2], t, h.z, lo.z);
      df_madd(sh[4 * q + 3], sl[4 * q + 3], t, h.w, lo.w);
    }
  };
  for (int j = threadIdx.x; j < dp; j += blockDim.x) {
    const int n = scnt[j];
    if (n > kPrerotLight) continue;
    float sh[TL], sl[TL];
#pragma unroll
    for (int l = 0; l < TL; ++l) sh[l] = sl[l] = 0.f;
    int2 nx = n > 0 ? ent[j] : make_int2(0, 0);
    for (int e = 0; e < n; ++e) {
      const int2 en = nx;
      if (e + 1 < n) nx = ent[(long long)(e + 1) * dp + j];
      madd(sh, sl, en);
    }
    sink(j, sh, sl);
  }
  for (int h = warp; h < nh; h += nwarp) {
    const int j = heavy[h], n = scnt[j];
    float sh[TL], sl[TL];
#pragma unroll
    for (int l = 0; l < TL; ++l) sh[l] = sl[l] = 0.f;
    for (int e = lane; e < n; e += 32) madd(sh, sl, ent[(long long)e * dp + j]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
      for (int l = 0; l < TL; ++l) {
        const float oh = __shfl_down_sync(0xffffffffu, sh[l], o), ol = __shfl_down_sync(0xffffffffu, sl[l], o);
        const float s = sh[l] + oh;
        const float bp = s - sh[l];
        const float err = (sh[l] - (s - bp)) + (oh - bp);
        sh[l] = s;
        sl[l] += ol + err;
      }
    }
    if (lane == 0) sink(j, sh, sl);
  }
}

// The same product in FP32 (in and the result u single words; sink(j, u)).
template <class Sink>
__device__ __forceinline__ void prerot_product_f32(const int2* __restrict__ ent, const int* scnt, const int* heavy,
                                                   int nh, int dp, const float* in, Sink sink) {
  constexpr int TL = kPrerotLines;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  auto madd = [&](float* u, int2 en) {
    const float t = __int_as_float(en.y);
    const float4* v4 = reinterpret_cast<const float4*>(in + en.x * TL);
#pragma unroll
    for (int q = 0; q < TL / 4; ++q) {
      const float4 v = v4[q];
      u[4 * q] = fmaf(-t, v.x, u[4 * q]);
      u[4 * q + 1] = fmaf(-t, v.y, u[4 * q + 1]);
      u[4 * q + 2] = fmaf(-t, v.z, u[4 * q + 2]);
      u[4 * q + 3] = fmaf(-t, v.w, u[4 * q + 3]);
    }
  };
  for (int j = threadIdx.x; j < dp; j += blockDim.x) {
    const int n = scnt[j];
    if (n > kPrerotLight) continue;
    float u[TL];
#pragma unroll
    for (int l = 0; l < TL; ++l) u[l] = 0.f;
    int2 nx = n > 0 ? ent[j] : make_int2(0, 0);
    for (int e = 0; e < n; ++e) {
      const int2 en = nx;
      if (e + 1 < n) nx = ent[(long long)(e + 1) * dp + j];
      madd(u, en);
    }
    sink(j, u);
  }
  for (int h = warp; h < nh; h += nwarp) {
    const int j = heavy[h], n = scnt[j];
    float u[TL];
#pragma unroll
    for (int l = 0; l < TL; ++l) u[l] = 0.f;
    for (int e = lane; e < n; e += 32) madd(u, ent[(long long)e * dp + j]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
      for (int l = 0; l < TL; ++l) u[l] += __shfl_down_sync(0xffffffffu, u[l], o);
    }
    if (lane == 0) sink(j, u);
  }
}

// v <- v X with X = I + A + A^2 / 2 + A^3 / 6 + A^4 / 24 for 8 lines v of one chain's dp x dp matrix
// at a time: the rows of the input (COLS false: the lines are rows, Z = M X) or its columns (COLS
// true: X^T Y, whose column c is Y[:, c] X). The input is FP64 (inb) or double-float pairs
// (IN_PAIRS: in2b); the output is double-float pairs (out2b, laid out as the input), the form the
// double-float Jacobi works in. With w1 = v A (A skew: (v A)_j = -sum_k theta_jk v_k) and
// w_{k+1} = w_k A, v X = v + w1 + w2 / 2 + w3 / 6 + w4 / 24, |w_k| <= ||A||_F^k |v| <= 1e-3k |v|:
// w1 and w2 are formed in double-float pairs (v as hi + lo, ~48 bits), w3 (<= 1e-9 |v|) and w4 in
// FP32, each within ~1e-16 |v|, and v + (their sum) by a double-float addition. An FP64 input is
// split once, and its pairs are kept in the output's places for that last addition. SYM (with
// COLS): the output is symmetric, and the CTA of column c writes both out[k][c] and out[c][k] for
// k <= c (each pair of mirrored entries has one writer). Grid (dp / 8, chains); shared memory
// 128 dp + 8 dp bytes; chains with mask 0 return. The summation order of every output is fixed
// (runs repeat bit for bit).
template <bool COLS, bool SYM, bool IN_PAIRS>
__global__ void __launch_bounds__(256) k_prerot_apply(const double* __restrict__ inb, const float2* __restrict__ in2b,
                                                      float2* __restrict__ out2b, const int2* __restrict__ entb,
                                                      const int* __restrict__ cntb, const int* __restrict__ mask,
                                                      int dp) {
  constexpr int TL = kPrerotLines;
  extern __shared__ float4 psf4[];
  __shared__ int nheavy;
  const int c = blockIdx.y;
  if (!mask[c]) return;
  const long long DD = (long long)dp * dp;
  const double* in = IN_PAIRS ? nullptr : inb + c * DD;
  const float2* in2 = IN_PAIRS ? in2b + c * DD : nullptr;
  float2* out = out2b + c * DD;
  const float2* vsrc = IN_PAIRS ? in2 : out;  // where the final addition reads v's pairs
  const int2* ent = entb + c * DD;
  const int* cnt = cntb + (long long)c * dp;
  const int l0 = blockIdx.x * TL, nl = min(TL, dp - l0);
  const int TD = TL * dp;
  // four [dp][8] FP32 arrays: P1, P2 = v (hi, lo), then w2 (hi, lo), then P2 = w3; P3, P4 = w1
  // (hi, lo), into which w2 / 2, w3 / 6 and w4 / 24 are folded
  float* P1 = reinterpret_cast<float*>(psf4);
  float* P2 = P1 + TD;
  float* P3 = P2 + TD;
  float* P4 = P3 + TD;
  int* heavy = reinterpret_cast<int*>(P4 + TD);  // [dp]
  int* scnt = heavy + dp;                        // [dp]
  if (threadIdx.x == 0) nheavy = 0;
  // v: element (k, l) of the lines is input[k][l0 + l] (COLS) or input[l0 + l][k]
  if (COLS) {
    for (int e = threadIdx.x; e < TD; e += blockDim.x) {
      const int k = e >> 3, l = e & 7;
      const long long i = (long long)k * dp + l0 + l;
      float2 v = make_float2(0.f, 0.f);
      if (l < nl) {
        if (IN_PAIRS) v = in2[i];
        else out[i] = v = df_split_bits(in[i]);
      }
      P1[e] = v.x;
      P2[e] = v.y;
    }
  } else {
    for (int k = threadIdx.x; k < dp; k += blockDim.x) {
#pragma unroll
      for (int l = 0; l < TL; ++l) {
        const long long i = (long long)(l0 + l) * dp + k;
        float2 v = make_float2(0.f, 0.f);
        if (l < nl) {
          if (IN_PAIRS) v = in2[i];
          else out[i] = v = df_split_bits(in[i]);
        }
        P1[k * TL + l] = v.x;
        P2[k * TL + l] = v.y;
      }
    }
  }
  for (int j = threadIdx.x; j < dp; j += blockDim.x) scnt[j] = cnt[j];
  __syncthreads();
  for (int j = threadIdx.x; j < dp; j += blockDim.x)
    if (scnt[j] > kPrerotLight) heavy[atomicAdd(&nheavy, 1)] = j;
  __syncthreads();
  const int nh = nheavy;
  // w1 = v A -> P3, P4
  prerot_product_df(ent, scnt, heavy, nh, dp, P1, P2, [&](int j, const float* h, const float* lo) {
#pragma unroll
    for (int l = 0; l < TL; ++l) {
      P3[j * TL + l] = h[l];
      P4[j * TL + l] = lo[l];
    }
  });
  __syncthreads();
  // w2 = w1 A -> P1, P2 (v is no longer read)
  prerot_product_df(ent, scnt, heavy, nh, dp, P3, P4, [&](int j, const float* h, const float* lo) {
#pragma unroll
    for (int l = 0; l < TL; ++l) {
      P1[j * TL + l] = h[l];
      P2[j * TL + l] = lo[l];
    }
  });
  __syncthreads();
  // w3 = w2 A from w2's high words (P1, read by every thread); each thread first folds its own
  // entry of w2 / 2 into w1 (two-sum of the high words), then keeps w3 in P2 (its own entry)
  prerot_product_f32(ent, scnt, heavy, nh, dp, P1, [&](int j, const float* u) {
#pragma unroll
    for (int l = 0; l < TL; ++l) {
      const int i = j * TL + l;
      const float a = 0.5f * P1[i];
      const float s = P3[i] + a;
      const float bp = s - P3[i];
      const float err = (P3[i] - (s - bp)) + (a - bp);
      P3[i] = s;
      P4[i] += fmaf(0.5f, P2[i], err);
      P2[i] = u[l];
    }
  });
  __syncthreads();
  // w4 = w3 A; w3 / 6 + w4 / 24 into the low words
  prerot_product_f32(ent, scnt, heavy, nh, dp, P2, [&](int j, const float* u) {
#pragma unroll
    for (int l = 0; l < TL; ++l) {
      const int i = j * TL + l;
      P4[i] += fmaf(u[l], 1.f / 24.f, P2[i] * (1.f / 6.f));
    }
  });
  __syncthreads();
  // v X = v + (P3 + P4): two-sum of the high words, the low words and the error added, renormalised
  auto finish = [&](int k, int l, long long i) -> float2 {
    const float2 v = vsrc[i];
    const float dh = P3[k * TL + l], dl = P4[k * TL + l];
    const float s = v.x + dh;
    const float bp = s - v.x;
    const float err = (v.x - (s - bp)) + (dh - bp);
    const float lo = v.y + dl + err;
    const float hi = s + lo;
    return make_float2(hi, lo - (hi - s));
  };
  if (COLS) {
    for (int e = threadIdx.x; e < TD; e += blockDim.x) {
      const int k = e >> 3, l = e & 7;
      if (l >= nl) continue;
      const long long i = (long long)k * dp + l0 + l;
      const float2 r = finish(k, l, i);
      if (!SYM) {
        out[i] = r;
      } else if (k <= l0 + l) {
        out[i] = r;
        out[(long long)(l0 + l) * dp + k] = r;
      }
    }
  } else {
    for (int k = threadIdx.x; k < dp; k += blockDim.x) {
#pragma unroll
      for (int l = 0; l < TL; ++l) {
        if (l >= nl) continue;
        const long long i = (long long)(l0 + l) * dp + k;
        out[i] = finish(k, l, i);
      }
    }
  }
}

// mask[c] = 1 for the chains that take the pre-rotation (some pair above the tolerance and
// ||A||_F <= kPrerotMaxA)
// (and, where counted, adds the chains and pairs pre-rotated to the eigen-update's counters)
__global__ void k_prerot_mask(const double* __restrict__ acc, int C, int* __restrict__ mask,
                              unsigned long long* __restrict__ counters) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  const int on = (acc[4 * c + 3] > 0.0 && acc[4 * c + 2] <= kPrerotMaxA * kPrerotMaxA) ? 1 : 0;
  mask[c] = on;
  if (counters && on) {
    counters[(long long)kJacStats * c + 6] += 1ull;
    counters[(long long)kJacStats * c + 7] += (unsigned long long)(acc[4 * c + 3] * 0.5);
  }
}

inline unsigned nblk(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// Double-float multiply-add throughput probe: eight independent Dot2 accumulations per thread (the
// inner step of the double-float Jacobi tiles), counted as 2 flops per step.
__global__ void k_df_peak(float* __restrict__ sink, int iters, float2 b) {
  float s[8], c[8];
  float2 a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    s[i] = 0.f;
    c[i] = 0.f;
    a[i] = make_float2(1.0f + threadIdx.x * 1e-3f + i, 1e-9f * i);
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
#pragma unroll
      for (int i = 0; i < 8; ++i) dot2_step(s[i], c[i], a[i], b);
    }
  }
  float t = 0.f;
#pragma unroll
  for (int i = 0; i < 8; ++i) t += s[i] + c[i];
  if (t == 12345.678f) sink[blockIdx.x * blockDim.x + threadIdx.x] = t;
}

rmhmc_status df_peak(void* cuda_stream, int ms_target, double* tflops_host) {
  if (!tflops_host || ms_target < 1) return RMHMC_EINVAL;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = sms * 4, threads = 256;
  float* sink = nullptr;
  if (cudaMalloc(&sink, (size_t)blocks * threads * sizeof(float)) != cudaSuccess) return RMHMC_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const float2 b = make_float2(0.9999f, 1e-8f);
  int iters = 16;
  float ms = 0.f;
  k_df_peak<<<blocks, threads, 0, s>>>(sink, 4, b);
  for (int rep = 0; rep < 12; ++rep) {
    cudaEventRecord(e0, s);
    k_df_peak<<<blocks, threads, 0, s>>>(sink, iters, b);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms >= 0.5f * ms_target || !(ms > 1e-3f)) break;
    iters = (int)fmin(1e7, iters * fmin(100.0, fmax(2.0, 0.8 * ms_target / ms)));
  }
  const double flops = 2.0 * blocks * threads * (double)iters * 16.0 * 8.0;
  *tflops_host = ms > 1e-3f ? flops / (ms * 1e-3) / 1e12 : 0.0;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  return cudaGetLastError() == cudaSuccess ? RMHMC_OK : RMHMC_ECUDA;
}

template <typename T>
rmhmc_status fma_peak(void* cuda_stream, int ms_target, double* tflops_host) {
  if (!tflops_host || ms_target < 1) return RMHMC_EINVAL;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = sms * 4, threads = 256;
  T* sink = nullptr;
  if (cudaMalloc(&sink, (size_t)blocks * threads * sizeof(T)) != cudaSuccess) return RMHMC_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int iters = 64;
  float ms = 0.f;
  k_fma_peak<T><<<blocks, threads, 0, s>>>(sink, 8, (T)0.9999, (T)1e-7);
  for (int rep = 0; rep < 12; ++rep) {
    cudaEventRecord(e0, s);
    k_fma_peak<T><<<blocks, threads, 0, s>>>(sink, iters, (T)0.9999, (T)1e-7);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms >= 0.5f * ms_target || !(ms > 1e-3f)) break;
    iters = (int)fmin(1e7, iters * fmin(100.0, fmax(2.0, 0.8 * ms_target / ms)));
  }
  const double flops = 2.0 * blocks * threads * (double)iters * 16.0 * 8.0;
  *tflops_host = ms > 1e-3f ? flops / (ms * 1e-3) / 1e12 : 0.0;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  return cudaGetLastError() == cudaSuccess ? RMHMC_OK : RMHMC_ECUDA;
}

}  // namespace

// ------------------------------------------------------------------------------------ the model

struct rmhmc_model {
  int device = 0;
  cudaStream_t stream = nullptr;
  ModelDev md{};
  int N = 0, n = 0, P = 0, d = 0, dp = 0, C = 0;
  int cluster = 1;
  int jacobi_sched = RMHMC_JACOBI_CYCLIC;  // rmhmc_jacobi_schedule
  int prerot = 1;  // first-order pre-rotation of warm eigen-updates in the mixed form
  bool cold = false;  // the next eigen-update starts from Psi = I (rmhmc_set_state)
  int tc_nt = 64;  // output tile width of the model's tensor-core GEMMs (64 or 32; rmhmc_autotune)
  bool has_state = false;
  int g_kind = 0, max_sweeps = 30, reorth_every = 10, precision = 0, jacobi_rule = 0, eigen_start = 0;
  double alpha = 1e6, tol = 1e-13;
  uint64_t iter = 0;
  std::vector<void*> allocs;
  // per (chain, kernel) N x N
  double *KL, *D1, *D2, *D3, *Kinv, *S, *Aux, *S2;
  double* spart;  // per (chain, kernel): partial sums of the statistics stages
  double* rdiag;  // per (chain, kernel): the reciprocal pivots of one Cholesky panel (32)
  double* cpart;  // per (chain, kernel): partial sums of the contraction's hyperparameter terms
  // per (chain, kernel) N-vectors
  double *fpk, *alpha_, *beta, *gamma, *eps2, *eps3, *delta, *fuu11;
  double* stats;
  // per chain N-vectors
  double *l0, *l1, *l2, *l3, *lraw;
  // per chain dp x dp
  double *H, *M, *PsiT, *W, *Y, *PsiT_save;
  // per chain dp-vectors
  double *q, *p, *ph, *q0, *v0, *vk, *t1, *dU, *dHdq, *lam, *g, *gp, *q_save, *z, *vtr, *xin;
  // per chain scalars
  double *U, *Ham0, *Ham1, *LL;
  int *status, *sweeps_last, *sweeps_acc, *eig_count, *eig_save, *acc, *sweeps_total;
  JacobiWork jw;
  // kernel-level profile (rmhmc_profile)
  bool prof = false;
  std::vector<cudaEvent_t> ev;
  size_t ev_next = 0;
  struct Rec { int cat; size_t a, b; };
  std::vector<Rec> recs;
  double prof_flops[RMHMC_PROF_NCAT] = {};
  long long prof_launch[RMHMC_PROF_NCAT] = {};
  size_t* plan_bytes = nullptr;  // set only while planning (rmhmc_plan_bytes)
  double *X_dev = nullptr, *y_dev = nullptr, *uf_dev = nullptr, *tau_dev = nullptr;
  // the primal (reduced-rank) model: kind == 1
  int kind = 0;
  PrimalDev pd{};
  double *Phi = nullptr;   // N x P features (shared by the chains)
  double *Z = nullptr;     // C x N x P: diag(l'') Phi, then Phi W[:P, :P]
  double *Fv = nullptr;    // C x N latent values F = Phi w
  double *rvec = nullptr;  // C x N: l''' o rowsum((Phi W) o Phi)
  double *ustat = nullptr; // C x 9: hyperparameter block of the Hessian
  double *Xg_dev = nullptr, *Xl_dev = nullptr;
  double *ld = nullptr;    // J = 2: (9, C, N) likelihood derivatives
  // the mixed form's tensor-core GEMMs: bf16 slices of the current A-side and B-side operands, and
  // of the two Psi^T views that W = Psi^T^T (C Psi^T) reads (kept until Psi^T changes)
  uint8_t *tcA = nullptr, *tcB = nullptr, *tcPA = nullptr, *tcPB = nullptr;
  bool tc_pa_ok = false, tc_pb_ok = false;
  // primal model: slices of Phi^T (the Hessian blocks Phi^T diag(l'') Phi) and of Phi (Phi W in the
  // contraction), split once since Phi is fixed
  uint8_t *tcPhiT = nullptr, *tcPhi = nullptr;
  bool tc_phi_ok = false;
  int* tcmask = nullptr;  // per chain: re-orthonormalisation due at this eigen-update
  // the pre-rotation: X^T M X product scratch (dp x dp per chain), per-chain norms and counts, and
  // the chains that take it
  double* Zp = nullptr;
  double* pr_acc = nullptr;
  int* pr_mask = nullptr;
  int2* pr_ent = nullptr;  // the pre-rotation's row lists (C x dp^2 entries, C x dp lengths)
  int* pr_cnt = nullptr;
};

namespace {

enum Cat {
  CAT_GEMM = 0, CAT_JACOBI, CAT_CHOL, CAT_TRINV, CAT_MODEL, CAT_CONTRACT, CAT_VECTOR, CAT_MGS, CAT_JACOBI_DF,
  CAT_GEMM_TC, CAT_PREROT
};
const char* kCatNames[RMHMC_PROF_NCAT] = {"gemm_f64", "jacobi_f64", "cholesky", "trinv", "model", "contract",
                                          "vector", "reorth", "jacobi_df", "gemm_tc", "prerotation"};

// bf16 slices of the mixed form's tensor-core GEMMs: 9 (63 bits, at or below FP64 GEMM rounding)
// for the K^-1 algebra, whose cond(K) ~ 1e8 amplification needs FP64-level products, and 7 (49 bits,
// the accuracy of the double-float rotations they feed) for the d x d products M = Psi^T H Psi,
// W = Psi C Psi^T and the re-orthonormalisation of Psi^T
constexpr int kSlicesK = 9, kSlicesD = 7;

// The mixed form uses the tensor cores for products whose output is at least one 128-row tile
// each way: below that the slicing launches cost more than the FP64 kernels they replace.
constexpr int kTcMin = 128;
inline bool use_tc(const rmhmc_model* m, int rows, int cols) {
  return m->precision == RMHMC_MIXED && rows >= kTcMin && cols >= kTcMin;
}

// Brackets one launch site with CUDA events on the model's stream while profiling is enabled.
struct ProfScope {
  rmhmc_model* m;
  int cat;
  size_t a = 0;
  bool on = false, once = true;
  ProfScope(rmhmc_model* mm, int c, double flops) : m(mm), cat(c) {
    if (!m->prof) return;
    m->prof_flops[c] += flops;
    m->prof_launch[c] += 1;
    if (m->ev_next + 2 > m->ev.size()) return;
    a = m->ev_next;
    m->ev_next += 2;
    cudaEventRecord(m->ev[a], m->stream);
    on = true;
  }
  ~ProfScope() {
    if (!on) return;
    cudaEventRecord(m->ev[a + 1], m->stream);
    m->recs.push_back({cat, a, a + 1});
  }
};
#define PROF(m, cat, flops) for (ProfScope _ps((m), (cat), (flops)); _ps.once; _ps.once = false)

inline double gemm_flops(double mm, double nn, double kk, bool sym, bool tri) {
  if (tri) return mm * mm * mm / 3.0;
  return sym ? mm * (mm + 1.0) * kk : 2.0 * mm * nn * kk;
}

// The dp x dp products of the eigen-update (M = Psi^T H Psi) and of W = Psi C Psi^T, batched over
// the chains: FP64, or on the tensor cores (gemm_tc, bf16 slices) in the mixed form.
void gemm_dd(rmhmc_model* m, bool ta, bool tb, const double* A, const double* B, double* out, bool sym);

// When planning (m->plan_bytes != nullptr) nothing is allocated: the bytes are only counted.
template <typename T>
rmhmc_status dalloc(rmhmc_model* m, T** p, size_t count) {
  if (m->plan_bytes) {
    *m->plan_bytes += ((count * sizeof(T) + 16 + 255) / 256) * 256;
    *p = nullptr;
    return RMHMC_OK;
  }
  void* ptr = nullptr;
  if (cudaMalloc(&ptr, count * sizeof(T) + 16) != cudaSuccess) return RMHMC_ENOMEM;
  cudaMemsetAsync(ptr, 0, count * sizeof(T) + 16, m->stream);
  m->allocs.push_back(ptr);
  *p = (T*)ptr;
  return RMHMC_OK;
}

rmhmc_status check_launch() {
  return cudaGetLastError() == cudaSuccess ? RMHMC_OK : RMHMC_ECUDA;
}

// The dual model layer: kernel matrices, Cholesky, K^-1 algebra, likelihood maps, U, dU and the
// Hessian; with `third`, also the third-derivative operator (A1, S^2 and the F-phase statistics).
void dual_model_layer(rmhmc_model* m, bool third) {
  cudaStream_t s = m->stream;
  const int N = m->N, n = m->n, C = m->C, dp = m->dp;
  const long long NN = (long long)N * N;
  const int B = C * n;
  const double Nf = N, Bf = B;
  const int ntile = (N + 31) / 32;
  PROF(m, CAT_MODEL, 0)
  dev::k_assemble<<<dim3(ntile * (ntile + 1) / 2, n, C), 256, 0, s>>>(m->md, m->q, dp, m->KL, m->D1, m->D2,
                                                                      m->D3);
  PROF(m, CAT_MODEL, 0)
  dev::k_lik<<<dim3(nblk(N), C), 256, 0, s>>>(m->md, m->q, dp, m->fpk, m->l0, m->l1, m->l2, m->l3, m->lraw);
  const bool tc = use_tc(m, N, N);
  PROF(m, CAT_CHOL, Bf * Nf * Nf * Nf / 3.0) {
    if (tc) cholesky_tc(s, m->KL, N, B, m->stats + ST_LOGDET, kStatSlots, m->status, n, m->tcA, m->tcB, m->rdiag);
    else cholesky_f64(s, m->KL, N, B, m->stats + ST_LOGDET, kStatSlots, m->status, n, m->rdiag);
  }
  PROF(m, CAT_TRINV, Bf * Nf * Nf * Nf / 3.0) {
    if (tc) trinv_lower_tc(s, m->KL, m->Aux, N, B, m->tcA, m->tcB, m->S, m->status, n);
    else trinv_lower_f64(s, m->KL, m->Aux, N, B);
  }
  const TcOperand ka = tc_operand(m->tcA, N, N, kSlicesK, B, false);
  const TcOperand kb = tc_operand(m->tcB, N, N, kSlicesK, B, true);
  // K^-1 = L^-T L^-1 (symmetric; the sum runs over k >= max(i, j) only)
  if (tc) {  // row i of op(A) and row j of op(B)^T are columns of L^-1
    PROF(m, CAT_GEMM_TC, 0) tc_split(s, m->Aux, N, NN, false, B, ka);
    PROF(m, CAT_GEMM_TC, 0) tc_split(s, m->Aux, N, NN, false, B, kb);
    PROF(m, CAT_GEMM_TC, gemm_tc_tensor_flops(ka, kb, B, true, m->tc_nt))
    gemm_tc(s, ka, kb, 1.0, 0.0, m->Kinv, N, NN, B, true, m->status, n, nullptr, m->tc_nt);
  } else {
    PROF(m, CAT_GEMM, Bf * gemm_flops(Nf, Nf, Nf, true, true))
    gemm_f64(s, true, false, N, N, N, 1.0, m->Aux, N, NN, m->Aux, N, NN, 0.0, m->Kinv, N, NN, B, true, true);
  }
  // t = L^-1 f (kept in beta for f . alpha = |t|^2) and alpha = L^-T t by substitution
  PROF(m, CAT_VECTOR, 2.0 * Bf * Nf * Nf)
  cholsolve_f64(s, m->KL, m->fpk, m->beta, m->alpha_, N, B);
  // S = K^-1 D1
  if (tc) {
    PROF(m, CAT_GEMM_TC, 0) tc_split(s, m->Kinv, N, NN, true, B, ka);
    PROF(m, CAT_GEMM_TC, 0) tc_split(s, m->D1, N, NN, false, B, kb);
    PROF(m, CAT_GEMM_TC, gemm_tc_tensor_flops(ka, kb, B, false, m->tc_nt))
    gemm_tc(s, ka, kb, 1.0, 0.0, m->S, N, NN, B, false, m->status, n, nullptr, m->tc_nt);
  } else {
    PROF(m, CAT_GEMM, Bf * gemm_flops(Nf, Nf, Nf, false, false))
    gemm_f64(s, false, false, N, N, N, 1.0, m->Kinv, N, NN, m->D1, N, NN, 0.0, m->S, N, NN, B, false, false);
  }
  if (third && tc) {
    // A1 = S K^-1 (K^-1 is exactly symmetric, so its columns are read as rows), then S^2 with the
    // slices of S's rows reused
    PROF(m, CAT_GEMM_TC, 0) tc_split(s, m->S, N, NN, true, B, ka);
    PROF(m, CAT_GEMM_TC, 0) tc_split(s, m->Kinv, N, NN, true, B, kb);
    PROF(m, CAT_GEMM_TC, gemm_tc_tensor_flops(ka, kb, B, true, m->tc_nt))
    gemm_tc(s, ka, kb, 1.0, 0.0, m->Aux, N, NN, B, true, m->status, n, nullptr, m->tc_nt);
    PROF(m, CAT_GEMM_TC, 0) tc_split(s, m->S, N, NN, false, B, kb);
    PROF(m, CAT_GEMM_TC, gemm_tc_tensor_flops(ka, kb, B, false, m->tc_nt))
    gemm_tc(s, ka, kb, 1.0, 0.0, m->S2, N, NN, B, false, m->status, n, nullptr, m->tc_nt);
  } else if (third) {
    PROF(m, CAT_GEMM, Bf * gemm_flops(Nf, Nf, Nf, true, false))
    gemm_f64(s, false, false, N, N, N, 1.0, m->S, N, NN, m->Kinv, N, NN, 0.0, m->Aux, N, NN, B, true, false);
    PROF(m, CAT_GEMM, Bf * gemm_flops(Nf, Nf, Nf, false, false))
    gemm_f64(s, false, false, N, N, N, 1.0, m->S, N, NN, m->S, N, NN, 0.0, m->S2, N, NN, B, false, false);
  }
  const dim3 sg((N + dev::kStatCols - 1) / dev::kStatCols, B);
  if (third) {
    PROF(m, CAT_MODEL, 0)
    dev::k_stats_cols<true><<<sg, 256, 0, s>>>(N, m->D1, m->D2, m->D3, m->Kinv, m->Aux, m->alpha_, m->beta,
                                               m->eps2, m->eps3, m->spart);
    PROF(m, CAT_MODEL, 0)
    dev::k_stats_gamma<true><<<sg, 256, 0, s>>>(N, m->Kinv, m->S, m->S2, m->beta, m->eps2, m->gamma, m->spart);
    PROF(m, CAT_MODEL, 0)
    dev::k_stats_delta<<<sg, 256, 0, s>>>(N, m->D1, m->alpha_, m->gamma, m->delta, m->spart);
    PROF(m, CAT_MODEL, 0)
    dev::k_stats_fuu<<<sg, 256, 0, s>>>(N, m->Kinv, m->delta, m->eps2, m->fuu11);
  } else {
    PROF(m, CAT_MODEL, 0)
    dev::k_stats_cols<false><<<sg, 256, 0, s>>>(N, m->D1, m->D2, m->D3, m->Kinv, m->Aux, m->alpha_, m->beta,
                                                m->eps2, m->eps3, m->spart);
    PROF(m, CAT_MODEL, 0)
    dev::k_stats_gamma<false><<<sg, 256, 0, s>>>(N, m->Kinv, m->S, m->S2, m->beta, m->eps2, m->gamma,
                                                 m->spart);
  }
  PROF(m, CAT_MODEL, 0)
  dev::k_stats_reduce<<<B, 32, 0, s>>>((int)sg.x, third ? 1 : 0, m->spart, m->stats);
  PROF(m, CAT_MODEL, 0)
  dev::k_udu<<<C, 256, 0, s>>>(m->md, m->q, dp, m->l0, m->l1, m->lraw, m->alpha_, m->stats, m->U,
                               m->dU, m->LL);
  const long long DD = (long long)dp * dp;
  PROF(m, CAT_MODEL, 0)
  dev::k_hessian<<<dim3(nblk(DD), C), 256, 0, s>>>(m->md, m->q, dp, m->Kinv, m->l2, m->alpha_,
                                                   m->gamma, m->stats, m->H);
}

// The primal model layer: F = Phi w, likelihood maps, U and dU (Phi^T l' + prior), the Hessian
// (Phi^T diag(l'') Phi + prior). The third-derivative operator needs only l''' (kept in l3).
// The primal model's fixed feature matrix, sliced once for the tensor-core GEMMs: op(A) = Phi^T
// (P rows over the N samples: the Hessian blocks) or Phi (N rows over the P features: Phi W).
TcOperand phi_operand(rmhmc_model* m, bool transposed) {
  const int N = m->N, P = m->pd.P;
  TcOperand op = transposed ? tc_operand(m->tcPhiT, P, N, kSlicesK, 1, false)
                            : tc_operand(m->tcPhi, N, P, kSlicesK, 1, false);
  op.shared = true;
  return op;
}

void primal_phi_slices(rmhmc_model* m) {
  if (m->tc_phi_ok) return;
  const int P = m->pd.P;
  PROF(m, CAT_GEMM_TC, 0) tc_split(m->stream, m->Phi, P, 0, false, 1, phi_operand(m, true));
  PROF(m, CAT_GEMM_TC, 0) tc_split(m->stream, m->Phi, P, 0, true, 1, phi_operand(m, false));
  m->tc_phi_ok = true;
}

void primal_model_layer(rmhmc_model* m) {
  cudaStream_t s = m->stream;
  const int N = m->N, C = m->C, dp = m->dp, P = m->pd.P, J = m->pd.J;
  const long long NP = (long long)N * P, DD = (long long)dp * dp, CN = (long long)C * N;
  const double Nf = N, Pf = P, Cf = C;
  for (int j = 0; j < J; ++j) {
    PROF(m, CAT_GEMM, 2.0 * Cf * Nf * Pf)
    gemm_f64(s, false, true, C, N, P, 1.0, m->q + j * P, dp, 0, m->Phi, P, 0, 0.0, m->Fv + j * CN, N, 0, 1,
             false, false);
  }
  if (J == 1) {
    PROF(m, CAT_MODEL, 0)
    dev::k_lik_primal<<<dim3(nblk(N), C), 256, 0, s>>>(m->pd, m->Fv, m->l0, m->l1, m->l2, m->l3, m->lraw);
  } else {
    PROF(m, CAT_MODEL, 0)
    dev::k_lik_meanvar<<<dim3(nblk(N), C), 256, 0, s>>>(m->pd, m->Fv, m->l0, m->lraw, m->ld);
  }
  for (int j = 0; j < J; ++j) {
    const double* lj = J == 1 ? m->l1 : m->ld + j * CN;
    PROF(m, CAT_GEMM, 2.0 * Cf * Nf * Pf)
    gemm_f64(s, false, false, C, P, N, 1.0, lj, N, 0, m->Phi, P, 0, 0.0, m->dU + j * P, dp, 0, 1, false, false);
  }
  PROF(m, CAT_MODEL, 0)
  dev::k_primal_udu<<<C, 256, 0, s>>>(m->pd, m->q, dp, m->l0, m->lraw, m->U, m->dU, m->LL, m->ustat);
  // the likelihood blocks Phi^T diag(l_jk) Phi of the Hessian ((j, k) and its mirror (k, j))
  const bool tc = use_tc(m, P, P);
  if (tc) primal_phi_slices(m);
  for (int j = 0; j < J; ++j) {
    for (int k = j; k < J; ++k) {
      const double* ljk = J == 1 ? m->l2 : m->ld + (2 + j + k) * CN;
      PROF(m, CAT_MODEL, 0)
      dev::k_rowscale<<<dim3(nblk(NP), C), 256, 0, s>>>(m->pd, ljk, m->Phi, m->Z);
      if (tc) {  // op(A) = Phi^T (shared slices), op(B) = Z = diag(l_jk) Phi: its columns
        const TcOperand pa = phi_operand(m, true);
        const TcOperand zb = tc_operand(m->tcB, P, N, kSlicesK, C, true);
        PROF(m, CAT_GEMM_TC, 0) tc_split(s, m->Z, P, NP, false, C, zb);
        PROF(m, CAT_GEMM_TC, gemm_tc_tensor_flops(pa, zb, C, true, m->tc_nt) * (k != j ? 2 : 1))
        {
          gemm_tc(s, pa, zb, 1.0, 0.0, m->H + (long long)j * P * dp + k * P, dp, DD, C, true, m->status, 1, nullptr, m->tc_nt);
          if (k != j)
            gemm_tc(s, pa, zb, 1.0, 0.0, m->H + (long long)k * P * dp + j * P, dp, DD, C, true, m->status, 1, nullptr, m->tc_nt);
        }
        continue;
      }
      PROF(m, CAT_GEMM, Cf * gemm_flops(Pf, Pf, Nf, true, false))
      gemm_f64(s, true, false, P, P, N, 1.0, m->Phi, P, 0, m->Z, P, NP, 0.0, m->H + (long long)j * P * dp + k * P,
               dp, DD, C, true, false);
      if (k != j) {
        PROF(m, CAT_GEMM, Cf * gemm_flops(Pf, Pf, Nf, true, false))
        gemm_f64(s, true, false, P, P, N, 1.0, m->Phi, P, 0, m->Z, P, NP, 0.0,
                 m->H + (long long)k * P * dp + j * P, dp, DD, C, true, false);
      }
    }
  }
  PROF(m, CAT_MODEL, 0)
  dev::k_primal_hess<<<dim3(nblk(DD), C), 256, 0, s>>>(m->pd, m->q, dp, m->ustat, m->H);
}

// --- geometry at the current q: U, dU, Hessian, warm-started eigendecomposition, g(lambda);
//     with `third`, also the third-derivative operator (the dual model's A1, S^2 and F-phase
//     statistics; the primal model needs no more than l''').
// The first-order pre-rotation of a warm eigen-update (see k_prerot_rows). A holds a few percent
// of nonzeros, so X is applied from the lists of A's rows (pr_ent, pr_cnt), for the chains in
// pr_mask: Z = M X into Zp (double-float pairs), X^T Z into the Jacobi's pair buffer for M (W) and
// X^T Psi^T into its pair buffer for Psi^T (Y); the double-float Jacobi then starts from those pairs
// for these chains. Eight lines per CTA, whose buffers (16 TL dp + 8 dp bytes) fit the 226 KB of
// shared memory up to dp = 1701; beyond it the pre-rotation is not taken.
inline size_t prerot_smem(int TL, int dp) { return (size_t)16 * TL * dp + (size_t)8 * dp; }
bool prerot_fits(int dp) { return prerot_smem(kPrerotLines, dp) <= (size_t)226 * 1024; }

void prerot_apply_all(rmhmc_model* m) {
  cudaStream_t s = m->stream;
  const int C = m->C, dp = m->dp;
  const size_t smem = prerot_smem(kPrerotLines, dp);
  // (the opt-in limit covers the kernel's static shared memory too: ask for what this launch needs)
  static size_t attr_bytes = 0;
  if (smem > attr_bytes) {
    cudaFuncSetAttribute(k_prerot_apply<false, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_prerot_apply<true, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_prerot_apply<true, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr_bytes = smem;
  }
  const dim3 grid((dp + kPrerotLines - 1) / kPrerotLines, C);
  const int* mk = m->pr_mask;
  float2* Z2 = reinterpret_cast<float2*>(m->Zp);
  PROF(m, CAT_PREROT, 0)
  k_prerot_apply<false, false, false><<<grid, 256, smem, s>>>(m->M, nullptr, Z2, m->pr_ent, m->pr_cnt, mk, dp);
  PROF(m, CAT_PREROT, 0)
  k_prerot_apply<true, true, true><<<grid, 256, smem, s>>>(nullptr, Z2, reinterpret_cast<float2*>(m->W), m->pr_ent,
                                                           m->pr_cnt, mk, dp);
  PROF(m, CAT_PREROT, 0)
  k_prerot_apply<true, false, false><<<grid, 256, smem, s>>>(m->PsiT, nullptr, reinterpret_cast<float2*>(m->Y),
                                                             m->pr_ent, m->pr_cnt, mk, dp);
}

void prerotate(rmhmc_model* m) {
  cudaStream_t s = m->stream;
  const int C = m->C, dp = m->dp, d = m->d;
  double* part = m->pr_acc + 4 * C;
  PROF(m, CAT_PREROT, 0)
  k_prerot_norms<<<dim3(kPrerotParts, C), 256, 0, s>>>(m->M, dp, d, m->pr_acc, part);
  PROF(m, CAT_PREROT, 0)
  k_prerot_rows<<<dim3((dp + 7) / 8, C), 256, 0, s>>>(m->M, part, dp, d, m->jacobi_rule, m->tol, m->status,
                                                      m->pr_ent, m->pr_cnt, m->pr_acc);
  PROF(m, CAT_PREROT, 0)
  k_prerot_mask<<<nblk(C), 256, 0, s>>>(m->pr_acc, C, m->pr_mask, m->jw.tiles);
  prerot_apply_all(m);
}

void eval_geometry(rmhmc_model* m, bool third) {
  cudaStream_t s = m->stream;
  const int C = m->C, dp = m->dp, d = m->d;
  const long long DD = (long long)dp * dp;
  m->tc_pa_ok = m->tc_pb_ok = false;  // Gram-Schmidt or the cold start may change Psi^T
  if (m->kind == 1) primal_model_layer(m);
  else dual_model_layer(m, third);
  // Sec. 2.4: Gram-Schmidt of Psi every reorth_every eigen-updates, then M = Psi^T H Psi
  // (the static ablation restarts every eigen-update from Psi = I instead)
  if (m->eigen_start == 1) {
    PROF(m, CAT_VECTOR, 0)
    k_set_identity<<<nblk((long long)C * DD), 256, 0, s>>>(m->PsiT, dp, C);
  } else if (m->reorth_every > 0 && use_tc(m, d, d)) {
    // one Newton-Schulz (polar) step P <- 1.5 P - 0.5 (P P^T) P on the first d rows of Psi^T, on
    // the tensor cores, for the chains that are due (the others skip every kernel)
    const int S = kSlicesD;
    PROF(m, CAT_MGS, 0)
    k_reorth_mask<<<nblk(C), 256, 0, s>>>(m->eig_count, m->reorth_every, C, m->tcmask);
    TcOperand pa = tc_operand(m->tcA, d, dp, S, C, false), pb = tc_operand(m->tcB, d, dp, S, C, true);
    PROF(m, CAT_MGS, 0) tc_split(s, m->PsiT, dp, DD, true, C, pa, m->tcmask);
    PROF(m, CAT_MGS, 0) tc_split(s, m->PsiT, dp, DD, true, C, pb, m->tcmask);
    PROF(m, CAT_MGS, 0) gemm_tc(s, pa, pb, 1.0, 0.0, m->Y, dp, DD, C, true, m->status, 1, m->tcmask, m->tc_nt);
    pa = tc_operand(m->tcA, d, d, S, C, false);
    pb = tc_operand(m->tcB, dp, d, S, C, true);
    PROF(m, CAT_MGS, 0) tc_split(s, m->Y, dp, DD, true, C, pa, m->tcmask);
    PROF(m, CAT_MGS, 0) tc_split(s, m->PsiT, dp, DD, false, C, pb, m->tcmask);
    PROF(m, CAT_MGS, 0) gemm_tc(s, pa, pb, -0.5, 1.5, m->PsiT, dp, DD, C, false, m->status, 1, m->tcmask, m->tc_nt);
  } else if (m->reorth_every > 0) {
    PROF(m, CAT_MGS, 0)
    mgs_rows_f64(s, m->PsiT, dp, d, C, m->eig_count, m->reorth_every, m->cluster);
  }
  gemm_dd(m, false, true, m->H, m->PsiT, m->Y, false);
  gemm_dd(m, false, false, m->PsiT, m->Y, m->M, true);
  // a cold start (Psi = I: rmhmc_set_state, or every update of the static ablation) takes the
  // cyclic order: the dynamic order's greedy matching is for the few couplings a warm start leaves
  // (on the dual model's cold start it can exceed the round limit), and the pre-rotation needs small
  // angles
  const bool cold = m->cold || m->eigen_start == 1;
  const int sched = cold ? RMHMC_JACOBI_CYCLIC : m->jacobi_sched;
  // (the pre-rotation is for the mixed form, whose Jacobi works in double-float pairs)
  const bool pre = m->prerot && !cold && use_tc(m, dp, dp) && prerot_fits(dp);
  if (pre) prerotate(m);
  if (m->precision == RMHMC_MIXED) {
    // rotations in double-float pairs; W and Y serve as the pair buffers (free during the update),
    // already filled by the pre-rotation for the chains in pr_mask
    PROF(m, CAT_JACOBI_DF, 0)
    jacobi_df(s, m->M, m->PsiT, m->lam, dp, d, C, m->jacobi_rule, m->tol, m->max_sweeps, m->status,
              m->sweeps_last, m->sweeps_acc, m->jw, m->cluster, m->W, m->Y, sched, pre ? m->pr_mask : nullptr);
  } else {
    PROF(m, CAT_JACOBI, 0)
    jacobi_f64(s, m->M, m->PsiT, m->lam, dp, d, C, m->jacobi_rule, m->tol, m->max_sweeps, m->status,
               m->sweeps_last, m->sweeps_acc, m->jw, m->cluster, sched);
  }
  m->tc_pa_ok = m->tc_pb_ok = false;  // the eigen-update rotated Psi^T
  PROF(m, CAT_VECTOR, 0)
  k_inc<<<nblk(C), 256, 0, s>>>(m->eig_count, C, m->sweeps_total, m->sweeps_last);
  PROF(m, CAT_VECTOR, 0)
  k_softabs<<<nblk((long long)C * dp), 256, 0, s>>>(m->lam, m->g, m->gp, dp, d, C, m->alpha, m->g_kind);
}

void gemm_dd(rmhmc_model* m, bool ta, bool tb, const double* A, const double* B, double* out, bool sym) {
  const int dp = m->dp;
  const long long DD = (long long)dp * dp;
  const double df = m->d, fl = m->C * gemm_flops(df, df, df, sym, false);
  if (use_tc(m, dp, dp)) {
    // tensor cores: op(A)'s rows and op(B)'s columns cut into bf16 slices; the two column views
    // of Psi^T (W = Psi^T^T (C Psi^T)) are kept until Psi^T changes
    const bool pa = A == m->PsiT && ta, pb = B == m->PsiT && !tb;
    const TcOperand oa = tc_operand(pa ? m->tcPA : m->tcA, dp, dp, kSlicesD, m->C, false);
    const TcOperand ob = tc_operand(pb ? m->tcPB : m->tcB, dp, dp, kSlicesD, m->C, true);
    if (!pa || !m->tc_pa_ok) {
      PROF(m, CAT_GEMM_TC, 0) tc_split(m->stream, A, dp, DD, !ta, m->C, oa);
      if (pa) m->tc_pa_ok = true;
    }
    if (!pb || !m->tc_pb_ok) {
      PROF(m, CAT_GEMM_TC, 0) tc_split(m->stream, B, dp, DD, tb, m->C, ob);
      if (pb) m->tc_pb_ok = true;
    }
    PROF(m, CAT_GEMM_TC, gemm_tc_tensor_flops(oa, ob, m->C, sym, m->tc_nt))
    gemm_tc(m->stream, oa, ob, 1.0, 0.0, out, dp, DD, m->C, sym, m->status, 1, nullptr, m->tc_nt);
  } else {
    PROF(m, CAT_GEMM, fl)
    gemm_f64(m->stream, ta, tb, dp, dp, dp, 1.0, A, dp, DD, B, dp, DD, 0.0, out, dp, DD, m->C, sym, false);
  }
}

// out = G^-1 x = Psi diag(1/g) Psi^T x
void ginv(rmhmc_model* m, const double* x, double* out) {
  cudaStream_t s = m->stream;
  const int dp = m->dp, C = m->C;
  const long long DD = (long long)dp * dp;
  const double v2 = 2.0 * C * (double)m->d * m->d;
  PROF(m, CAT_VECTOR, v2)
  gemv_f64(s, false, dp, dp, m->PsiT, dp, DD, x, dp, m->t1, dp, C, 1.0, 0.0);
  PROF(m, CAT_VECTOR, 0)
  k_scale_g<<<nblk((long long)C * dp), 256, 0, s>>>(m->t1, m->g, dp, m->d, C, 0);
  PROF(m, CAT_VECTOR, v2)
  gemv_f64(s, true, dp, dp, m->PsiT, dp, DD, m->t1, dp, out, dp, C, 1.0, 0.0);
}

// out = dH/dq(q, x) = dU + tr((W2 - W1) dH_i) / 2
void grad_h(rmhmc_model* m, const double* x, double* out) {
  cudaStream_t s = m->stream;
  const int dp = m->dp, C = m->C, N = m->N, n = m->n;
  const long long DD = (long long)dp * dp;
  const double df = m->d, Cf = C;
  PROF(m, CAT_VECTOR, 2.0 * Cf * df * df)
  gemv_f64(s, false, dp, dp, m->PsiT, dp, DD, x, dp, m->t1, dp, C, 1.0, 0.0);
  const int ct = (dp + 31) / 32;
  PROF(m, CAT_VECTOR, 0)
  k_build_c<<<dim3(ct * (ct + 1) / 2, C), 256, 0, s>>>(m->t1, m->lam, m->g, m->gp, m->M, dp, m->d, m->alpha,
                                                       m->g_kind);
  // W = Psi C Psi^T = PsiT^T (C PsiT)
  gemm_dd(m, false, false, m->M, m->PsiT, m->Y, false);
  gemm_dd(m, true, false, m->PsiT, m->Y, m->W, true);
  if (m->kind == 1) {
    // Sec. 2.3 ordering: v_j = Phi^T [sum_kl l_jkl o rowsum((Phi W_kl) o Phi)] + the prior parts
    const int P = m->pd.P, J = m->pd.J;
    const long long NP = (long long)N * P, CN = (long long)C * N;
    const double Nf = N, Pf = P;
    for (int j = 0; j < J; ++j) {
      for (int k = j; k < J; ++k) {
        const double* Wjk = m->W + (long long)j * P * dp + k * P;
        if (use_tc(m, N, P)) {  // op(A) = Phi (shared slices), op(B) = W_jk: its columns
          primal_phi_slices(m);
          const TcOperand pa = phi_operand(m, false);
          const TcOperand wb = tc_operand(m->tcB, P, P, kSlicesK, C, true);
          PROF(m, CAT_GEMM_TC, 0) tc_split(s, Wjk, dp, DD, false, C, wb);
          PROF(m, CAT_GEMM_TC, gemm_tc_tensor_flops(pa, wb, C, false, m->tc_nt))
          gemm_tc(s, pa, wb, 1.0, 0.0, m->Z, P, NP, C, false, m->status, 1, nullptr, m->tc_nt);
        } else {
          PROF(m, CAT_GEMM, 2.0 * Cf * Nf * Pf * Pf)
          gemm_f64(s, false, false, N, P, P, 1.0, m->Phi, P, 0, Wjk, dp, DD, 0.0, m->Z, P, NP, C, false, false);
        }
        PROF(m, CAT_CONTRACT, 2.0 * Cf * Nf * Pf)
        dev::k_primal_rowdot<<<dim3((N + 7) / 8, C), 256, 0, s>>>(m->pd, m->Z, m->Phi, J == 1 ? m->l3 : nullptr,
                                                                   m->rvec + (j + k) * CN);
      }
    }
    if (J == 2) {
      PROF(m, CAT_CONTRACT, 0)
      dev::k_mv_combine<<<nblk(CN), 256, 0, s>>>(m->pd, m->rvec, m->ld, m->rvec + 3 * CN);
    }
    for (int j = 0; j < J; ++j) {
      PROF(m, CAT_GEMM, 2.0 * Cf * Nf * Pf)
      gemm_f64(s, false, false, C, P, N, 1.0, m->rvec + (J == 1 ? 0 : (3 + j) * CN), N, 0, m->Phi, P, 0, 0.0,
               m->vtr + j * P, dp, 0, 1, false, false);
    }
    PROF(m, CAT_CONTRACT, 0)
    dev::k_primal_contract<<<C, 256, 0, s>>>(m->pd, m->q, dp, m->W, m->vtr);
  } else {
    const dim3 cg((N + dev::kStatCols - 1) / dev::kStatCols, C * n);
    PROF(m, CAT_CONTRACT, 0)
    dev::k_contract<<<cg, 256, 2 * N * sizeof(double), s>>>(m->md, m->q, dp, m->W, m->Kinv, m->Aux, m->l3,
                                                            m->alpha_, m->gamma, m->fuu11, m->vtr, m->cpart);
    PROF(m, CAT_CONTRACT, 0)
    dev::k_contract_hyp<<<C * n, 32, 0, s>>>(m->md, m->q, dp, m->W, m->stats, m->cpart, (int)cg.x, m->vtr);
  }
  PROF(m, CAT_VECTOR, 0)
  k_axpy<<<nblk((long long)C * dp), 256, 0, s>>>(out, m->dU, m->vtr, 0.5, (long long)C * dp);
}

void hamiltonian(rmhmc_model* m, const double* x, double* Ham) {
  ginv(m, x, m->vk);
  PROF(m, CAT_VECTOR, 0)
  k_hamiltonian<<<m->C, 256, 0, m->stream>>>(m->U, m->g, x, m->vk, m->dp, m->d, Ham);
}

// One generalized leapfrog (Eq. leapfrog) from the geometry at q (third-derivative operator ready).
void leapfrog_step(rmhmc_model* m, double eps, int n_fp) {
  cudaStream_t s = m->stream;
  const long long nv = (long long)m->C * m->dp;
  const unsigned g = nblk(nv);
  cudaMemcpyAsync(m->ph, m->p, nv * sizeof(double), cudaMemcpyDeviceToDevice, s);
  for (int k = 0; k < n_fp; ++k) {
    grad_h(m, m->ph, m->dHdq);
    PROF(m, CAT_VECTOR, 0)
    k_axpy<<<g, 256, 0, s>>>(m->ph, m->p, m->dHdq, -0.5 * eps, nv);
  }
  ginv(m, m->ph, m->v0);
  cudaMemcpyAsync(m->q0, m->q, nv * sizeof(double), cudaMemcpyDeviceToDevice, s);
  for (int k = 0; k < n_fp; ++k) {
    if (k == 0) {
      PROF(m, CAT_VECTOR, 0)
      k_axpy2<<<g, 256, 0, s>>>(m->q, m->q0, m->v0, m->v0, 0.5 * eps, nv);
    } else {
      eval_geometry(m, false);
      ginv(m, m->ph, m->vk);
      PROF(m, CAT_VECTOR, 0)
      k_axpy2<<<g, 256, 0, s>>>(m->q, m->q0, m->v0, m->vk, 0.5 * eps, nv);
    }
  }
  eval_geometry(m, true);
  grad_h(m, m->ph, m->dHdq);
  PROF(m, CAT_VECTOR, 0)
  k_axpy<<<g, 256, 0, s>>>(m->p, m->ph, m->dHdq, -0.5 * eps, nv);
}

// Every device buffer of a model, in one place for allocation and for rmhmc_plan_bytes.
rmhmc_status allocate_model(rmhmc_model* m, int n_cov) {
  const int N = m->N, n = m->n, C = m->C, dp = m->dp;
  const size_t NN = (size_t)N * N, DD = (size_t)dp * dp;
  const size_t B = (size_t)C * n;
  rmhmc_status st = RMHMC_OK;
#define ALLOC(ptr, cnt) \
  if (st == RMHMC_OK) st = dalloc(m, &(ptr), (cnt))
  ALLOC(m->y_dev, (size_t)N);
  ALLOC(m->tau_dev, (size_t)C);
  if (m->kind == 1) {
    const size_t P = (size_t)m->pd.P;
    if (m->pd.Dg) ALLOC(m->Xg_dev, (size_t)N * m->pd.Dg);
    if (m->pd.Dl) ALLOC(m->Xl_dev, (size_t)N * m->pd.Dl);
    const size_t J = (size_t)m->pd.J;
    ALLOC(m->Phi, (size_t)N * P);
    ALLOC(m->Z, (size_t)C * N * P);
    ALLOC(m->Fv, J * C * N);
    ALLOC(m->rvec, (J == 1 ? 1 : 5) * (size_t)C * N);  // J = 2: s_00, s_01, s_11, r_0, r_1
    ALLOC(m->ustat, (size_t)C * 9);
    if (J == 2) ALLOC(m->ld, (size_t)9 * C * N);
  } else {
    ALLOC(m->X_dev, (size_t)N * n_cov);
    ALLOC(m->uf_dev, (size_t)2 * n);
    ALLOC(m->KL, B * NN);
    ALLOC(m->D1, B * NN);
    ALLOC(m->D2, B * NN);
    ALLOC(m->D3, B * NN);
    ALLOC(m->spart, B * dev::kStatMaxBlocks * ST_COUNT);
    ALLOC(m->rdiag, B * 32);
    ALLOC(m->cpart, B * dev::kStatMaxBlocks * dev::kContractParts);
    ALLOC(m->Kinv, B * NN);
    ALLOC(m->S, B * NN);
    ALLOC(m->Aux, B * NN);
    ALLOC(m->S2, B * NN);
    ALLOC(m->fpk, B * N);
    ALLOC(m->alpha_, B * N);
    ALLOC(m->beta, B * N);
    ALLOC(m->gamma, B * N);
    ALLOC(m->eps2, B * N);
    ALLOC(m->eps3, B * N);
    ALLOC(m->delta, B * N);
    ALLOC(m->fuu11, B * N);
    ALLOC(m->stats, B * kStatSlots);
  }
  ALLOC(m->l0, (size_t)C * N);
  ALLOC(m->l1, (size_t)C * N);
  ALLOC(m->l2, (size_t)C * N);
  ALLOC(m->l3, (size_t)C * N);
  ALLOC(m->lraw, (size_t)C * N);
  ALLOC(m->H, C * DD);
  ALLOC(m->M, C * DD);
  ALLOC(m->PsiT, C * DD);
  ALLOC(m->W, C * DD);
  ALLOC(m->Y, C * DD);
  ALLOC(m->PsiT_save, C * DD);
  {  // tensor-core slices: the K^-1 algebra (dual model) and the d x d products share tcA / tcB
    size_t ba = tc_operand_bytes(dp, dp, kSlicesD, C, false), bb = tc_operand_bytes(dp, dp, kSlicesD, C, true);
    if (m->kind != 1) {
      ba = std::max(ba, tc_operand_bytes(N, N, kSlicesK, (int)B, false));
      bb = std::max(bb, tc_operand_bytes(N, N, kSlicesK, (int)B, true));
    } else {  // Z = diag(l) Phi and the W blocks as B operands; Phi^T and Phi kept
      const int P = m->pd.P;
      bb = std::max(bb, tc_operand_bytes(P, N, kSlicesK, C, true));
      bb = std::max(bb, tc_operand_bytes(P, P, kSlicesK, C, true));
      ALLOC(m->tcPhiT, tc_operand_bytes(P, N, kSlicesK, 1, false));
      ALLOC(m->tcPhi, tc_operand_bytes(N, P, kSlicesK, 1, false));
    }
    ALLOC(m->tcA, ba);
    ALLOC(m->tcB, bb);
    ALLOC(m->tcPA, tc_operand_bytes(dp, dp, kSlicesD, C, false));
    ALLOC(m->tcPB, tc_operand_bytes(dp, dp, kSlicesD, C, true));
  }
  double** vecs[] = {&m->q, &m->p, &m->ph, &m->q0, &m->v0, &m->vk, &m->t1, &m->dU, &m->dHdq,
                     &m->lam, &m->g, &m->gp, &m->q_save, &m->z, &m->vtr, &m->xin};
  for (double** v : vecs) ALLOC(*v, (size_t)C * dp);
  ALLOC(m->U, (size_t)C);
  ALLOC(m->Ham0, (size_t)C);
  ALLOC(m->Ham1, (size_t)C);
  ALLOC(m->LL, (size_t)C);
  int** ivecs[] = {&m->status, &m->sweeps_last, &m->sweeps_acc, &m->eig_count, &m->eig_save, &m->acc,
                   &m->sweeps_total, &m->tcmask};
  for (int** v : ivecs) ALLOC(*v, (size_t)C);
  const int np = dp / kJacBlk / 2;
  ALLOC(m->jw.V, (size_t)C * np * 256);
  ALLOC(m->jw.D, (size_t)C * np * 256);
  ALLOC(m->jw.slots, (size_t)C * 64);
  ALLOC(m->jw.flags, (size_t)C * np);
  ALLOC(m->jw.tiles, (size_t)kJacStats * C);
  ALLOC(m->jw.crit, (size_t)C * (dp / kJacBlk) * (dp / kJacBlk));
  ALLOC(m->Zp, (size_t)C * DD);
  ALLOC(m->pr_acc, (size_t)(4 + 2 * kPrerotParts) * C);
  ALLOC(m->pr_mask, (size_t)C);
  ALLOC(m->pr_ent, (size_t)C * DD);
  ALLOC(m->pr_cnt, (size_t)C * dp);
#undef ALLOC
  return st;
}

rmhmc_status check_integ(const rmhmc_model* m, const rmhmc_integrator* in, bool for_state) {
  if (!in) return RMHMC_EINVAL;
  if (in->precision != RMHMC_FP64 && in->precision != RMHMC_MIXED) return RMHMC_EINVAL;
  if (in->g_kind != RMHMC_G_COTH && in->g_kind != RMHMC_G_SQRT) return RMHMC_EINVAL;
  if (!(in->alpha > 0.0) || !(in->jacobi_tol > 0.0) || in->max_sweeps < 0 || in->reorth_every < 0)
    return RMHMC_EINVAL;
  if (in->jacobi_rule != RMHMC_JACOBI_METRIC && in->jacobi_rule != RMHMC_JACOBI_RELATIVE)
    return RMHMC_EINVAL;
  if (in->eigen_start != 0 && in->eigen_start != 1) return RMHMC_EINVAL;
  if (!for_state) {
    if (!m->has_state) return RMHMC_EINVAL;
    if (in->g_kind != m->g_kind || in->alpha != m->alpha || in->jacobi_tol != m->tol ||
        in->precision != m->precision ||
        in->max_sweeps != m->max_sweeps || in->reorth_every != m->reorth_every ||
        in->jacobi_rule != m->jacobi_rule || in->eigen_start != m->eigen_start)
      return RMHMC_EINVAL;
    if (!(in->eps > 0.0) || in->n_fp < 1) return RMHMC_EINVAL;
  }
  return RMHMC_OK;
}

}  // namespace

// ------------------------------------------------------------------------- uneven batches

struct rmhmc_batch {
  std::vector<rmhmc_model*> models;
  cudaStream_t stream = nullptr;
  cudaEvent_t fork = nullptr, post = nullptr;
  std::vector<cudaEvent_t> joins, pre;
  cudaGraphExec_t exec = nullptr;
  double eps = 0.0;
  int n_fp = 0;
};

// ----------------------------------------------------------------------------------- C ABI

extern "C" {

rmhmc_status rmhmc_batch_create(rmhmc_model* const* models, int n_models, void* cuda_stream,
                                rmhmc_batch** out) {
  if (!models || n_models < 1 || !out) return RMHMC_EINVAL;
  *out = nullptr;
  cudaStream_t bs = (cudaStream_t)cuda_stream;
  if (bs == nullptr) return RMHMC_EINVAL;  // the legacy default stream cannot be captured
  for (int i = 0; i < n_models; ++i) {
    rmhmc_model* m = models[i];
    if (!m || !m->has_state || m->stream == nullptr || m->stream == bs) return RMHMC_EINVAL;
    for (int j = 0; j < i; ++j)
      if (models[j] == m || models[j]->stream == m->stream) return RMHMC_EINVAL;
  }
  rmhmc_batch* b = new rmhmc_batch();
  b->models.assign(models, models + n_models);
  b->stream = bs;
  b->joins.resize(n_models);
  b->pre.resize(n_models);
  bool ok = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->post, cudaEventDisableTiming) == cudaSuccess;
  for (auto& e : b->joins) ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
  for (auto& e : b->pre) ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    rmhmc_batch_free(b);
    return RMHMC_ECUDA;
  }
  *out = b;
  return RMHMC_OK;
}

void rmhmc_batch_free(rmhmc_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->post) cudaEventDestroy(b->post);
  for (cudaEvent_t e : b->joins)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : b->pre)
    if (e) cudaEventDestroy(e);
  delete b;
}

rmhmc_status rmhmc_batch_leapfrog(rmhmc_batch* b, const rmhmc_integrator* integ, int n_steps) {
  if (!b || n_steps < 0) return RMHMC_EINVAL;
  for (rmhmc_model* m : b->models) {
    rmhmc_status st = check_integ(m, integ, false);
    if (st != RMHMC_OK) return st;
    if (m->prof) return RMHMC_EINVAL;
  }
  if (!b->exec || b->eps != integ->eps || b->n_fp != integ->n_fp) {
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      return RMHMC_ECUDA;
    }
    cudaEventRecord(b->fork, b->stream);
    for (size_t i = 0; i < b->models.size(); ++i) {
      rmhmc_model* m = b->models[i];
      cudaStreamWaitEvent(m->stream, b->fork, 0);
      leapfrog_step(m, integ->eps, integ->n_fp);
      cudaEventRecord(b->joins[i], m->stream);
      cudaStreamWaitEvent(b->stream, b->joins[i], 0);
    }
    cudaGraph_t g = nullptr;
    if (cudaStreamEndCapture(b->stream, &g) != cudaSuccess || !g) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return RMHMC_ECUDA;
    }
    const cudaError_t e = cudaGraphInstantiate(&b->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      b->exec = nullptr;
      cudaGetLastError();
      return RMHMC_ECUDA;
    }
    b->eps = integ->eps;
    b->n_fp = integ->n_fp;
  }
  // the replay waits for work already queued on every model's stream, and later calls on a
  // model's own stream wait for the replay
  for (size_t i = 0; i < b->models.size(); ++i) {
    cudaEventRecord(b->pre[i], b->models[i]->stream);
    cudaStreamWaitEvent(b->stream, b->pre[i], 0);
  }
  for (int i = 0; i < n_steps; ++i)
    if (cudaGraphLaunch(b->exec, b->stream) != cudaSuccess) return RMHMC_ECUDA;
  cudaEventRecord(b->post, b->stream);
  for (rmhmc_model* m : b->models) cudaStreamWaitEvent(m->stream, b->post, 0);
  return check_launch();
}

rmhmc_status rmhmc_autotune(rmhmc_model* m, const rmhmc_integrator* integ, int* cluster_out,
                            int* sched_out, int* tile_out, int* prerot_out) {
  if (!m || !m->has_state || m->prof) return RMHMC_EINVAL;
  rmhmc_status st = check_integ(m, integ, false);
  if (st != RMHMC_OK) return st;
  cudaStream_t s = m->stream;
  const int C = m->C, dp = m->dp;
  const long long DD = (long long)dp * dp, nv = (long long)C * dp;
  // the state to come back to: q, p and Psi^T on the device (scratch that only rmhmc_sample
  // uses), the per-chain counters and status on the host
  std::vector<int> h_eig(C), h_status(C), h_sw_last(C), h_sw_acc(C), h_sw_total(C);
  int* const ivec[5] = {m->eig_count, m->status, m->sweeps_last, m->sweeps_acc, m->sweeps_total};
  std::vector<int>* const hvec[5] = {&h_eig, &h_status, &h_sw_last, &h_sw_acc, &h_sw_total};
  if (cudaStreamSynchronize(s) != cudaSuccess) return RMHMC_ECUDA;
  for (int i = 0; i < 5; ++i) cudaMemcpy(hvec[i]->data(), ivec[i], C * sizeof(int), cudaMemcpyDeviceToHost);
  cudaMemcpyAsync(m->q_save, m->q, nv * sizeof(double), cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(m->z, m->p, nv * sizeof(double), cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(m->PsiT_save, m->PsiT, C * DD * sizeof(double), cudaMemcpyDeviceToDevice, s);
  auto counters_back = [&]() {
    for (int i = 0; i < 5; ++i)
      cudaMemcpyAsync(ivec[i], hvec[i]->data(), C * sizeof(int), cudaMemcpyHostToDevice, s);
  };
  // back to the saved point, its geometry re-evaluated there (from the saved basis, which is
  // already converged at q: U, dU and the Hessian are recomputed exactly, the basis is re-checked)
  auto restore = [&]() {
    cudaMemcpyAsync(m->q, m->q_save, nv * sizeof(double), cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(m->p, m->z, nv * sizeof(double), cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(m->PsiT, m->PsiT_save, C * DD * sizeof(double), cudaMemcpyDeviceToDevice, s);
    counters_back();
    eval_geometry(m, true);
    counters_back();
    cudaStreamSynchronize(s);
  };
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return RMHMC_ECUDA;
  const int cands[4] = {1, 2, 4, 8};
  const int scheds[2] = {RMHMC_JACOBI_CYCLIC, RMHMC_JACOBI_DYNAMIC};
  const int tiles[2] = {64, 32};
  double best = 1e300;
  int best_c = m->cluster, best_s = m->jacobi_sched, best_t = m->tc_nt;
  // a candidate's time: from the restored state, one untimed leapfrog (the eigen-updates settle
  // into the candidate's steady state), then two timed ones
  auto trial = [&](float* ms) -> bool {
    restore();
    leapfrog_step(m, integ->eps, integ->n_fp);
    cudaEventRecord(e0, s);
    leapfrog_step(m, integ->eps, integ->n_fp);
    leapfrog_step(m, integ->eps, integ->n_fp);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) return false;
    cudaEventElapsedTime(ms, e0, e1);
    return true;
  };
  int sms = 148;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device) != cudaSuccess || sms < 1) sms = 148;
  // one untimed trial first (first-launch costs); then one generalized leapfrog per (cluster size,
  // rotation order) at the current tile width, then the other tile width with the best of those
  // (a tile width only matters where the mixed form's products run on the tensor cores)
  float ms = 0.f;
  if (!trial(&ms)) return RMHMC_ECUDA;
  for (int t = 0; t < 8; ++t) {
    // cluster sizes whose CTAs (two per SM) would not all be resident at once run in waves
    if (cands[t % 4] > 1 && (long long)C * cands[t % 4] > 2LL * sms) continue;
    m->jacobi_sched = scheds[t / 4];
    m->cluster = cands[t % 4];
    if (!trial(&ms)) return RMHMC_ECUDA;
    if (ms < best) {
      best = ms;
      best_c = m->cluster;
      best_s = m->jacobi_sched;
    }
  }
  m->cluster = best_c;
  m->jacobi_sched = best_s;
  int best_p = m->prerot;
  if (m->precision == RMHMC_MIXED) {
    for (int t : tiles) {
      if (t == best_t) continue;
      m->tc_nt = t;
      if (!trial(&ms)) return RMHMC_ECUDA;
      if (ms < best) {
        best = ms;
        best_t = t;
      }
    }
    m->tc_nt = best_t;
    // and the first-order pre-rotation of warm eigen-updates, on or off
    m->prerot = 1 - best_p;
    if (!trial(&ms)) return RMHMC_ECUDA;
    if (ms < best) {
      best = ms;
      best_p = m->prerot;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  m->tc_nt = best_t;
  m->prerot = best_p;
  restore();
  if (cluster_out) *cluster_out = best_c;
  if (sched_out) *sched_out = best_s;
  if (tile_out) *tile_out = best_t;
  if (prerot_out) *prerot_out = best_p;
  return check_launch();
}

rmhmc_status rmhmc_stream_create(void** stream_out) {
  if (!stream_out) return RMHMC_EINVAL;
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return RMHMC_ECUDA;
  }
  *stream_out = s;
  return RMHMC_OK;
}

rmhmc_status rmhmc_stream_destroy(void* stream) {
  if (!stream) return RMHMC_EINVAL;
  return cudaStreamDestroy((cudaStream_t)stream) == cudaSuccess ? RMHMC_OK : RMHMC_ECUDA;
}

rmhmc_status rmhmc_set_gemm_tile(rmhmc_model* m, int nt) {
  if (!m || (nt != 64 && nt != 32)) return RMHMC_EINVAL;
  m->tc_nt = nt;
  return RMHMC_OK;
}

rmhmc_status rmhmc_set_prerotation(rmhmc_model* m, int enable) {
  if (!m || (enable != 0 && enable != 1)) return RMHMC_EINVAL;
  m->prerot = enable;
  return RMHMC_OK;
}

rmhmc_status rmhmc_set_jacobi(rmhmc_model* m, int cluster, int sched) {
  if (!m) return RMHMC_EINVAL;
  if (cluster != 0 && cluster != 1 && cluster != 2 && cluster != 4 && cluster != 8) return RMHMC_EINVAL;
  if (sched != RMHMC_JACOBI_CYCLIC && sched != RMHMC_JACOBI_DYNAMIC) return RMHMC_EINVAL;
  m->cluster = cluster == 0 ? jacobi_cluster_size(m->C) : cluster;
  m->jacobi_sched = sched;
  return RMHMC_OK;
}


const char* rmhmc_status_string(rmhmc_status s) {
  switch (s) {
    case RMHMC_OK: return "ok";
    case RMHMC_EINVAL: return "invalid argument";
    case RMHMC_ENOMEM: return "device allocation failed";
    case RMHMC_ECUDA: return "CUDA runtime error";
    case RMHMC_ENOTCONV: return "Jacobi did not converge";
    case RMHMC_ENONFINITE: return "non-finite value";
    case RMHMC_ETIMEOUT: return "bounded device wait gave up";
    case RMHMC_ENOTIMPL: return "not implemented in this build";
    case RMHMC_ENOTPD: return "kernel matrix not positive definite";
    case RMHMC_ESCRATCH: return "batch exceeds the fixed workspace of rmhmc_eigh_noalloc";
  }
  return "unknown status";
}

const char* rmhmc_version(void) { return "rmhmc sm_103a fp64 + f32x2 + tcgen05 bf16 slices"; }


rmhmc_status rmhmc_fp64_peak(void* cuda_stream, int ms_target, double* tflops_host) {
  return fma_peak<double>(cuda_stream, ms_target, tflops_host);
}

rmhmc_status rmhmc_fp32_peak(void* cuda_stream, int ms_target, double* tflops_host) {
  return fma_peak<float>(cuda_stream, ms_target, tflops_host);
}

rmhmc_status rmhmc_df_peak(void* cuda_stream, int ms_target, double* tflops_host) {
  return df_peak(cuda_stream, ms_target, tflops_host);
}

const char* rmhmc_profile_category(int i) {
  return (i >= 0 && i < RMHMC_PROF_NCAT) ? kCatNames[i] : "";
}

rmhmc_status rmhmc_profile(rmhmc_model* m, int enable) {
  if (!m) return RMHMC_EINVAL;
  if (enable) {
    if (m->ev.empty()) {
      m->ev.resize(1 << 15);
      for (auto& e : m->ev)
        if (cudaEventCreate(&e) != cudaSuccess) return RMHMC_ECUDA;
    }
    m->ev_next = 0;
    m->recs.clear();
    for (int i = 0; i < RMHMC_PROF_NCAT; ++i) {
      m->prof_flops[i] = 0.0;
      m->prof_launch[i] = 0;
    }
    cudaMemsetAsync(m->sweeps_total, 0, m->C * sizeof(int), m->stream);
    cudaMemsetAsync(m->jw.tiles, 0, (size_t)kJacStats * m->C * sizeof(unsigned long long), m->stream);
  }
  m->prof = enable != 0;
  return RMHMC_OK;
}

rmhmc_status rmhmc_jacobi_counters(rmhmc_model* m, long long* counters_host) {
  if (!m || !counters_host) return RMHMC_EINVAL;
  if (cudaStreamSynchronize(m->stream) != cudaSuccess) return RMHMC_ECUDA;
  std::vector<unsigned long long> tl((size_t)kJacStats * m->C);
  if (cudaMemcpy(tl.data(), m->jw.tiles, tl.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost) !=
      cudaSuccess)
    return RMHMC_ECUDA;
  for (int k = 0; k < 8; ++k) {
    long long v = 0;
    for (int c = 0; c < m->C; ++c) v += (long long)tl[(size_t)kJacStats * c + k];
    counters_host[k] = v;
  }
  return RMHMC_OK;
}

rmhmc_status rmhmc_profile_read(rmhmc_model* m, double* ms_host, double* flops_host,
                                long long* launches_host) {
  if (!m) return RMHMC_EINVAL;
  if (cudaStreamSynchronize(m->stream) != cudaSuccess) return RMHMC_ECUDA;
  double ms[RMHMC_PROF_NCAT] = {};
  for (const auto& r : m->recs) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, m->ev[r.a], m->ev[r.b]) == cudaSuccess) ms[r.cat] += t;
  }
  // Jacobi work = the 16 x 16 x 16 rotation tile products of phase 2 (2 * 16^3 flops each; tiles
  // skipped because both rotations were the identity are not counted) + the rotation rounds of
  // phase 1 (8 rotations applied to a 16 x 16 block by 2 x 2 blocks, 28 off-diagonal and 8
  // diagonal, and to its accumulated rotation: 976 FP64 multiply / FMA instructions, counted as
  // 2 flops each like the DFMA peak)
  std::vector<unsigned long long> tl((size_t)kJacStats * m->C);
  cudaMemcpy(tl.data(), m->jw.tiles, tl.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
  double tiles = 0.0, rounds = 0.0, prerot_pairs = 0.0;
  for (int c = 0; c < m->C; ++c) {
    tiles += (double)tl[(size_t)kJacStats * c];
    rounds += (double)tl[(size_t)kJacStats * c + 1];
    prerot_pairs += (double)tl[(size_t)kJacStats * c + 7];
  }
  // pre-rotation work = the double-float multiply-adds of its first- and second-order products:
  // per pre-rotated chain, 2 entries of A per pair x dp lines x 2 products x 3 applications, 2 flops
  // each (the FP32 third- and fourth-order products and the element-wise passes are not counted)
  const double prerot_flops = prerot_pairs * 2.0 * m->dp * 2.0 * 3.0 * 2.0;
  for (int i = 0; i < RMHMC_PROF_NCAT; ++i) {
    if (ms_host) ms_host[i] = ms[i];
    if (flops_host)
      flops_host[i] = (i == CAT_JACOBI || i == CAT_JACOBI_DF)
                          ? (m->prof_launch[i] ? tiles * 8192.0 + rounds * 1952.0 : 0.0)
                      : i == CAT_PREROT ? (m->prof_launch[i] ? prerot_flops : 0.0)
                                        : m->prof_flops[i];
    if (launches_host) launches_host[i] = m->prof_launch[i];
  }
  return RMHMC_OK;
}

int rmhmc_dim(const rmhmc_model* m) { return m ? m->d : -1; }
int rmhmc_n_chains(const rmhmc_model* m) { return m ? m->C : -1; }

void rmhmc_free_model(rmhmc_model* m) {
  if (!m) return;
  cudaStreamSynchronize(m->stream);
  for (void* p : m->allocs) cudaFree(p);
  for (cudaEvent_t e : m->ev) cudaEventDestroy(e);
  delete m;
}

namespace {

rmhmc_status validate_desc(const rmhmc_model_desc* desc, int n_chains, const double* tau_host) {
  if (!desc || n_chains < 1 || n_chains > 65535) return RMHMC_EINVAL;

  if (desc->N < 1 || desc->N > kMaxN || desc->n_cov < 1 || !desc->X || !desc->y) return RMHMC_EINVAL;
  if (desc->n_kernels < 1 || desc->n_kernels > RMHMC_MAX_KERNELS || !desc->kernels) return RMHMC_EINVAL;
  if (desc->lik != RMHMC_LIK_BERNOULLI_LOGIT && desc->lik != RMHMC_LIK_GAUSSIAN) return RMHMC_EINVAL;
  if (desc->lik == RMHMC_LIK_GAUSSIAN && !(desc->noise_var > 0.0)) return RMHMC_EINVAL;
  if (!desc->sample_hypers && !desc->u_fixed) return RMHMC_EINVAL;
  for (int k = 0; k < desc->n_kernels; ++k) {
    const rmhmc_kernel_desc& kd = desc->kernels[k];
    if (kd.kind < 0 || kd.kind > 2 || kd.n_cols < 1 || kd.n_cols > RMHMC_MAX_COLS) return RMHMC_EINVAL;
    if (!(kd.jitter > 0.0)) return RMHMC_EINVAL;
    for (int t = 0; t < kd.n_cols; ++t)
      if (kd.cols[t] < 0 || kd.cols[t] >= desc->n_cov) return RMHMC_EINVAL;
    for (int h = 0; h < 2; ++h)
      if (!(kd.prior_a[h] > 0.0) || !(kd.prior_b[h] > 0.0)) return RMHMC_EINVAL;
  }
  if (tau_host)
    for (int c = 0; c < n_chains; ++c)
      if (!(tau_host[c] >= 0.0) || tau_host[c] > 1.0) return RMHMC_EINVAL;

  return RMHMC_OK;
}

// Sizes and the device-side description (without device pointers) of a model for desc.
void setup_fields(rmhmc_model* m, const rmhmc_model_desc* desc, int n_chains, void* cuda_stream) {
  cudaGetDevice(&m->device);
  m->stream = (cudaStream_t)cuda_stream;
  m->N = desc->N;
  m->n = desc->n_kernels;
  m->P = desc->sample_hypers ? 2 * m->n : 0;
  m->d = m->n * m->N + m->P;
  m->dp = ((m->d + kJacSB - 1) / kJacSB) * kJacSB;
  m->C = n_chains;
  m->cluster = jacobi_cluster_size(n_chains);
  ModelDev& md = m->md;
  md.N = m->N;
  md.n = m->n;
  md.P = m->P;
  md.d = m->d;
  md.dp = m->dp;
  md.ncov = desc->n_cov;
  md.lik = desc->lik;
  md.sample_hypers = desc->sample_hypers ? 1 : 0;
  md.n_chains = n_chains;
  md.noise_var = desc->noise_var;
  for (int k = 0; k < m->n; ++k) {
    const rmhmc_kernel_desc& kd = desc->kernels[k];
    md.k[k].kind = kd.kind;
    md.k[k].n_cols = kd.n_cols;
    for (int t = 0; t < RMHMC_MAX_COLS; ++t) md.k[k].cols[t] = t < kd.n_cols ? kd.cols[t] : 0;
    md.k[k].jitter = kd.jitter;
    for (int h = 0; h < 2; ++h) {
      md.k[k].a[h] = kd.prior_a[h];
      md.k[k].b[h] = kd.prior_b[h];
    }
  }
}

}  // namespace

rmhmc_status rmhmc_plan_bytes(const rmhmc_model_desc* desc, int n_chains, size_t* bytes) {
  if (!bytes) return RMHMC_EINVAL;
  *bytes = 0;
  rmhmc_status st = validate_desc(desc, n_chains, nullptr);
  if (st != RMHMC_OK) return st;
  rmhmc_model m;
  setup_fields(&m, desc, n_chains, nullptr);
  size_t total = 0;
  m.plan_bytes = &total;
  st = allocate_model(&m, desc->n_cov);
  *bytes = total;
  return st;
}

rmhmc_status rmhmc_init_model(const rmhmc_model_desc* desc, int n_chains, const double* tau_host,
                              void* cuda_stream, rmhmc_model** out) {
  if (!out) return RMHMC_EINVAL;
  *out = nullptr;
  rmhmc_status vst = validate_desc(desc, n_chains, tau_host);
  if (vst != RMHMC_OK) return vst;
  rmhmc_model* m = new rmhmc_model();
  setup_fields(m, desc, n_chains, cuda_stream);
  ModelDev& md = m->md;
  const int N = m->N, n = m->n, C = m->C;
  rmhmc_status st = allocate_model(m, desc->n_cov);
  if (st != RMHMC_OK) {
    rmhmc_free_model(m);
    return st;
  }
  std::vector<double> tauv(C, 1.0);
  if (tau_host) memcpy(tauv.data(), tau_host, C * sizeof(double));
  std::vector<double> ufv(2 * n, 0.0);
  if (!desc->sample_hypers) memcpy(ufv.data(), desc->u_fixed, 2 * n * sizeof(double));
  double *X = m->X_dev, *y = m->y_dev, *uf = m->uf_dev, *tau = m->tau_dev;
  cudaError_t e = cudaMemcpyAsync(X, desc->X, (size_t)N * desc->n_cov * sizeof(double),
                                  cudaMemcpyHostToDevice, m->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(y, desc->y, N * sizeof(double), cudaMemcpyHostToDevice, m->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(uf, ufv.data(), 2 * n * sizeof(double), cudaMemcpyHostToDevice, m->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(tau, tauv.data(), C * sizeof(double), cudaMemcpyHostToDevice, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) {
    rmhmc_free_model(m);
    return RMHMC_ECUDA;
  }
  md.X = X;
  md.y = y;
  md.u_fixed = uf;
  md.tau = tau;
  *out = m;
  return RMHMC_OK;
}

namespace {

rmhmc_status validate_primal(const rmhmc_primal_desc* desc, int n_chains, const double* tau_host) {
  if (!desc || n_chains < 1 || n_chains > 65535) return RMHMC_EINVAL;
  if (desc->N < 1 || desc->N > (1 << 20) || !desc->y) return RMHMC_EINVAL;
  if (desc->n_gauss < 0 || desc->n_linear < 0 || desc->n_gauss + desc->n_linear < 1) return RMHMC_EINVAL;
  if ((desc->n_gauss > 0 && !desc->Xg) || (desc->n_linear > 0 && !desc->Xl)) return RMHMC_EINVAL;
  if (desc->n_gauss > 0 && (desc->M < 1 || !(desc->L > 0.0))) return RMHMC_EINVAL;
  if (desc->J != 1 && desc->J != 2) return RMHMC_EINVAL;
  const long long d =
      desc->J * ((long long)(desc->n_gauss > 0 ? desc->M : 0) * desc->n_gauss + desc->n_linear + 1) + 3;
  if (d > 4096) return RMHMC_EINVAL;
  if (desc->J == 1 && desc->lik != RMHMC_LIK_BERNOULLI_LOGIT && desc->lik != RMHMC_LIK_GAUSSIAN)
    return RMHMC_EINVAL;
  if (desc->J == 2 && (desc->lik != RMHMC_LIK_MEANVAR || !(desc->delta >= 0.0))) return RMHMC_EINVAL;
  if (desc->lik == RMHMC_LIK_GAUSSIAN && !(desc->noise_var > 0.0)) return RMHMC_EINVAL;
  if (!(desc->bias_var > 0.0)) return RMHMC_EINVAL;
  for (int j = 0; j < 3; ++j)
    if (!(desc->prior_a[j] > 0.0) || !(desc->prior_b[j] > 0.0)) return RMHMC_EINVAL;
  if (tau_host)
    for (int c = 0; c < n_chains; ++c)
      if (!(tau_host[c] >= 0.0) || tau_host[c] > 1.0) return RMHMC_EINVAL;
  return RMHMC_OK;
}

void setup_primal(rmhmc_model* m, const rmhmc_primal_desc* desc, int n_chains, void* cuda_stream) {
  cudaGetDevice(&m->device);
  m->stream = (cudaStream_t)cuda_stream;
  m->kind = 1;
  PrimalDev& pd = m->pd;
  pd.N = desc->N;
  pd.Dg = desc->n_gauss;
  pd.Dl = desc->n_linear;
  pd.M = desc->n_gauss > 0 ? desc->M : 0;
  pd.P = pd.M * pd.Dg + pd.Dl + 1;
  pd.J = desc->J;
  pd.JP = pd.J * pd.P;
  pd.d = pd.JP + 3;
  pd.delta = desc->delta;
  pd.dp = ((pd.d + kJacSB - 1) / kJacSB) * kJacSB;
  pd.lik = desc->lik;
  pd.n_chains = n_chains;
  pd.noise_var = desc->noise_var;
  pd.L = desc->L;
  pd.bias_var = desc->bias_var;
  for (int j = 0; j < 3; ++j) {
    pd.a[j] = desc->prior_a[j];
    pd.b[j] = desc->prior_b[j];
  }
  m->N = pd.N;
  m->n = 1;
  m->P = 3;
  m->d = pd.d;
  m->dp = pd.dp;
  m->C = n_chains;
  m->cluster = jacobi_cluster_size(n_chains);
}

}  // namespace

rmhmc_status rmhmc_plan_bytes_primal(const rmhmc_primal_desc* desc, int n_chains, size_t* bytes) {
  if (!bytes) return RMHMC_EINVAL;
  *bytes = 0;
  rmhmc_status st = validate_primal(desc, n_chains, nullptr);
  if (st != RMHMC_OK) return st;
  rmhmc_model m;
  setup_primal(&m, desc, n_chains, nullptr);
  size_t total = 0;
  m.plan_bytes = &total;
  st = allocate_model(&m, 0);
  *bytes = total;
  return st;
}

rmhmc_status rmhmc_init_primal(const rmhmc_primal_desc* desc, int n_chains, const double* tau_host,
                               void* cuda_stream, rmhmc_model** out) {
  if (!out) return RMHMC_EINVAL;
  *out = nullptr;
  rmhmc_status vst = validate_primal(desc, n_chains, tau_host);
  if (vst != RMHMC_OK) return vst;
  rmhmc_model* m = new rmhmc_model();
  setup_primal(m, desc, n_chains, cuda_stream);
  rmhmc_status st = allocate_model(m, 0);
  if (st != RMHMC_OK) {
    rmhmc_free_model(m);
    return st;
  }
  PrimalDev& pd = m->pd;
  const int N = pd.N, C = m->C;
  std::vector<double> tauv(C, 1.0);
  if (tau_host) memcpy(tauv.data(), tau_host, C * sizeof(double));
  cudaError_t e = cudaMemcpyAsync(m->y_dev, desc->y, N * sizeof(double), cudaMemcpyHostToDevice, m->stream);
  if (e == cudaSuccess && pd.Dg)
    e = cudaMemcpyAsync(m->Xg_dev, desc->Xg, (size_t)N * pd.Dg * sizeof(double), cudaMemcpyHostToDevice,
                        m->stream);
  if (e == cudaSuccess && pd.Dl)
    e = cudaMemcpyAsync(m->Xl_dev, desc->Xl, (size_t)N * pd.Dl * sizeof(double), cudaMemcpyHostToDevice,
                        m->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(m->tau_dev, tauv.data(), C * sizeof(double), cudaMemcpyHostToDevice, m->stream);
  pd.Xg = m->Xg_dev;
  pd.Xl = m->Xl_dev;
  pd.y = m->y_dev;
  pd.tau = m->tau_dev;
  if (e == cudaSuccess) {
    const long long NP = (long long)N * pd.P;
    dev::k_phi<<<nblk(NP), 256, 0, m->stream>>>(pd, m->Phi);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) {
    rmhmc_free_model(m);
    return RMHMC_ECUDA;
  }
  *out = m;
  return RMHMC_OK;
}

rmhmc_status rmhmc_set_state(rmhmc_model* m, const rmhmc_integrator* integ, const double* q_dev,
                             const double* p_dev) {
  if (!m || !q_dev) return RMHMC_EINVAL;
  rmhmc_status st = check_integ(m, integ, true);
  if (st != RMHMC_OK) return st;
  m->g_kind = integ->g_kind;
  m->alpha = integ->alpha;
  m->tol = integ->jacobi_tol;
  m->max_sweeps = integ->max_sweeps;
  m->reorth_every = integ->reorth_every;
  m->precision = integ->precision;
  m->jacobi_rule = integ->jacobi_rule;
  m->eigen_start = integ->eigen_start;
  cudaStream_t s = m->stream;
  const int C = m->C, dp = m->dp, d = m->d;
  k_restride<<<nblk((long long)C * dp), 256, 0, s>>>(m->q, dp, q_dev, d, d, C);
  k_restride<<<nblk((long long)C * dp), 256, 0, s>>>(m->p, dp, p_dev, d, d, C);
  cudaMemsetAsync(m->status, 0, C * sizeof(int), s);
  cudaMemsetAsync(m->eig_count, 0, C * sizeof(int), s);
  cudaMemsetAsync(m->sweeps_acc, 0, C * sizeof(int), s);
  k_set_identity<<<nblk((long long)C * dp * dp), 256, 0, s>>>(m->PsiT, dp, C);
  m->cold = true;
  eval_geometry(m, true);
  m->cold = false;
  m->has_state = true;
  return check_launch();
}

rmhmc_status rmhmc_leapfrog(rmhmc_model* m, const rmhmc_integrator* integ, int n_steps,
                            const double* p_in_dev, double* q_dev, double* p_dev, double* H_dev,
                            int* status_dev) {
  if (!m || n_steps < 0) return RMHMC_EINVAL;
  rmhmc_status st = check_integ(m, integ, false);
  if (st != RMHMC_OK) return st;
  cudaStream_t s = m->stream;
  const int C = m->C, dp = m->dp, d = m->d;
  if (p_in_dev) {
    PROF(m, CAT_VECTOR, 0)
    k_restride<<<nblk((long long)C * dp), 256, 0, s>>>(m->p, dp, p_in_dev, d, d, C);
  }
  for (int i = 0; i < n_steps; ++i) leapfrog_step(m, integ->eps, integ->n_fp);
  if (q_dev) {
    PROF(m, CAT_VECTOR, 0)
    k_restride<<<nblk((long long)C * d), 256, 0, s>>>(q_dev, d, m->q, dp, d, C);
  }
  if (p_dev) {
    PROF(m, CAT_VECTOR, 0)
    k_restride<<<nblk((long long)C * d), 256, 0, s>>>(p_dev, d, m->p, dp, d, C);
  }
  if (H_dev) hamiltonian(m, m->p, H_dev);
  PROF(m, CAT_VECTOR, 0)
  k_flag_nonfinite<<<C, 128, 0, s>>>(m->status, status_dev, m->q, m->p, m->U, H_dev, dp, d);
  return check_launch();
}

rmhmc_status rmhmc_sample(rmhmc_model* m, const rmhmc_integrator* integ, int n_iter, int n_burn,
                          uint64_t seed, double* q_samples_dev, double* logp_dev,
                          double* loglik_dev, int* accept_dev, int* sweeps_dev,
                          int* chain_status_dev) {
  if (!m || n_iter < 0 || n_burn < 0) return RMHMC_EINVAL;
  rmhmc_status st = check_integ(m, integ, false);
  if (st != RMHMC_OK) return st;
  if (integ->n_leapfrog < 1) return RMHMC_EINVAL;
  cudaStream_t s = m->stream;
  const int C = m->C, dp = m->dp, d = m->d;
  const long long nv = (long long)C * dp, DD = (long long)dp * dp;
  if (chain_status_dev) cudaMemsetAsync(chain_status_dev, 0, C * sizeof(int), s);
  for (int it = 0; it < n_burn + n_iter; ++it) {
    const uint64_t l = m->iter++;
    const bool rec = it >= n_burn;
    const long long ro = rec ? (long long)(it - n_burn) : 0;
    // p = G^{1/2} z (symmetric root)
    PROF(m, CAT_VECTOR, 0)
    k_normals<<<dim3(nblk((dp + 3) / 4, 128), C), 128, 0, s>>>(m->z, dp, d, C, seed, l);
    PROF(m, CAT_VECTOR, 2.0 * C * (double)d * d)
    gemv_f64(s, false, dp, dp, m->PsiT, dp, DD, m->z, dp, m->t1, dp, C, 1.0, 0.0);
    PROF(m, CAT_VECTOR, 0)
    k_scale_g<<<nblk(nv), 256, 0, s>>>(m->t1, m->g, dp, d, C, 1);
    PROF(m, CAT_VECTOR, 2.0 * C * (double)d * d)
    gemv_f64(s, true, dp, dp, m->PsiT, dp, DD, m->t1, dp, m->p, dp, C, 1.0, 0.0);
    hamiltonian(m, m->p, m->Ham0);
    cudaMemcpyAsync(m->q_save, m->q, nv * sizeof(double), cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(m->PsiT_save, m->PsiT, C * DD * sizeof(double), cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(m->eig_save, m->eig_count, C * sizeof(int), cudaMemcpyDeviceToDevice, s);
    cudaMemsetAsync(m->sweeps_acc, 0, C * sizeof(int), s);
    for (int L = 0; L < integ->n_leapfrog; ++L) leapfrog_step(m, integ->eps, integ->n_fp);
    hamiltonian(m, m->p, m->Ham1);
    PROF(m, CAT_VECTOR, 0)
    k_accept<<<nblk(C), 256, 0, s>>>(m->Ham0, m->Ham1, m->status, m->acc, C, seed, l,
                                     (rec && accept_dev) ? accept_dev + ro * C : nullptr,
                                     (rec && sweeps_dev) ? sweeps_dev + ro * C : nullptr,
                                     m->sweeps_acc, chain_status_dev);
    PROF(m, CAT_VECTOR, 0)
    k_restore<<<dim3(nblk(DD), C), 256, 0, s>>>(m->acc, m->q, m->q_save, m->PsiT, m->PsiT_save,
                                                m->eig_count, m->eig_save, dp);
    eval_geometry(m, true);
    if (rec && (q_samples_dev || logp_dev || loglik_dev))
      PROF(m, CAT_VECTOR, 0)
      k_record<<<nblk((long long)C * d), 256, 0, s>>>(m->q, m->U, m->LL, dp, d, C,
                                                       q_samples_dev ? q_samples_dev + ro * C * d : nullptr,
                                                       logp_dev ? logp_dev + ro * C : nullptr,
                                                       loglik_dev ? loglik_dev + ro * C : nullptr);
  }
  return check_launch();
}

rmhmc_status rmhmc_geometry(rmhmc_model* m, double* U_dev, double* dU_dev, double* hess_dev,
                            double* lam_dev, double* G_dev, int* sweeps_dev) {
  if (!m || !m->has_state) return RMHMC_EINVAL;
  cudaStream_t s = m->stream;
  const int C = m->C, dp = m->dp, d = m->d;
  const long long DD = (long long)dp * dp;
  if (U_dev) cudaMemcpyAsync(U_dev, m->U, C * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (dU_dev) k_restride<<<nblk((long long)C * d), 256, 0, s>>>(dU_dev, d, m->dU, dp, d, C);
  if (lam_dev) k_restride<<<nblk((long long)C * d), 256, 0, s>>>(lam_dev, d, m->lam, dp, d, C);
  if (sweeps_dev) cudaMemcpyAsync(sweeps_dev, m->sweeps_last, C * sizeof(int), cudaMemcpyDeviceToDevice, s);
  if (hess_dev) k_compact<<<nblk((long long)C * d * d), 256, 0, s>>>(hess_dev, m->H, dp, d, C);
  if (G_dev) {
    // G = Psi diag(g) Psi^T = PsiT^T (diag(g) PsiT), built in scratch and compacted
    k_scale_rows<<<dim3(nblk(DD), C), 256, 0, s>>>(m->Y, m->PsiT, m->g, dp, d);
    gemm_f64(s, true, false, dp, dp, dp, 1.0, m->PsiT, dp, DD, m->Y, dp, DD, 0.0, m->W, dp, DD, C, true, false);
    k_compact<<<nblk((long long)C * d * d), 256, 0, s>>>(G_dev, m->W, dp, d, C);
  }
  return check_launch();
}

rmhmc_status rmhmc_hamiltonian_grad(rmhmc_model* m, const double* p_dev, double* dHdq_dev,
                                    double* Ginv_p_dev, double* H_dev) {
  if (!m || !m->has_state || !p_dev) return RMHMC_EINVAL;
  cudaStream_t s = m->stream;
  const int C = m->C, dp = m->dp, d = m->d;
  k_restride<<<nblk((long long)C * dp), 256, 0, s>>>(m->xin, dp, p_dev, d, d, C);
  if (dHdq_dev) {
    grad_h(m, m->xin, m->dHdq);
    k_restride<<<nblk((long long)C * d), 256, 0, s>>>(dHdq_dev, d, m->dHdq, dp, d, C);
  }
  if (Ginv_p_dev) {
    ginv(m, m->xin, m->v0);
    k_restride<<<nblk((long long)C * d), 256, 0, s>>>(Ginv_p_dev, d, m->v0, dp, d, C);
  }
  if (H_dev) hamiltonian(m, m->xin, H_dev);
  return check_launch();
}

}  // extern "C"
