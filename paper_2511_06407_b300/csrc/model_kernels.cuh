// Device kernels of the model layer: kernel matrices, likelihood maps, hyperparameter statistics,
// Hessian assembly, the third-derivative contraction and the soft-abs map. Included once, by
// rmhmc.cu.
#pragma once
#include <math.h>

#include "internal.cuh"

namespace rmhmc {
namespace dev {

constexpr double LOG2PI = 1.8378770664093454835606594728112;

__device__ __forceinline__ double hyper_u(const ModelDev& md, const double* q, int dp, int c, int k,
                                          int h) {
  return md.sample_hypers ? q[(long long)c * dp + md.n * md.N + 2 * k + h] : md.u_fixed[2 * k + h];
}

// K(x_i, x_j) and its first three derivatives in u_1 = log theta (Eq. BMKL kernels, log-parametrised).
// Every derivative in u_0 = log c returns the same value, so these four cover all mixed derivatives.
__device__ __forceinline__ void kern_derivs(const KernelDev& kd, const double* __restrict__ X, int ncov,
                                            int i, int j, double c, double th, double D[4]) {
  const double* xi = X + (long long)i * ncov;
  const double* xj = X + (long long)j * ncov;
  const double diag = (i == j) ? c * kd.jitter : 0.0;
  if (kd.kind == RMHMC_K_SE) {
    double sq = 0.0;
    for (int t = 0; t < kd.n_cols; ++t) {
      const double dd = xi[kd.cols[t]] - xj[kd.cols[t]];
      sq = fma(dd, dd, sq);
    }
    const double r = sq / (th * th);
    const double E = c * exp(-0.5 * r);
    D[0] = E + diag;
    D[1] = E * r;
    D[2] = E * (r * r - 2.0 * r);
    D[3] = E * (r * r * r - 6.0 * r * r + 4.0 * r);
  } else if (kd.kind == RMHMC_K_LINEAR) {
    double g = 0.0;
    for (int t = 0; t < kd.n_cols; ++t) g = fma(xi[kd.cols[t]], xj[kd.cols[t]], g);
    D[0] = c * (g + th) + diag;
    D[1] = c * th;
    D[2] = D[1];
    D[3] = D[1];
  } else {
    double h = 0.0;
    for (int t = 0; t < kd.n_cols; ++t) h += (xi[kd.cols[t]] != xj[kd.cols[t]]) ? 1.0 : 0.0;
    const double s = h / th;
    const double E = c * exp(-s);
    D[0] = E + diag;
    D[1] = E * s;
    D[2] = E * (s * s - s);
    D[3] = E * (s * s * s - 3.0 * s * s + s);
  }
}

// K and D1, D2, D3 = d^r K / du_1^r for every (chain, kernel): grid (32 x 32 tiles of the lower
// triangle, n, C). kern_derivs is exactly symmetric in (i, j), so each tile below the diagonal is
// evaluated once and written twice (the mirror through a shared-memory transpose, both coalesced).
__global__ void __launch_bounds__(256) k_assemble(ModelDev md, const double* __restrict__ q, int dp,
                                                  double* __restrict__ K, double* __restrict__ D1,
                                                  double* __restrict__ D2, double* __restrict__ D3) {
  const int k = blockIdx.y, c = blockIdx.z, N = md.N;
  const int t = blockIdx.x;
  int ti = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);  // tile (ti, tj), tj <= ti, t = ti (ti + 1) / 2 + tj
  while (ti * (ti + 1) / 2 > t) --ti;
  while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
  const int tj = t - ti * (ti + 1) / 2;
  __shared__ double hyp[2];
  __shared__ double tile[4][32][33];
  if (threadIdx.x == 0) {
    hyp[0] = exp(hyper_u(md, q, dp, c, k, 0));
    hyp[1] = exp(hyper_u(md, q, dp, c, k, 1));
  }
  __syncthreads();
  const double cc = hyp[0], th = hyp[1];
  const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
  const long long base = ((long long)c * md.n + k) * N * N;
  double* out[4] = {K, D1, D2, D3};
  for (int r = wy; r < 32; r += 8) {
    const int i = ti * 32 + r, j = tj * 32 + lane;
    double D[4] = {0.0, 0.0, 0.0, 0.0};
    if (i < N && j < N && (ti != tj || j <= i)) {
      kern_derivs(md.k[k], md.X, md.ncov, i, j, cc, th, D);
      const long long o = base + (long long)i * N + j;
#pragma unroll
      for (int m = 0; m < 4; ++m) out[m][o] = D[m];
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) tile[m][r][lane] = D[m];
  }
  __syncthreads();
  for (int r = wy; r < 32; r += 8) {  // (j, i) = mirror of the tile's (i, j), strictly above the diagonal
    const int jr = tj * 32 + r, ic = ti * 32 + lane;
    if (jr < N && ic < N && ic > jr) {
      const long long o = base + (long long)jr * N + ic;
#pragma unroll
      for (int m = 0; m < 4; ++m) out[m][o] = tile[m][lane][r];
    }
  }
}

// Latent blocks f_k packed contiguously per (chain, kernel), and tau-scaled likelihood maps of
// F = sum_k f_k (Sec. 2.5 logistic / Gaussian): l, l', l'', l''' per (chain, sample).
// Negative log likelihood l of one sample and its first three derivatives in F (untempered):
// Bernoulli-logit (y in {0,1}): l = softplus(F) - y F; Gaussian: l = (y - F)^2 / (2v) + log(2 pi v)/2.
__device__ __forceinline__ void lik_point(int lik, double y, double F, double v, double& a0, double& a1,
                                          double& a2, double& a3) {
  if (lik == RMHMC_LIK_BERNOULLI_LOGIT) {
    const double s = 1.0 / (1.0 + exp(-F));
    a0 = fmax(F, 0.0) + log1p(exp(-fabs(F))) - y * F;
    a1 = s - y;
    a2 = s * (1.0 - s);
    a3 = a2 * (1.0 - 2.0 * s);
  } else {
    a0 = (y - F) * (y - F) / (2.0 * v) + 0.5 * log(2.0 * M_PI * v);
    a1 = (F - y) / v;
    a2 = 1.0 / v;
    a3 = 0.0;
  }
}

__global__ void k_lik(ModelDev md, const double* __restrict__ q, int dp, double* __restrict__ fpk,
                      double* __restrict__ l0, double* __restrict__ l1, double* __restrict__ l2,
                      double* __restrict__ l3, double* __restrict__ lraw) {
  const int c = blockIdx.y, N = md.N;
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= N) return;
  const double* qc = q + (long long)c * dp;
  double F = 0.0;
  for (int k = 0; k < md.n; ++k) {
    const double f = qc[k * N + m];
    fpk[((long long)c * md.n + k) * N + m] = f;
    F += f;
  }
  const double tau = md.tau[c];
  double a0, a1, a2, a3;
  lik_point(md.lik, md.y[m], F, md.noise_var, a0, a1, a2, a3);
  const long long o = (long long)c * N + m;
  lraw[o] = a0;
  l0[o] = tau * a0;
  l1[o] = tau * a1;
  l2[o] = tau * a2;
  l3[o] = tau * a3;
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
  return s;  // valid in thread 0
}

// Per (chain, kernel) vectors and scalars the Hessian (THIRD = false) and the third-derivative
// operator (THIRD = true) need, with S = K^-1 D1, A1 = S K^-1, S2 = S S and D1, D2, D3 from
// k_assemble. On entry `beta` holds t = L^-1 f (used for f . alpha = |t|^2) and is then overwritten:
//   beta = D1 a, eps2 = D2 a, eps3 = D3 a, gamma = K^-1 beta (= S a), delta = D1 gamma,
//   fuu11 = K^-1 (2 delta - eps2);  scalars in the Stat slots.
// Every matrix is symmetric except S and S2, so column sums read rows (coalesced). Each stage runs
// on a grid (column blocks of 32, chain x kernel): lane = column, the 8 warps split the rows, and
// the block's part of every scalar goes to part[b][block][slot]; k_stats_reduce adds the parts in a
// fixed order, so the results do not depend on scheduling.
constexpr int kStatCols = 32;
constexpr int kStatMaxBlocks = kMaxN / kStatCols;

__device__ __forceinline__ void stat_part(double v, double* red, double* part_slot) {
  // sum of v over the CTA (256 threads) into *part_slot; red: 8 doubles of shared memory
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w];
    *part_slot = s;
  }
}

// Sum over the 8 warps of a per-(warp, lane) value: the column total, valid in warp 0.
__device__ __forceinline__ double column_total(double v, double (*col)[kStatCols]) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  col[w][lane] = v;
  __syncthreads();
  double s = 0.0;
  if (w == 0)
    for (int r = 0; r < 8; ++r) s += col[r][lane];
  __syncthreads();
  return s;
}

// Stage 1: beta, eps2, eps3 and the traces <K^-1, D1>, <K^-1, D2>, <K^-1, D3>, <A1, D2>.
template <bool THIRD>
__global__ void __launch_bounds__(256) k_stats_cols(int N, const double* __restrict__ D1b,
                                                    const double* __restrict__ D2b,
                                                    const double* __restrict__ D3b,
                                                    const double* __restrict__ Kinvb,
                                                    const double* __restrict__ A1b,
                                                    const double* __restrict__ alphab,
                                                    double* __restrict__ betab, double* __restrict__ eps2b,
                                                    double* __restrict__ eps3b, double* __restrict__ part) {
  const int b = blockIdx.y, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * kStatCols + lane;
  const long long mo = (long long)b * N * N, vo = (long long)b * N;
  const double* al = alphab + vo;
  __shared__ double col[8][kStatCols];
  __shared__ double red[8];
  double bi = 0, e2 = 0, e3 = 0, trS = 0, trR2 = 0, trR3 = 0, trSR2 = 0;
  if (i < N) {
    for (int j = w; j < N; j += 8) {
      const long long o = mo + (long long)j * N + i;
      const double aj = al[j], kij = Kinvb[o], d1 = D1b[o], d2 = D2b[o];
      bi = fma(d1, aj, bi);
      e2 = fma(d2, aj, e2);
      trS = fma(kij, d1, trS);
      trR2 = fma(kij, d2, trR2);
      if (THIRD) {
        const double d3 = D3b[o];
        e3 = fma(d3, aj, e3);
        trR3 = fma(kij, d3, trR3);
        trSR2 = fma(A1b[o], d2, trSR2);
      }
    }
  }
  bi = column_total(bi, col);
  e2 = column_total(e2, col);
  if (THIRD) e3 = column_total(e3, col);
  double fa = 0, ab = 0, ae2 = 0, ae3 = 0;
  if (w == 0 && i < N) {
    const double ti = betab[vo + i];  // t = L^-1 f on entry
    fa = ti * ti;
    betab[vo + i] = bi;
    eps2b[vo + i] = e2;
    if (THIRD) eps3b[vo + i] = e3;
    ab = al[i] * bi;
    ae2 = al[i] * e2;
    ae3 = al[i] * e3;
  }
  double* pp = part + ((long long)b * kStatMaxBlocks + blockIdx.x) * ST_COUNT;
  stat_part(fa, red, pp + ST_FA);
  stat_part(ab, red, pp + ST_AB);
  stat_part(ae2, red, pp + ST_AE2);
  stat_part(trS, red, pp + ST_TRS);
  stat_part(trR2, red, pp + ST_TRR2);
  if (THIRD) {
    stat_part(ae3, red, pp + ST_AE3);
    stat_part(trR3, red, pp + ST_TRR3);
    stat_part(trSR2, red, pp + ST_TRSR2);
  }
}

// Stage 2: gamma = K^-1 beta, gamma . beta, gamma . eps2, tr(S^2) = sum S_ij S_ji and
// tr(S^3) = sum (S^2)_ij S_ji; the transposed reads go through a 32 x 33 shared tile.
template <bool THIRD>
__global__ void __launch_bounds__(256) k_stats_gamma(int N, const double* __restrict__ Kinvb,
                                                     const double* __restrict__ Sb,
                                                     const double* __restrict__ S2b,
                                                     const double* __restrict__ betab,
                                                     const double* __restrict__ eps2b,
                                                     double* __restrict__ gammab, double* __restrict__ part) {
  const int b = blockIdx.y, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i0 = blockIdx.x * kStatCols, i = i0 + lane;
  const long long mo = (long long)b * N * N, vo = (long long)b * N;
  const double* be = betab + vo;
  __shared__ double col[8][kStatCols];
  __shared__ double red[8];
  __shared__ double tS[kStatCols][kStatCols + 1], tS2[kStatCols][kStatCols + 1];
  double gi = 0, s2 = 0, s3 = 0;
  for (int j0 = 0; j0 < N; j0 += kStatCols) {
    // rows i0.. of S (and S2) at columns j0..: tS[ii][jj] = S[i0 + ii][j0 + jj]
    for (int r = w; r < kStatCols; r += 8) {
      const int ii = i0 + r, jj = j0 + lane;
      const bool in = ii < N && jj < N;
      tS[r][lane] = in ? Sb[mo + (long long)ii * N + jj] : 0.0;
      if (THIRD) tS2[r][lane] = in ? S2b[mo + (long long)ii * N + jj] : 0.0;
    }
    __syncthreads();
    for (int r = w; r < kStatCols; r += 8) {
      const int j = j0 + r;
      if (j < N && i < N) {
        const long long o = mo + (long long)j * N + i;
        gi = fma(Kinvb[o], be[j], gi);
        const double sji = Sb[o];
        s2 = fma(tS[lane][r], sji, s2);
        if (THIRD) s3 = fma(tS2[lane][r], sji, s3);
      }
    }
    __syncthreads();
  }
  gi = column_total(gi, col);
  double gb = 0, ge2 = 0;
  if (w == 0 && i < N) {
    gammab[vo + i] = gi;
    gb = gi * be[i];
    ge2 = gi * eps2b[vo + i];
  }
  double* pp = part + ((long long)b * kStatMaxBlocks + blockIdx.x) * ST_COUNT;
  stat_part(gb, red, pp + ST_GB);
  stat_part(ge2, red, pp + ST_GE2);
  stat_part(s2, red, pp + ST_TRS2);
  if (THIRD) stat_part(s3, red, pp + ST_TRS3);
}

// Stage 3 (THIRD): delta = D1 gamma, alpha . delta, gamma . delta.
__global__ void __launch_bounds__(256) k_stats_delta(int N, const double* __restrict__ D1b,
                                                     const double* __restrict__ alphab,
                                                     const double* __restrict__ gammab,
                                                     double* __restrict__ deltab, double* __restrict__ part) {
  const int b = blockIdx.y, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * kStatCols + lane;
  const long long mo = (long long)b * N * N, vo = (long long)b * N;
  __shared__ double col[8][kStatCols];
  __shared__ double red[8];
  double di = 0;
  if (i < N)
    for (int j = w; j < N; j += 8) di = fma(D1b[mo + (long long)j * N + i], gammab[vo + j], di);
  di = column_total(di, col);
  double ad = 0, gd = 0;
  if (w == 0 && i < N) {
    deltab[vo + i] = di;
    ad = alphab[vo + i] * di;
    gd = gammab[vo + i] * di;
  }
  double* pp = part + ((long long)b * kStatMaxBlocks + blockIdx.x) * ST_COUNT;
  stat_part(ad, red, pp + ST_AD);
  stat_part(gd, red, pp + ST_GD);
}

// Stage 4 (THIRD): fuu11 = K^-1 (2 delta - eps2).
__global__ void __launch_bounds__(256) k_stats_fuu(int N, const double* __restrict__ Kinvb,
                                                   const double* __restrict__ deltab,
                                                   const double* __restrict__ eps2b,
                                                   double* __restrict__ fuu11b) {
  const int b = blockIdx.y, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * kStatCols + lane;
  const long long mo = (long long)b * N * N, vo = (long long)b * N;
  __shared__ double col[8][kStatCols];
  double v = 0;
  if (i < N)
    for (int j = w; j < N; j += 8)
      v = fma(Kinvb[mo + (long long)j * N + i], 2.0 * deltab[vo + j] - eps2b[vo + j], v);
  v = column_total(v, col);
  if (w == 0 && i < N) fuu11b[vo + i] = v;
}

// stats[b][slot] = the blocks' parts of the slots the stages wrote, added in block order.
__global__ void k_stats_reduce(int nblocks, int third, const double* __restrict__ part,
                               double* __restrict__ stats) {
  const int b = blockIdx.x, slot = threadIdx.x;
  if (slot >= ST_COUNT || slot == ST_LOGDET) return;
  const bool third_slot = slot == ST_AE3 || slot == ST_AD || slot == ST_GD || slot == ST_TRS3 ||
                          slot == ST_TRR3 || slot == ST_TRSR2;
  if (third_slot && !third) return;
  double s = 0.0;
  for (int k = 0; k < nblocks; ++k) s += part[((long long)b * kStatMaxBlocks + k) * ST_COUNT + slot];
  stats[(long long)b * kStatSlots + slot] = s;
}

__device__ __forceinline__ double log_prior_u(double a, double b, double u) {
  return a * log(b) - lgamma(a) - a * u - b * exp(-u);
}

// U = -log P_tau(q), dU/dq and the untempered log-likelihood LL = ln P(y | F) per chain (one CTA
// per chain).
__global__ void __launch_bounds__(256) k_udu(ModelDev md, const double* __restrict__ q, int dp,
                                             const double* __restrict__ l0,
                                             const double* __restrict__ l1,
                                             const double* __restrict__ lraw,
                                             const double* __restrict__ alphab,
                                             const double* __restrict__ stats,
                                             double* __restrict__ U, double* __restrict__ dU,
                                             double* __restrict__ LL) {
  const int c = blockIdx.x, N = md.N, n = md.n;
  __shared__ double sh[32];
  double s = 0.0, sr = 0.0;
  for (int m = threadIdx.x; m < N; m += blockDim.x) {
    s += l0[(long long)c * N + m];
    sr += lraw[(long long)c * N + m];
  }
  for (int e = threadIdx.x; e < n * N; e += blockDim.x) {
    const int k = e / N, m = e % N;
    dU[(long long)c * dp + e] = l1[(long long)c * N + m] + alphab[((long long)c * n + k) * N + m];
  }
  for (int e = md.d + threadIdx.x; e < dp; e += blockDim.x) dU[(long long)c * dp + e] = 0.0;
  const double tot = block_sum(s, sh);
  const double totr = block_sum(sr, sh);
  if (threadIdx.x == 0) {
    LL[c] = -totr;
    double Uc = tot;
    for (int k = 0; k < n; ++k) {
      const double* st = stats + ((long long)c * n + k) * kStatSlots;
      Uc += 0.5 * st[ST_FA] + 0.5 * st[ST_LOGDET] + 0.5 * N * LOG2PI;
      if (md.sample_hypers) {
        const KernelDev& kd = md.k[k];
        const double u0 = hyper_u(md, q, dp, c, k, 0), u1 = hyper_u(md, q, dp, c, k, 1);
        Uc -= log_prior_u(kd.a[0], kd.b[0], u0) + log_prior_u(kd.a[1], kd.b[1], u1);
        const long long base = (long long)c * dp + n * N + 2 * k;
        dU[base] = -0.5 * st[ST_FA] + 0.5 * N + kd.a[0] - kd.b[0] * exp(-u0);
        dU[base + 1] = -0.5 * st[ST_AB] + 0.5 * st[ST_TRS] + kd.a[1] - kd.b[1] * exp(-u1);
      }
    }
    U[c] = Uc;
  }
}

// Hessian of U (d x d inside the dp x dp padded storage; padding is zero):
//   H[f_a, f_b] = diag(tau l'') + [a = b] K_a^-1
//   H[f_k, u_k0] = -alpha_k, H[f_k, u_k1] = -gamma_k  (= -K^-1 K_h alpha)
//   H[u_k, u_k] = [[ fa/2 + b0 e^-u0,  ab/2 ], [ ab/2,  gb - ae2/2 + trR2/2 - trS2/2 + b1 e^-u1 ]]
__global__ void k_hessian(ModelDev md, const double* __restrict__ q, int dp,
                          const double* __restrict__ Kinvb, const double* __restrict__ l2,
                          const double* __restrict__ alphab, const double* __restrict__ gammab,
                          const double* __restrict__ stats, double* __restrict__ H) {
  const int c = blockIdx.y, N = md.N, n = md.n, nN = n * N, d = md.d;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)dp * dp) return;
  const int r = (int)(e / dp), s = (int)(e % dp);
  double v = 0.0;
  if (r < d && s < d) {
    if (r < nN && s < nN) {
      const int a = r / N, i = r % N, bb = s / N, j = s % N;
      if (a == bb) v += Kinvb[(((long long)c * n + a) * N + i) * N + j];
      if (i == j) v += l2[(long long)c * N + i];
    } else if (r < nN || s < nN) {
      const int fr = r < nN ? r : s, ur = (r < nN ? s : r) - nN;
      const int a = fr / N, i = fr % N, k = ur / 2, h = ur % 2;
      if (a == k) {
        const long long vo = ((long long)c * n + k) * N + i;
        v = h == 0 ? -alphab[vo] : -gammab[vo];
      }
    } else {
      const int ur = r - nN, us = s - nN;
      const int k = ur / 2, h1 = ur % 2, k2 = us / 2, h2 = us % 2;
      if (k == k2) {
        const double* st = stats + ((long long)c * n + k) * kStatSlots;
        const KernelDev& kd = md.k[k];
        if (h1 == 0 && h2 == 0)
          v = 0.5 * st[ST_FA] + kd.b[0] * exp(-hyper_u(md, q, dp, c, k, 0));
        else if (h1 != h2)
          v = 0.5 * st[ST_AB];
        else
          v = st[ST_GB] - 0.5 * st[ST_AE2] + 0.5 * st[ST_TRR2] - 0.5 * st[ST_TRS2] +
              kd.b[1] * exp(-hyper_u(md, q, dp, c, k, 1));
      }
    }
  }
  H[(long long)c * dp * dp + e] = v;
}

// d^3 U / du_j du_k du_l for the two hyperparameters of one kernel (j, k, l in {0, 1}), from the
// scalars in the Stat slots. With gamma_0 = alpha, gamma_1 = gamma, K_0 = K, K_1 = D1,
// K_{..} = D_{number of 1 indices}, S_0 = I, S_1 = S:
//   - g_j K_k g_l - g_k K_j g_l - g_k K_l g_j + (K_jk a) g_l + g_k (K_jl a) + (K_kl a) g_j
//   - a K_jkl a / 2 - tr(S_j K^-1 K_kl) / 2 + tr(K^-1 K_jkl) / 2 + tr(S_j S_k S_l) / 2
//   + tr(S_k S_j S_l) / 2 - tr(K^-1 K_jk S_l) / 2 - tr(S_k K^-1 K_jl) / 2 - [j = k = l] b e^-u
__device__ __forceinline__ double g_k_g(const double* st, int x, int y, int z) {
  const int yz = y + z;  // K_y gamma_z: 0 -> f, 1 -> beta, 2 -> delta
  if (x == 0) return yz == 0 ? st[ST_FA] : (yz == 1 ? st[ST_AB] : st[ST_AD]);
  return yz == 0 ? st[ST_AB] : (yz == 1 ? st[ST_GB] : st[ST_GD]);
}
__device__ __forceinline__ double km_a_g(const double* st, int m, int l) {
  // (K_m alpha) . gamma_l, K_m alpha: 0 -> f, 1 -> beta, 2 -> eps2
  if (l == 0) return m == 0 ? st[ST_FA] : (m == 1 ? st[ST_AB] : st[ST_AE2]);
  return m == 0 ? st[ST_AB] : (m == 1 ? st[ST_GB] : st[ST_GE2]);
}
__device__ __forceinline__ double tr_skm(const double* st, int N, int x, int m) {
  // tr(S_x K^-1 K_m), m = number of 1 indices (0..2)
  if (x == 0) return m == 0 ? (double)N : (m == 1 ? st[ST_TRS] : st[ST_TRR2]);
  return m == 0 ? st[ST_TRS] : (m == 1 ? st[ST_TRS2] : st[ST_TRSR2]);
}
__device__ __forceinline__ double tr_km(const double* st, int N, int m) {
  return m == 0 ? (double)N : (m == 1 ? st[ST_TRS] : (m == 2 ? st[ST_TRR2] : st[ST_TRR3]));
}
__device__ __forceinline__ double tr_spow(const double* st, int N, int m) {
  return m == 0 ? (double)N : (m == 1 ? st[ST_TRS] : (m == 2 ? st[ST_TRS2] : st[ST_TRS3]));
}
__device__ __forceinline__ double a_km_a(const double* st, int m) {
  return m == 0 ? st[ST_FA] : (m == 1 ? st[ST_AB] : (m == 2 ? st[ST_AE2] : st[ST_AE3]));
}
__device__ double uuu(const double* st, int N, int j, int k, int l, double b_e) {
  double v = -g_k_g(st, j, k, l) - g_k_g(st, k, j, l) - g_k_g(st, k, l, j);
  v += km_a_g(st, j + k, l) + km_a_g(st, j + l, k) + km_a_g(st, k + l, j);
  v -= 0.5 * a_km_a(st, j + k + l);
  v -= 0.5 * tr_skm(st, N, j, k + l);
  v += 0.5 * tr_km(st, N, j + k + l);
  v += tr_spow(st, N, j + k + l);
  v -= 0.5 * tr_skm(st, N, l, j + k);
  v -= 0.5 * tr_skm(st, N, k, j + l);
  if (j == k && k == l) v -= b_e;
  return v;
}

// v_i = tr(W dH_i) for every coordinate i of one (chain, kernel), W = W2 - W1 (Eq. Betancourt_formula
// contracted with the third derivatives in the model's structure, Sec. 2.3; all O(N^2)):
//   i = f_{k,m}:  tau l'''_m sum_{a,b} W[f_a m, f_b m] - 2 (K^-1 w_0 + A1 w_1)_m
//                 + W_00 alpha_m + 2 W_01 gamma_m + W_11 fuu11_m,        w_h = W[f_k, u_kh]
//   i = u_{k,j}:  -<W[f_k, f_k], A_j> + 2 sum_h <w_h, fuu_{j h}> + sum_{h h'} W_{h h'} uuu(j, h, h')
//   with A_0 = K^-1, A_1 = A1, fuu_00 = alpha, fuu_01 = gamma, fuu_11 = fuu11.
// Grid (32-column blocks of m, chain x kernel), lane = m, the 8 warps split r (all reads coalesced);
// the f-coordinates are written here, the block's parts of the hyperparameter sums go to
// part[b][block][0..6] = (<W[f_k, f_k], K^-1>, <W[f_k, f_k], A1>, w0.alpha, w0.gamma, w1.gamma,
// w1.fuu11, unused) and k_contract_hyp adds them in a fixed order.
constexpr int kContractParts = 8;
__global__ void __launch_bounds__(256) k_contract(ModelDev md, const double* __restrict__ q, int dp,
                                                  const double* __restrict__ Wb,
                                                  const double* __restrict__ Kinvb,
                                                  const double* __restrict__ A1b,
                                                  const double* __restrict__ l3,
                                                  const double* __restrict__ alphab,
                                                  const double* __restrict__ gammab,
                                                  const double* __restrict__ fuu11b,
                                                  double* __restrict__ vout, double* __restrict__ part) {
  const int b = blockIdx.y, n = md.n, N = md.N, nN = n * N;
  const int c = b / n, k = b % n;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m = blockIdx.x * kStatCols + lane;
  const double* W = Wb + (long long)c * dp * dp;
  const long long mo = (long long)b * N * N, vo = (long long)b * N;
  const double* Kinv = Kinvb + mo;
  const double* A1 = A1b + mo;
  double* v = vout + (long long)c * dp;
  const bool hyp = md.sample_hypers != 0;
  extern __shared__ double shm[];
  double* w0 = shm;
  double* w1 = shm + N;
  __shared__ double col[8][kStatCols];
  __shared__ double red[8];
  const int u0i = nN + 2 * k, u1i = nN + 2 * k + 1;
  if (hyp)
    for (int r = threadIdx.x; r < N; r += blockDim.x) {
      w0[r] = W[(long long)(k * N + r) * dp + u0i];
      w1[r] = W[(long long)(k * N + r) * dp + u1i];
    }
  __syncthreads();
  double k01 = 0.0, t0 = 0.0, t1 = 0.0;  // (K^-1 w0 + A1 w1)_m and column m of <W[f_k, f_k], A_j>
  if (hyp && m < N)
    for (int r = w; r < N; r += 8) {
      const double kr = Kinv[(long long)r * N + m], ar = A1[(long long)r * N + m];
      const double wr = W[(long long)(k * N + r) * dp + k * N + m];
      k01 = fma(kr, w0[r], fma(ar, w1[r], k01));
      t0 = fma(wr, kr, t0);
      t1 = fma(wr, ar, t1);
    }
  k01 = column_total(k01, col);
  double pa[6] = {0, 0, 0, 0, 0, 0};
  if (w == 0 && m < N) {
    double diag = 0.0;
    for (int a = 0; a < n; ++a)
      for (int bb = 0; bb < n; ++bb) diag += W[(long long)(a * N + m) * dp + bb * N + m];
    double val = l3[(long long)c * N + m] * diag;
    if (hyp) {
      const double W00 = W[(long long)u0i * dp + u0i], W01 = W[(long long)u0i * dp + u1i],
                   W11 = W[(long long)u1i * dp + u1i];
      const double al = alphab[vo + m], ga = gammab[vo + m], fu = fuu11b[vo + m];
      val += -2.0 * k01 + W00 * al + 2.0 * W01 * ga + W11 * fu;
      pa[2] = w0[m] * al;
      pa[3] = w0[m] * ga;
      pa[4] = w1[m] * ga;
      pa[5] = w1[m] * fu;
    }
    v[k * N + m] = val;
  }
  if (!hyp) return;  // uniform per CTA
  pa[0] = t0;
  pa[1] = t1;
  double* pp = part + ((long long)b * kStatMaxBlocks + blockIdx.x) * kContractParts;
  for (int e = 0; e < 6; ++e) stat_part(pa[e], red, pp + e);
}

// The hyperparameter coordinates of tr(W dH_i) for one (chain, kernel), from the parts of k_contract:
//   v[u_kj] = -<W[f_k, f_k], A_j> + 2 sum_h <w_h, fuu_{j h}> + sum_{h h'} W_{h h'} uuu(j, h, h').
__global__ void k_contract_hyp(ModelDev md, const double* __restrict__ q, int dp,
                               const double* __restrict__ Wb, const double* __restrict__ stats,
                               const double* __restrict__ part, int nblocks, double* __restrict__ vout) {
  const int b = blockIdx.x, n = md.n, N = md.N, nN = n * N;
  const int c = b / n, k = b % n;
  if (threadIdx.x != 0 || !md.sample_hypers) return;
  double sm[6] = {0, 0, 0, 0, 0, 0};
  for (int blk = 0; blk < nblocks; ++blk)
    for (int e = 0; e < 6; ++e) sm[e] += part[((long long)b * kStatMaxBlocks + blk) * kContractParts + e];
  const double* W = Wb + (long long)c * dp * dp;
  const int u0i = nN + 2 * k, u1i = nN + 2 * k + 1;
  const double W00 = W[(long long)u0i * dp + u0i], W01 = W[(long long)u0i * dp + u1i],
               W11 = W[(long long)u1i * dp + u1i];
  const double* st = stats + (long long)b * kStatSlots;
  const KernelDev& kd = md.k[k];
  const double be0 = kd.b[0] * exp(-hyper_u(md, q, dp, c, k, 0));
  const double be1 = kd.b[1] * exp(-hyper_u(md, q, dp, c, k, 1));
  const double Wh[2][2] = {{W00, W01}, {W01, W11}};
  // <w_h, fuu_{j h}>: fuu_00 = alpha, fuu_01 = fuu_10 = gamma, fuu_11 = fuu11
  const double wf[2][2] = {{sm[2], sm[4]}, {sm[3], sm[5]}};  // [j][h]
  double* v = vout + (long long)c * dp;
  for (int j = 0; j < 2; ++j) {
    double val = -sm[j] + 2.0 * (wf[j][0] + wf[j][1]);
    const double bej = j == 0 ? be0 : be1;
    for (int h = 0; h < 2; ++h)
      for (int h2 = 0; h2 < 2; ++h2) val += Wh[h][h2] * uuu(st, N, j, h, h2, bej);
    v[nN + 2 * k + j] = val;
  }
}

}  // namespace dev
}  // namespace rmhmc
