// Warm-started ("dynamically programmed") Jacobi eigendecomposition, Sec. 2.4.
//
// Given Psi from the previous point, M = Psi^T H Psi is nearly diagonal; cyclic Jacobi drives its
// off-diagonal part below the tolerance zeta and the accumulated rotations update Psi <- Psi Q. This is
// the parallel (round-robin) block form of cyclic Jacobi: the indices are cut into nb blocks of 8;
// in each of the nb - 1 rounds of a sweep the blocks are paired by the circle method and every
// pair's 16 x 16 diagonal sub-problem is diagonalised exactly by an inner cyclic Jacobi (one warp,
// shared memory), giving an orthogonal V_P; then all pairs are applied at once as the two-sided
// block transform M[P, Q] <- V_P^T M[P, Q] V_Q (only P <= Q is computed; the mirror is written),
// and Psi^T[P, :] <- V_P^T Psi^T[P, :]. One thread-block cluster works on one chain; the rounds
// are separated by hardware cluster barriers, so the whole eigen-update (all sweeps) is one launch
// with no host round trip. M and Psi^T live in global memory (they stay in the 126 MB L2 for the
// batch sizes used); accesses are 64-byte row segments, and loads bypass L1 (ld.global.cg) so that
// writes by other CTAs of the cluster are seen after each barrier.
//
// Stopping rule (per pair, with a rounding floor; rmhmc_jacobi_rule): sweeps continue while some
// pair j != l has |m_jl| > max(zeta * den(j, l), 4 u ||M||_F), den = |m_jj m_ll| / min_i |m_ii|
// (METRIC: the first-order error that coupling puts into G^-1, W1, W2 and log|G| stays below zeta
// relative) or den = sqrt(|m_jj m_ll|) (RELATIVE: every eigenpair resolved). The test runs before
// each sweep, so an unchanged basis costs 0 sweeps; hitting max_sweeps marks the chain
// RMHMC_CHAIN_NOTCONV. A Frobenius rule ||offdiag||_F <= zeta ||M||_F would leave couplings of
// ~zeta ||H|| between the small eigenpairs, which dominate G^-1; the floor stops the rule from
// chasing rounding noise (rotations against entries of size ||M|| leave ~u ||M|| behind). In the
// dual GP model K^-1 puts ~N eigenvalues of H in a near-degenerate cluster near 1/(c jitter),
// which every change of q re-mixes: RELATIVE needs 6-10 sweeps per update there, METRIC 2-3.
// Each 2 x 2 rotation is the symmetric Schur decomposition (Golub and Van Loan, Matrix
// Computations, Sec. 8.5).
#include <cooperative_groups.h>
#include <math.h>

#include <atomic>
#include <mutex>

#include "df.cuh"
#include "internal.cuh"

namespace cg = cooperative_groups;

namespace rmhmc {

namespace {

constexpr int NW = 8;            // warps per CTA
constexpr int SB = kJacSB;       // 16
constexpr int BL = kJacBlk;      // 8
constexpr int SBP = SB + 1;
constexpr int MAX_INNER = 8;
constexpr int WARP_SMEM = 4 * SB * SBP;  // doubles per warp
constexpr int kMaxPairs = 256;           // dp <= 16 * kMaxPairs = 4096

__device__ __forceinline__ void circle_pair(int r, int p, int nb, int& I, int& J) {
  const int m1 = nb - 1;
  if (p == 0) {
    I = r;
    J = nb - 1;
  } else {
    I = (r + p) % m1;
    J = (r - p + m1) % m1;
  }
}

__device__ __forceinline__ int gidx(int I, int J, int t) { return t < BL ? I * BL + t : J * BL + (t - BL); }

// Symmetric Schur rotation zeroing A_ab: (c, s, t = s / c) with J = [[c, s], [-s, c]] on (a, b).
// The tangent t is the root of smaller magnitude of A_ab t^2 + (A_bb - A_aa) t - A_ab = 0
// (t = sign(theta) / (|theta| + sqrt(1 + theta^2)), theta = (A_bb - A_aa) / (2 A_ab)). B300's FP64
// division and square root cost tens of FP64-pipe slots each, so t is first taken in FP32 and then
// refined by one Newton step on that quadratic in FP64 (the FP32 reciprocal of the derivative is
// enough for a step of relative size 1e-7): the result is accurate to ~1e-14, so setting the
// rotated pair to zero commits an error of ~1e-14 |A_ab|. c = (1 + t^2)^-1/2 comes from the FP32
// reciprocal square root refined by two FP64 Newton steps, s = t c, so the rotation is orthogonal
// to FP64 rounding. Where theta is out of FP32 range the FP64 formulas are used.
__device__ __forceinline__ void schur2(double app, double aqq, double apq, double& c, double& s,
                                       double& t) {
  if (fabs(apq) < 1e-300) {
    c = 1.0;
    s = 0.0;
    t = 0.0;
    return;
  }
  const double num = aqq - app, den = 2.0 * apq;
  const double an = fabs(num), ad = fabs(den);
  t = 0.0;
  bool fast = ad > 1e-30 && ad < 1e30 && an < 1e30;
  if (fast) {
    const float th = __fdividef((float)num, (float)den);
    const float ath = fabsf(th);
    const float tf = ath > 1e15f ? 0.5f / th : copysignf(1.0f, th) / (ath + sqrtf(fmaf(th, th, 1.0f)));
    fast = tf != 0.0f && isfinite(tf);
    if (fast) {
      t = (double)tf;
      const double f = fma(fma(apq, t, num), t, -apq);   // A_ab t^2 + (A_bb - A_aa) t - A_ab
      const double fp = fma(2.0 * apq, t, num);          // its derivative
      t -= f * (double)__frcp_rn((float)fp);
    }
  }
  if (!fast) {
    const double theta = num / den;
    if (fabs(theta) > 1e150) t = 0.5 / theta;
    else t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(1.0 + theta * theta));
  }
  const double x = fma(t, t, 1.0);
  double y = (double)rsqrtf((float)x);
  y = y * fma(-0.5 * x, y * y, 1.5);
  y = y * fma(-0.5 * x, y * y, 1.5);
  c = y;
  s = t * y;
}

// Inner exact solve of one 16 x 16 sub-problem by a single warp: A <- V^T A V diagonal. Returns
// false when the block already met the tolerance (then V = I exactly and A is unchanged).
// Stopping test for one pair (no FP64 division): true when m_jl^2 > max(tol2 * den, floor2), with
// den = |m_jj m_ll| (RELATIVE) or (m_jj m_ll)^2 / dmin^2 (METRIC, compared as m_jl^2 dmin^2 against
// tol2 (m_jj m_ll)^2).
__device__ __forceinline__ bool pair_unconverged(double v, double djj, double dll, double tol2,
                                                 double floor2, int rule, double dmin2) {
  const double v2 = v * v;
  if (!(v2 > floor2)) return false;
  const double p = fabs(djj * dll);
  if (rule == RMHMC_JACOBI_METRIC) return v2 * dmin2 > tol2 * p * p;
  return v2 > tol2 * p;
}

// Floor for a coupling between diagonal entries x and y: 1e-13 max(|x|, |y|) (about 450 units of
// FP64 rounding of the larger entry), never above the caller's floor2. A coupling below it moves
// G^-1 by at most ~1e-13 / min(|x|, |y|) relative.
__device__ __forceinline__ double local_floor2(double x, double y, double floor2) {
  return fmin(floor2, fmax(1e-26 * fmax(x * x, y * y), 1e-300));
}

// The floor of the stopping tests: the caller's floor ~4u ||M||_F under METRIC (the sampler's
// rule: a residual coupling's effect on G^-1 is what matters, and the floor keeps the sweep count
// low); the pair-local floor under RELATIVE, whose purpose is every eigenpair resolved, the small
// ones included.
__device__ __forceinline__ double stop_floor2(double x, double y, double floor2, int rule) {
  return rule == RMHMC_JACOBI_RELATIVE ? local_floor2(x, y, floor2) : floor2;
}

__device__ bool inner_solve(double* A, double* V, double* cs, double tol2, double floor2, int rule,
                            double dmin2, unsigned int& nround) {
  const int lane = threadIdx.x & 31;
  bool rotated = false;
  for (int e = lane; e < SB * SB; e += 32) V[(e / SB) * SBP + e % SB] = (e / SB == e % SB) ? 1.0 : 0.0;
  __syncwarp();
  for (int it = 0; it < MAX_INNER; ++it) {
    bool unconv = false;
    for (int e = lane; e < SB * SB; e += 32) {
      const int i = e / SB, j = e % SB;
      const double v = A[i * SBP + j];
      if (i != j && v != 0.0) {
        const double aii = A[i * SBP + i], ajj = A[j * SBP + j];
        unconv |= pair_unconverged(v, aii, ajj, tol2, stop_floor2(aii, ajj, floor2, rule), rule, dmin2) ||
                  !isfinite(v);
      }
    }
    if (!__any_sync(0xffffffffu, unconv)) break;
    rotated = true;
    for (int r = 0; r < SB - 1; ++r) {
      // the pairs of this round above the tolerance are rotated, the others left alone; a round
      // with none to rotate is skipped (warp-uniform). Within a sweep that runs, a pair is rotated
      // unless it is at the tolerance or at the level of its own diagonal entries (local_floor2),
      // so the small eigenpairs that dominate G^-1 are resolved to their relative accuracy, not to
      // the caller's floor ~4u ||M||_F (which decides only whether another sweep runs)
      bool need = false;
      if (lane < SB / 2) {
        int a, b;
        circle_pair(r, lane, SB, a, b);
        const double app = A[a * SBP + a], aqq = A[b * SBP + b], apq = A[a * SBP + b];
        need = !isfinite(apq) || pair_unconverged(apq, app, aqq, tol2, local_floor2(app, aqq, floor2), rule, dmin2);
        double c = 1.0, sn = 0.0, t = 0.0;
        if (need) schur2(app, aqq, apq, c, sn, t);
        cs[3 * lane] = c;
        cs[3 * lane + 1] = sn;
        cs[3 * lane + 2] = t;
      }
      if (!__any_sync(0xffffffffu, need)) continue;
      ++nround;
      __syncwarp();
      // A <- J^T A J by 2 x 2 blocks, each written once with its mirror: lane l < 28 owns the
      // off-diagonal block of pairs (P, Q), P < Q; lanes 28..31 own two diagonal blocks each, whose
      // update is A_aa - t A_ab, A_bb + t A_ab and a zero coupling (the Schur rotation's identities)
      if (lane < 28) {
        int P = 0, rem = lane;
        while (rem >= SB / 2 - 1 - P) {
          rem -= SB / 2 - 1 - P;
          ++P;
        }
        const int Q = P + 1 + rem;
        int a, b, e, f;
        circle_pair(r, P, SB, a, b);
        circle_pair(r, Q, SB, e, f);
        const double cp = cs[3 * P], sp = cs[3 * P + 1], cq = cs[3 * Q], sq = cs[3 * Q + 1];
        const double x00 = A[a * SBP + e], x01 = A[a * SBP + f], x10 = A[b * SBP + e], x11 = A[b * SBP + f];
        const double y00 = cp * x00 - sp * x10, y01 = cp * x01 - sp * x11;
        const double y10 = sp * x00 + cp * x10, y11 = sp * x01 + cp * x11;
        const double z00 = cq * y00 - sq * y01, z01 = sq * y00 + cq * y01;
        const double z10 = cq * y10 - sq * y11, z11 = sq * y10 + cq * y11;
        A[a * SBP + e] = z00;
        A[e * SBP + a] = z00;
        A[a * SBP + f] = z01;
        A[f * SBP + a] = z01;
        A[b * SBP + e] = z10;
        A[e * SBP + b] = z10;
        A[b * SBP + f] = z11;
        A[f * SBP + b] = z11;
      } else {
        for (int P = 2 * (lane - 28); P < 2 * (lane - 28) + 2; ++P) {
          if (cs[3 * P + 1] == 0.0) continue;
          int a, b;
          circle_pair(r, P, SB, a, b);
          const double t = cs[3 * P + 2], apq = A[a * SBP + b];
          A[a * SBP + a] -= t * apq;
          A[b * SBP + b] += t * apq;
          A[a * SBP + b] = 0.0;
          A[b * SBP + a] = 0.0;
        }
      }
      // V <- V J
      for (int task = lane; task < (SB / 2) * SB; task += 32) {
        const int pr = task / SB, u = task % SB;
        int a, b;
        circle_pair(r, pr, SB, a, b);
        const double c = cs[3 * pr], s = cs[3 * pr + 1];
        const double va = V[u * SBP + a], vb = V[u * SBP + b];
        V[u * SBP + a] = c * va - s * vb;
        V[u * SBP + b] = s * va + c * vb;
      }
      __syncwarp();
    }
  }
  return rotated;
}

// Y = Vp^T X Vq, all 16 x 16 in shared memory (a null Vp or Vq stands for the identity); T is
// scratch.
__device__ __forceinline__ void tile_transform(const double* X, const double* Vp, const double* Vq,
                                               double* T, double* Y) {
  const int lane = threadIdx.x & 31;
  const int t = lane >> 1, u0 = (lane & 1) * 8;
  const double* src = X;
  if (Vq) {
    double acc[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j] = 0.0;
#pragma unroll 4
    for (int v = 0; v < SB; ++v) {
      const double x = X[t * SBP + v];
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[j] = fma(x, Vq[v * SBP + u0 + j], acc[j]);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) T[t * SBP + u0 + j] = acc[j];
    __syncwarp();
    src = T;
  }
  double acc[8];
  if (Vp) {
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j] = 0.0;
#pragma unroll 4
    for (int v = 0; v < SB; ++v) {
      const double p = Vp[v * SBP + t];
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[j] = fma(p, src[v * SBP + u0 + j], acc[j]);
    }
  } else {
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j] = src[t * SBP + u0 + j];
  }
  __syncwarp();
#pragma unroll
  for (int j = 0; j < 8; ++j) Y[t * SBP + u0 + j] = acc[j];
  __syncwarp();
}

// ------------------------------------------------------------------ element types
// The FP64 path keeps M and Psi^T in double; the mixed path holds them as double-float pairs
// (df.cuh) in scratch for the whole kernel, with the 16 x 16 inner solves (phase 1), the stopping
// test and the conversions in FP64 and the phase-2 tile products in double-float arithmetic.

// Y = Vp^T X Vq on 16 x 16 double-float tiles in shared memory (null Vp / Vq = identity).
__device__ __forceinline__ void tile_transform_df(const float2* X, const float2* Vp, const float2* Vq,
                                                  float2* T, float2* Y) {
  const int lane = threadIdx.x & 31;
  const int t = lane >> 1, u0 = (lane & 1) * 8;
  const float2* src = X;
  if (Vq) {
    float sh[8], cl[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) { sh[j] = 0.f; cl[j] = 0.f; }
#pragma unroll 4
    for (int v = 0; v < SB; ++v) {
      const float2 x = X[t * SBP + v];
#pragma unroll
      for (int j = 0; j < 8; ++j) dot2_step(sh[j], cl[j], x, Vq[v * SBP + u0 + j]);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) T[t * SBP + u0 + j] = df_renorm(sh[j], cl[j]);
    __syncwarp();
    src = T;
  }
  float2 out[8];
  if (Vp) {
    float sh[8], cl[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) { sh[j] = 0.f; cl[j] = 0.f; }
#pragma unroll 4
    for (int v = 0; v < SB; ++v) {
      const float2 p = Vp[v * SBP + t];
#pragma unroll
      for (int j = 0; j < 8; ++j) dot2_step(sh[j], cl[j], p, src[v * SBP + u0 + j]);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) out[j] = df_renorm(sh[j], cl[j]);
  } else {
#pragma unroll
    for (int j = 0; j < 8; ++j) out[j] = src[t * SBP + u0 + j];
  }
  __syncwarp();
#pragma unroll
  for (int j = 0; j < 8; ++j) Y[t * SBP + u0 + j] = out[j];
  __syncwarp();
}

struct ElemF64 {
  using T = double;
  static constexpr bool kPairs = false;
  static constexpr double kFloorUnit2 = 16.0 * 1.2325951644078310e-32;  // (4 u)^2, u = 2^-53
  static __device__ __forceinline__ T ld(const T* p) { return __ldcg(p); }
  static __device__ __forceinline__ void st(T* p, T v) { __stcg(p, v); }
  static __device__ __forceinline__ double join(T v) { return v; }
  static __device__ __forceinline__ T split(double v) { return v; }
  // the value the coupling criterion (a log-domain test to FP32 rounding) reads
  using CV = double;
  static __device__ __forceinline__ CV cv(T v) { return v; }
  static __device__ __forceinline__ void transform(const T* X, const T* Vp, const T* Vq, T* Tt, T* Y) {
    tile_transform(X, Vp, Vq, Tt, Y);
  }
};

struct ElemDF {
  using T = float2;
  static constexpr bool kPairs = true;
  static constexpr double kFloorUnit2 = 16.0 * 1.2621774483536189e-29;  // (4 * 2^-48)^2
  static __device__ __forceinline__ T ld(const T* p) { return __ldcg(p); }
  static __device__ __forceinline__ void st(T* p, T v) { __stcg(p, v); }
  static __device__ __forceinline__ double join(T v) { return df_join(v); }
  static __device__ __forceinline__ T split(double v) { return df_split(v); }
  // the value the coupling criterion reads: hi + lo rounded to FP32 (within 2^-24 of the pair's
  // value, below the criterion's own FP32-logarithm rounding; no FP64 instruction, whose pipe is
  // 1/64 of the FP32 rate; an unnormalised pair with hi = 0 still gives its lo)
  using CV = float;
  static __device__ __forceinline__ CV cv(T v) { return v.x + v.y; }
  static __device__ __forceinline__ void transform(const T* X, const T* Vp, const T* Vq, T* Tt, T* Y) {
    tile_transform_df(X, Vp, Vq, Tt, Y);
  }
};

template <class E>
__device__ __forceinline__ void load_tile_v(typename E::T* dst, const typename E::T* src) {
  const int lane = threadIdx.x & 31;
  for (int e = lane; e < SB * SB; e += 32) dst[(e / SB) * SBP + e % SB] = E::ld(src + e);
}

// Constants of the coupling criterion, fixed for one eigen-update: log2 of zeta^2, of the floor
// 4u ||M||_F squared and of min_i |m_ii| squared.
struct CritConst {
  float ltol2, lfloor2, ldmin2;
  int rule;
};

// The coupling criterion of the stopping rule in the log domain:
// log2(m_jl^2 / max(zeta^2 den(j, l), floor)), positive where pair_unconverged holds (to FP32
// rounding of the logarithms, ~1e-6 relative in the ratio). den = (m_jj m_ll)^2 / d_min^2 (METRIC)
// or |m_jj m_ll| (RELATIVE); the floor is the rule's (stop_floor2). A non-finite entry gives +inf
// (the caller treats it as a failed update).
// log2 |x| for a finite float, from its exponent field and the FP32 log2 of its significand; zero
// gives -2000, a subnormal the log2 of 2^-127.
__device__ __forceinline__ float log2_abs(float x) {
  const unsigned b = __float_as_uint(x) & 0x7fffffffu;
  if (b == 0) return -2000.f;
  const int e = (int)(b >> 23) - 127;
  return (float)e + __log2f(__uint_as_float(0x3f800000u | (b & 0x7fffffu)));
}

__device__ __forceinline__ float coupling_log_ratio_l(float lv, float lj, float ll, const CritConst& k);
// (double: the FP64 kernel's values; float: the double-float kernel's pairs as FP32 values)
__device__ __forceinline__ float coupling_log_ratio(double v, double djj, double dll, const CritConst& k) {
  if (!isfinite(v)) return INFINITY;
  return coupling_log_ratio_l(log2_abs(v), log2_abs(djj), log2_abs(dll), k);
}
__device__ __forceinline__ float coupling_log_ratio(float v, float djj, float dll, const CritConst& k) {
  if (!isfinite(v)) return INFINITY;
  return coupling_log_ratio_l(log2_abs(v), log2_abs(djj), log2_abs(dll), k);
}
__device__ __forceinline__ float coupling_log_ratio_l(float lv, float lj, float ll, const CritConst& k) {
  float lthr, lfl;
  if (k.rule == RMHMC_JACOBI_METRIC) {
    lthr = k.ltol2 + 2.f * (lj + ll) - k.ldmin2;
    lfl = k.lfloor2;
  } else {
    lthr = k.ltol2 + lj + ll;
    // local_floor2: min(floor2, max(1e-26 max(x^2, y^2), 1e-300))
    lfl = fminf(k.lfloor2, fmaxf(-86.37013f + 2.f * fmaxf(lj, ll), -996.578f));
  }
  return 2.f * lv - fmaxf(lthr, lfl);
}

// warp-wide maximum (every lane receives it)
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

constexpr int kTop = 4;              // partners kept per block for the dynamic matching
constexpr int kMaxBlocks = 2 * kMaxPairs;

// Warm-started block Jacobi, both schedules (sched: RMHMC_JACOBI_CYCLIC or RMHMC_JACOBI_DYNAMIC).
//
// CYCLIC: each sweep is nb - 1 rounds of the circle pairing (every block pair once per sweep);
// the stopping test runs before each sweep.
// DYNAMIC: the kernel keeps, per pair of 8-wide blocks (I, J), the largest coupling ratio of their
// 8 x 8 block of M (crit, nb x nb floats per chain, symmetric; the diagonal entry is the block's own
// internal coupling). It is computed for all blocks by the stopping test and updated in phase 2
// for every tile that a round rewrites, from the tile's new values and the new diagonal. Each round
// then pairs the blocks greedily, largest coupling first (every CTA of the cluster computes the same
// matching from the same crit): each block's kTop most coupled partners are found, the blocks whose
// largest coupling or internal coupling is above 1 are taken in decreasing order and matched with
// their most coupled free partner; the remaining blocks are paired in index order. Only pairs with a
// coupling above 1 are solved in phase 1 (typically a few per round instead of nb / 2), and phase 2
// applies only their rotations. Rounds continue while some pair is above 1; the stopping test then
// re-checks every block with the current diagonal (it decides convergence exactly as in the cyclic
// schedule). sweeps_out reports rounds / (nb - 1) rounded up (cyclic-sweep equivalents), and
// max_sweeps bounds the rounds at max_sweeps (nb - 1).
template <class E>
__global__ void __launch_bounds__(NW * 32)
    k_jacobi_t(double* __restrict__ Mb, double* __restrict__ Pb, double* __restrict__ lamb, int dp, int d,
               int rule, double tol, int max_sweeps, int* __restrict__ status, int* __restrict__ sweeps_out,
               int* __restrict__ sweeps_acc, double* __restrict__ Vb, double* __restrict__ Db,
               double* __restrict__ slotsb, int* __restrict__ flagsb,
               unsigned long long* __restrict__ tiles, typename E::T* __restrict__ Mwb,
               typename E::T* __restrict__ Pwb, float* __restrict__ critb, int sched,
               const int* __restrict__ pre) {
  using T = typename E::T;
  static_assert(sizeof(T) == sizeof(double), "tiles of V and D are stored in double-sized slots");
  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int chain = blockIdx.x / C;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nb = dp / BL, np = nb / 2;
  const bool dyn = sched == RMHMC_JACOBI_DYNAMIC && critb != nullptr;
  if (np > kMaxPairs) {  // larger than any model or batch the library accepts
    if (rank == 0 && tid == 0) {
      atomicOr(&status[chain], RMHMC_CHAIN_NOTCONV);
      sweeps_out[chain] = 0;
    }
    return;  // uniform for the whole cluster
  }
  if (status[chain] != 0) {
    if (rank == 0 && tid == 0) sweeps_out[chain] = 0;
    return;  // uniform for the whole cluster
  }
  const long long DD = (long long)dp * dp;
  double* M = Mb + (long long)chain * DD;
  double* P = Pb + (long long)chain * DD;
  T* Mw = E::kPairs ? Mwb + (long long)chain * DD : reinterpret_cast<T*>(M);
  T* Pw = E::kPairs ? Pwb + (long long)chain * DD : reinterpret_cast<T*>(P);
  T* V = reinterpret_cast<T*>(Vb + (long long)chain * np * SB * SB);
  T* D = reinterpret_cast<T*>(Db + (long long)chain * np * SB * SB);
  double* slots = slotsb + (long long)chain * 64;
  int* flags = flagsb + (long long)chain * np;
  float* crit = dyn ? critb + (long long)chain * nb * nb : nullptr;
  extern __shared__ double smem[];
  double* ws = smem + warp * WARP_SMEM;
  double* Xd = ws;                    // phase 1 (FP64)
  double* Vd = ws + 2 * SB * SBP;
  T* X = reinterpret_cast<T*>(ws);    // phase 2, same bytes
  T* Tt = reinterpret_cast<T*>(ws + SB * SBP);
  T* Va = reinterpret_cast<T*>(ws + 2 * SB * SBP);
  T* Vq = reinterpret_cast<T*>(ws + 3 * SB * SBP);
  __shared__ double red[2][NW];
  __shared__ double cs[NW][3 * SB / 2];  // (c, s, t) of the 8 rotations of a round, per warp
  __shared__ unsigned char sflag[kMaxPairs];  // pair rotated in this round
  __shared__ short sact[kMaxPairs];           // the rotated pairs, in order
  __shared__ int scum[kMaxPairs];             // cumulative active M tiles per column
  __shared__ int snact;
  __shared__ short2 spair[kMaxPairs];         // the two blocks of pair p in this round
  __shared__ unsigned char sneed[kMaxPairs];  // pair p is solved in phase 1 of this round
  __shared__ short ssolve[kMaxPairs];         // the pairs solved, in order
  __shared__ int snsolve, snmatch, sbad;
  __shared__ typename E::CV sdg[NW][2 * SB];  // phase 2: new diagonal of a tile's rows and columns
  // dynamic matching
  __shared__ float stopv[kMaxBlocks][kTop];
  __shared__ short stopj[kMaxBlocks][kTop];
  __shared__ float sown[kMaxBlocks];
  __shared__ float skey[kMaxBlocks];
  __shared__ short sorder[kMaxBlocks];
  __shared__ unsigned char sused[kMaxBlocks];

  if constexpr (E::kPairs) {
    // (chains flagged in pre arrive with M and Psi^T already in the pair buffers)
    if (!(pre && pre[chain]))
      for (long long e = (long long)rank * blockDim.x + tid; e < DD; e += (long long)C * blockDim.x) {
        E::st(Mw + e, E::split(__ldcg(M + e)));
        E::st(Pw + e, E::split(__ldcg(P + e)));
      }
    cluster.sync();
  }

  const int gw = rank * NW + warp, nwt = C * NW;
  const int nct = dp / SB;
  const int max_rounds = max_sweeps * (nb - 1);
  int sweeps = 0;           // cyclic: sweeps run
  int rounds = 0;           // dynamic: rounds run
  bool converged = false, failed = false;
  double tot0 = 0.0;        // ||M||_F^2 from the first pass
  unsigned int ntile = 0;   // 16 x 16 x 16 tile products this warp executed (phase 2)
  unsigned int nround = 0;  // rounds of 8 rotations this warp applied to a 16 x 16 block (phase 1)
  unsigned int nsolved = 0, nrotated = 0;  // 16 x 16 sub-problems this warp solved / that rotated
  for (int pass = 0;; ++pass) {
    // ---- convergence test. Pass 1: ||M||_F^2 and min_i<d |m_ii|. Pass 2: the coupling criterion
    //      under the chosen rule, with floor = 4 u ||M||_F (rounding level); the dynamic schedule
    //      also records it per 8 x 8 block. ||M||_F is invariant under the rotations: summed over
    //      M in the first pass only; later passes read the diagonal (a non-finite diagonal entry
    //      still poisons tot)
    double tot = 0.0, dmin = 1e308;
    if (pass == 0) {
      // (pairs: the FP32 values, one FP64 conversion and FMA each for ||M||_F^2, which only sets
      // the rounding floor)
      for (long long e = (long long)rank * blockDim.x + tid; e < DD; e += (long long)C * blockDim.x) {
        const double v = E::kPairs ? (double)E::cv(E::ld(Mw + e)) : E::join(E::ld(Mw + e));
        tot = fma(v, v, tot);
        const int i = (int)(e / dp);
        if (i < d && (long long)i * dp + i == e) dmin = fmin(dmin, fabs(v));
      }
    } else {
      for (int i = rank * blockDim.x + tid; i < d; i += C * blockDim.x) {
        const double v = E::join(E::ld(Mw + (long long)i * dp + i));
        if (!isfinite(v)) tot = v;
        dmin = fmin(dmin, fabs(v));
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      tot += __shfl_xor_sync(0xffffffffu, tot, o);
      dmin = fmin(dmin, __shfl_xor_sync(0xffffffffu, dmin, o));
    }
    if (lane == 0) { red[0][warp] = tot; red[1][warp] = dmin; }
    __syncthreads();
    if (tid == 0) {
      double a = 0.0, b = 1e308;
      for (int w = 0; w < NW; ++w) { a += red[0][w]; b = fmin(b, red[1][w]); }
      __stcg(slots + (pass & 1) * 32 + 2 * rank, a);
      __stcg(slots + (pass & 1) * 32 + 2 * rank + 1, b);
    }
    cluster.sync();
    tot = 0.0;
    dmin = 1e308;
    for (int r = 0; r < C; ++r) {
      tot += __ldcg(slots + (pass & 1) * 32 + 2 * r);
      dmin = fmin(dmin, __ldcg(slots + (pass & 1) * 32 + 2 * r + 1));
    }
    if (pass == 0) tot0 = tot;
    else if (isfinite(tot)) tot = tot0;
    const double dmin2 = fmax(dmin * dmin, 1e-300);
    const double floor2 = fmax(E::kFloorUnit2 * tot, 1e-300);
    const double tol2 = tol * tol;
    const CritConst ck{log2_abs(tol2), log2_abs(floor2), log2_abs(dmin2), rule};
    double critv = 0.0, bad = isfinite(tot) ? 0.0 : 1.0;
    if (dyn) {
      // one warp per 8 x 8 block (I <= J; the diagonal block's upper triangle)
      for (int bi = gw; bi < nb * nb; bi += nwt) {
        const int I = bi / nb, J = bi % nb;
        if (I > J) continue;
        float rmax = -INFINITY;
        bool nf = false;
        for (int e = lane; e < BL * BL; e += 32) {
          const int a = e / BL, b = e % BL;
          if (I == J && a >= b) continue;
          const int j = I * BL + a, l = J * BL + b;
          const typename E::CV v = E::cv(E::ld(Mw + (long long)j * dp + l));
          if (v == 0) continue;
          if (!isfinite(v)) { nf = true; continue; }
          const typename E::CV djj = E::cv(E::ld(Mw + (long long)j * dp + j));
          const typename E::CV dll = E::cv(E::ld(Mw + (long long)l * dp + l));
          rmax = fmaxf(rmax, coupling_log_ratio(v, djj, dll, ck));
        }
        rmax = warp_max(rmax);
        nf = __any_sync(0xffffffffu, nf);
        if (lane == 0) {
          __stcg(crit + (long long)I * nb + J, rmax);
          __stcg(crit + (long long)J * nb + I, rmax);
        }
        if (rmax > 0.f) critv = 1.0;
        if (nf || rmax == INFINITY) bad = 1.0;
      }
    } else {
      for (long long e = (long long)rank * blockDim.x + tid; e < DD; e += (long long)C * blockDim.x) {
        const int j = (int)(e / dp), l = (int)(e % dp);
        if (j >= l) continue;  // M is kept symmetric: the upper triangle decides
        if constexpr (E::kPairs) {
          // the log-domain criterion on the pairs' FP32 values (as the dynamic schedule's test)
          const float v = E::cv(E::ld(Mw + e));
          if (v == 0.f) continue;
          if (!isfinite(v)) bad = 1.0;
          if (coupling_log_ratio(v, E::cv(E::ld(Mw + (long long)j * dp + j)),
                                 E::cv(E::ld(Mw + (long long)l * dp + l)), ck) > 0.f)
            critv = 1.0;
        } else {
          const double v = E::join(E::ld(Mw + e));
          if (v == 0.0) continue;
          if (!isfinite(v)) bad = 1.0;
          const double djj = E::join(E::ld(Mw + (long long)j * dp + j));
          const double dll = E::join(E::ld(Mw + (long long)l * dp + l));
          if (pair_unconverged(v, djj, dll, tol2, stop_floor2(djj, dll, floor2, rule), rule, dmin2))
            critv = 1.0;
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      critv = fmax(critv, __shfl_xor_sync(0xffffffffu, critv, o));
      bad = fmax(bad, __shfl_xor_sync(0xffffffffu, bad, o));
    }
    __syncthreads();
    if (lane == 0) { red[0][warp] = critv; red[1][warp] = bad; }
    __syncthreads();
    if (tid == 0) {
      double a = 0.0, b = 0.0;
      for (int w = 0; w < NW; ++w) { a = fmax(a, red[0][w]); b = fmax(b, red[1][w]); }
      __stcg(slots + (pass & 1) * 32 + 16 + 2 * rank, a);
      __stcg(slots + (pass & 1) * 32 + 16 + 2 * rank + 1, b);
    }
    cluster.sync();
    critv = 0.0;
    bad = 0.0;
    for (int r = 0; r < C; ++r) {
      critv = fmax(critv, __ldcg(slots + (pass & 1) * 32 + 16 + 2 * r));
      bad = fmax(bad, __ldcg(slots + (pass & 1) * 32 + 16 + 2 * r + 1));
    }
    if (bad != 0.0 || failed) break;
    if (critv == 0.0) { converged = true; break; }
    if (dyn ? rounds >= max_rounds : sweeps >= max_sweeps) break;
    const double itol2 = 1e-4 * tol2;  // inner problems are solved 100x tighter
    const int rounds0 = rounds;

    for (int r = 0; dyn || r < nb - 1; ++r) {
      if (dyn && rounds >= max_rounds) break;
      // ---- the pairs of this round (every CTA of the cluster computes the same table)
      if (!dyn) {
        for (int p = tid; p < np; p += blockDim.x) {
          int I, J;
          circle_pair(r, p, nb, I, J);
          spair[p] = make_short2((short)I, (short)J);
          sneed[p] = 1;
          ssolve[p] = (short)p;
        }
        if (tid == 0) snsolve = np;
        __syncthreads();
      } else {
        if (tid == 0) sbad = 0;
        __syncthreads();
        // (1) per block: its internal coupling and its kTop most coupled partners
        for (int I = warp; I < nb; I += NW) {
          float rv[kMaxBlocks / 32];
#pragma unroll
          for (int k = 0; k < kMaxBlocks / 32; ++k) {
            const int J = lane + 32 * k;
            rv[k] = (J < nb && J != I) ? __ldcg(crit + (long long)I * nb + J) : -INFINITY;
          }
          const float own = __ldcg(crit + (long long)I * nb + I);
          bool nf = own == INFINITY;
#pragma unroll
          for (int k = 0; k < kMaxBlocks / 32; ++k) nf |= rv[k] == INFINITY;
          if (__any_sync(0xffffffffu, nf) && lane == 0) sbad = 1;
#pragma unroll 1
          for (int t = 0; t < kTop; ++t) {
            float bv = -INFINITY;
            int bj = -1;
#pragma unroll
            for (int k = 0; k < kMaxBlocks / 32; ++k)
              if (rv[k] > bv) { bv = rv[k]; bj = lane + 32 * k; }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {  // largest value, then smallest block index
              const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
              const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
              if (ov > bv || (ov == bv && oj >= 0 && (bj < 0 || oj < bj))) { bv = ov; bj = oj; }
            }
            if (lane == 0) { stopv[I][t] = bv; stopj[I][t] = (short)bj; }
#pragma unroll
            for (int k = 0; k < kMaxBlocks / 32; ++k)
              if (lane + 32 * k == bj) rv[k] = -INFINITY;
          }
          if (lane == 0) { sown[I] = own; sused[I] = 0; }
        }
        __syncthreads();
        // (2) the candidate blocks (largest or internal coupling above 1), in decreasing order
        for (int I = tid; I < nb; I += blockDim.x) {
          const float k0 = fmaxf(stopv[I][0], sown[I]);
          skey[I] = k0 > 0.f ? k0 : 0.f;
        }
        __syncthreads();
        int K = 0;
        for (int base = 0; base < nb; base += blockDim.x) {
          const int I = base + tid;
          const float kI = I < nb ? skey[I] : 0.f;
          if (kI > 0.f) {
            int rk = 0;
            for (int J = 0; J < nb; ++J) {
              const float kJ = skey[J];
              rk += (kJ > kI || (kJ == kI && J < I)) ? 1 : 0;
            }
            sorder[rk] = (short)I;
          }
          K += __syncthreads_count(kI > 0.f);
        }
        // (3) greedy matching, largest first
        if (tid == 0) {
          int nm = 0;
          for (int k = 0; k < K; ++k) {
            const int I = sorder[k];
            if (sused[I]) continue;
            const bool any_partner = sown[I] > 0.f;
            for (int t = 0; t < kTop; ++t) {
              const int J = stopj[I][t];
              if (J < 0 || (!(stopv[I][t] > 0.f) && !any_partner)) break;
              if (!sused[J]) {
                sused[I] = sused[J] = 1;
                spair[nm] = make_short2((short)min(I, J), (short)max(I, J));
                ++nm;
                break;
              }
            }
          }
          snmatch = nm;
        }
        __syncthreads();
        // (4) the other blocks paired in index order; a pair is solved if it was matched, or if
        //     one of its blocks or their coupling is above 1; then the list of pairs to solve
        if (warp == 0) {
          int nfree = 0;
          for (int b0 = 0; b0 < nb; b0 += 32) {
            const int b = b0 + lane;
            const bool f = b < nb && !sused[b];
            const unsigned bal = __ballot_sync(0xffffffffu, f);
            if (f) sorder[nfree + __popc(bal & ((1u << lane) - 1u))] = (short)b;
            nfree += __popc(bal);
          }
          __syncwarp();
          const int nm = snmatch;
          for (int i = lane; i < nm; i += 32) sneed[i] = 1;
          for (int i = lane; i < nfree / 2; i += 32) {
            const int a = sorder[2 * i], b = sorder[2 * i + 1];
            spair[nm + i] = make_short2((short)a, (short)b);
            sneed[nm + i] = (sown[a] > 0.f || sown[b] > 0.f || __ldcg(crit + (long long)a * nb + b) > 0.f) ? 1 : 0;
          }
          __syncwarp();
          int ns = 0;
          for (int p0 = 0; p0 < np; p0 += 32) {
            const int p = p0 + lane;
            const bool f = p < np && sneed[p];
            const unsigned bal = __ballot_sync(0xffffffffu, f);
            if (f) ssolve[ns + __popc(bal & ((1u << lane) - 1u))] = (short)p;
            ns += __popc(bal);
          }
          if (lane == 0) snsolve = ns;
        }
        __syncthreads();
        if (sbad) { failed = true; break; }   // a non-finite coupling: the test pass reports it
        if (snsolve == 0) break;              // no coupling above 1 left: re-check and stop
      }
      // ---- phase 1: exact 16 x 16 solves, one warp per pair to solve, dealt to the cluster's CTAs
      //      in turn (warp w of CTA r takes solves w C + r, ...) so that the FP64-heavy solves of a
      //      round with few of them spread over the cluster's SMs instead of sharing one SM's FP64 pipe
      const int nsolve = snsolve;
      for (int k = warp * C + rank; k < nsolve; k += nwt) {
        const int p = ssolve[k];
        const int I = spair[p].x, J = spair[p].y;
        for (int e = lane; e < SB * SB; e += 32) {
          const int a = e / SB, b = e % SB;
          Xd[a * SBP + b] = E::join(E::ld(Mw + (long long)gidx(I, J, a) * dp + gidx(I, J, b)));
        }
        __syncwarp();
        const bool rot = inner_solve(Xd, Vd, cs[warp], itol2, floor2, rule, dmin2, nround);
        ++nsolved;
        nrotated += rot ? 1u : 0u;
        if (rot) {
          for (int e = lane; e < SB * SB; e += 32) {
            const int a = e / SB, b = e % SB;
            E::st(V + (long long)p * SB * SB + e, E::split(Vd[a * SBP + b]));
            E::st(D + (long long)p * SB * SB + e, E::split(Xd[a * SBP + b]));
          }
        }
        if (lane == 0) __stcg(flags + p, rot ? 1 : 0);
        __syncwarp();
      }
      for (int p = gw; p < np; p += nwt)
        if (!sneed[p] && lane == 0) __stcg(flags + p, 0);
      cluster.sync();
      // ---- the pairs rotated in phase 1, in order (every CTA of the cluster builds the same list)
      // and, per column Q of M's tiles, the cumulative count of active tiles (P <= Q with P or Q
      // rotated): column Q holds Q + 1 of them if Q rotated, else as many as rotated pairs P < Q
      if (warp == 0) {
        int base = 0, run = 0;
        for (int p0 = 0; p0 < np; p0 += 32) {
          const int p = p0 + lane;
          const bool f = p < np && __ldcg(flags + p) != 0;
          const unsigned bal = __ballot_sync(0xffffffffu, f);
          const int before = base + __popc(bal & ((1u << lane) - 1u));  // rotated pairs < p
          if (p < np) sflag[p] = f ? 1 : 0;
          if (f) sact[before] = (short)p;
          int c = p < np ? (f ? p + 1 : before) : 0;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {  // inclusive warp scan
            const int v = __shfl_up_sync(0xffffffffu, c, o);
            if (lane >= o) c += v;
          }
          if (p < np) scum[p] = run + c;
          run += __shfl_sync(0xffffffffu, c, 31);
          base += __popc(bal);
        }
        if (lane == 0) snact = base;
      }
      __syncthreads();
      // ---- phase 2: apply all rotations to M (P <= Q tiles) and to the rows of Psi^T over the
      //      active jobs only, dealt round-robin to the cluster's warps: the M tiles (P <= Q) of
      //      which P or Q rotated, then the Psi^T row tiles of the rotated pairs. The dynamic
      //      schedule records the new coupling criterion of every 8 x 8 block it rewrites.
      const int k = scum[np - 1];  // active M tiles
      for (int i = gw; i < k; i += nwt) {
        int lo = 0, hi = np - 1;  // the column: smallest Q with scum[Q] > i
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (scum[mid] > i) hi = mid;
          else lo = mid + 1;
        }
        const int Q = lo, o = i - (Q > 0 ? scum[Q - 1] : 0);
        const int fQ = sflag[Q];
        const int Pp = fQ ? o : sact[o];
        const int fP = sflag[Pp];
        const int I1 = spair[Pp].x, J1 = spair[Pp].y, I2 = spair[Q].x, J2 = spair[Q].y;
        if (Pp == Q) {
          const T* Dp = D + (long long)Pp * SB * SB;
          for (int e = lane; e < SB * SB; e += 32) {
            const int a = e / SB, b = e % SB;
            E::st(Mw + (long long)gidx(I1, J1, a) * dp + gidx(I1, J1, b), E::ld(Dp + e));
          }
          if (dyn) {
            // blocks (I1, I1), (I1, J1), (J1, J1) of the solved 16 x 16 block (upper triangle)
            float r00 = -INFINITY, r01 = -INFINITY, r11 = -INFINITY;
            for (int e = lane; e < SB * SB; e += 32) {
              const int a = e / SB, b = e % SB;
              if (a >= b) continue;
              const typename E::CV v = E::cv(E::ld(Dp + e));
              if (v == 0) continue;
              const float rr = coupling_log_ratio(v, E::cv(E::ld(Dp + a * SB + a)), E::cv(E::ld(Dp + b * SB + b)), ck);
              if (b < BL) r00 = fmaxf(r00, rr);
              else if (a >= BL) r11 = fmaxf(r11, rr);
              else r01 = fmaxf(r01, rr);
            }
            r00 = warp_max(r00);
            r01 = warp_max(r01);
            r11 = warp_max(r11);
            if (lane == 0) {
              __stcg(crit + (long long)I1 * nb + I1, r00);
              __stcg(crit + (long long)J1 * nb + J1, r11);
              __stcg(crit + (long long)I1 * nb + J1, r01);
              __stcg(crit + (long long)J1 * nb + I1, r01);
            }
          }
        } else {
          for (int e = lane; e < SB * SB; e += 32) {
            const int a = e / SB, b = e % SB;
            X[a * SBP + b] = E::ld(Mw + (long long)gidx(I1, J1, a) * dp + gidx(I2, J2, b));
          }
          if (fP) load_tile_v<E>(Va, V + (long long)Pp * SB * SB);
          if (fQ) load_tile_v<E>(Vq, V + (long long)Q * SB * SB);
          if (dyn) {
            // the diagonal after this round: from D for a rotated pair, else M's (unchanged)
            const int pq = lane < SB ? Pp : Q, a = lane & (SB - 1);
            const bool fr = lane < SB ? fP : fQ;
            const int I = lane < SB ? I1 : I2, J = lane < SB ? J1 : J2;
            sdg[warp][lane] = fr ? E::cv(E::ld(D + (long long)pq * SB * SB + a * SB + a))
                                 : E::cv(E::ld(Mw + (long long)gidx(I, J, a) * dp + gidx(I, J, a)));
          }
          __syncwarp();
          E::transform(X, fP ? Va : nullptr, fQ ? Vq : nullptr, Tt, X);
          ntile += (fP ? 1u : 0u) + (fQ ? 1u : 0u);
          const int t = lane >> 1, u0 = (lane & 1) * 8;
#pragma unroll
          for (int j = 0; j < 8; ++j)
            E::st(Mw + (long long)gidx(I1, J1, t) * dp + gidx(I2, J2, u0 + j), X[t * SBP + u0 + j]);
#pragma unroll
          for (int j = 0; j < 8; ++j)
            E::st(Mw + (long long)gidx(I2, J2, t) * dp + gidx(I1, J1, u0 + j), X[(u0 + j) * SBP + t]);
          if (dyn) {
            // lane (t, u0) covers 8 entries of one 8 x 8 block: rows of block (t < 8 ? I1 : J1),
            // columns of block (u0 < 8 ? I2 : J2); lanes 2, 4, 8 apart share it
            float rr = -INFINITY;
            const typename E::CV djj = sdg[warp][t];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const typename E::CV v = E::cv(X[t * SBP + u0 + j]);
              if (v != 0) rr = fmaxf(rr, coupling_log_ratio(v, djj, sdg[warp][SB + u0 + j], ck));
            }
            rr = fmaxf(rr, __shfl_xor_sync(0xffffffffu, rr, 2));
            rr = fmaxf(rr, __shfl_xor_sync(0xffffffffu, rr, 4));
            rr = fmaxf(rr, __shfl_xor_sync(0xffffffffu, rr, 8));
            if ((lane & 14) == 0) {
              const int rb = t < BL ? I1 : J1, cb = u0 < BL ? I2 : J2;
              __stcg(crit + (long long)rb * nb + cb, rr);
              __stcg(crit + (long long)cb * nb + rb, rr);
            }
          }
        }
        __syncwarp();
      }
      const int nPsi = snact * nct;
      for (int j = ((gw - k) % nwt + nwt) % nwt; j < nPsi; j += nwt) {
        const int Pp = sact[j / nct], ct = j % nct;
        const int I1 = spair[Pp].x, J1 = spair[Pp].y;
        for (int e = lane; e < SB * SB; e += 32) {
          const int a = e / SB, b = e % SB;
          X[a * SBP + b] = E::ld(Pw + (long long)gidx(I1, J1, a) * dp + ct * SB + b);
        }
        load_tile_v<E>(Va, V + (long long)Pp * SB * SB);
        __syncwarp();
        E::transform(X, Va, nullptr, Tt, X);
        ++ntile;
        const int t = lane >> 1, u0 = (lane & 1) * 8;
#pragma unroll
        for (int j2 = 0; j2 < 8; ++j2)
          E::st(Pw + (long long)gidx(I1, J1, t) * dp + ct * SB + u0 + j2, X[t * SBP + u0 + j2]);
        __syncwarp();
      }
      cluster.sync();
      ++rounds;
    }
    // the selection and the test use the same criterion, so a pass that found a coupling above the
    // tolerance always runs a round; should none run, stop (reported as not converged)
    if (dyn && rounds == rounds0) break;
    ++sweeps;
  }
  if constexpr (E::kPairs) {
    for (long long e = (long long)rank * blockDim.x + tid; e < DD; e += (long long)C * blockDim.x) {
      __stcg(M + e, E::join(E::ld(Mw + e)));
      __stcg(P + e, E::join(E::ld(Pw + e)));
    }
  }
  for (int i = rank * blockDim.x + tid; i < dp; i += C * blockDim.x)
    lamb[(long long)chain * dp + i] = E::join(E::ld(Mw + (long long)i * dp + i));
  if (tiles && lane == 0) {
    unsigned long long* t = tiles + (long long)kJacStats * chain;
    if (ntile) atomicAdd(t + 0, (unsigned long long)ntile);
    if (nround) atomicAdd(t + 1, (unsigned long long)nround);
    if (nsolved) atomicAdd(t + 3, (unsigned long long)nsolved);
    if (nrotated) atomicAdd(t + 4, (unsigned long long)nrotated);
    if (rank == 0 && warp == 0) {
      atomicAdd(t + 2, (unsigned long long)rounds);
      atomicAdd(t + 5, 1ull);
    }
  }
  if (rank == 0 && tid == 0) {
    const int sw = dyn ? (rounds + nb - 2) / (nb - 1) : sweeps;
    sweeps_out[chain] = sw;
    if (sweeps_acc) sweeps_acc[chain] += sw;
    if (!converged) atomicOr(&status[chain], RMHMC_CHAIN_NOTCONV);
  }
}

// Right-looking modified Gram-Schmidt on the first d rows of Psi^T, one cluster per chain:
// at step j every later row k loses its component along row j (using ||row_j||^2, so row j need
// not be normalised yet); the rows are normalised at the end.
__global__ void __launch_bounds__(NW * 32) k_mgs(double* __restrict__ Pb, int dp, int d,
                                                const int* __restrict__ eig_count, int every) {
  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int chain = blockIdx.x / C;
  const int cnt = eig_count[chain];
  if (every <= 0 || cnt <= 0 || (cnt % every) != 0) return;  // uniform per cluster
  double* P = Pb + (long long)chain * dp * dp;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int gw = rank * NW + warp, nwt = C * NW;
  for (int j = 0; j + 1 < d; ++j) {
    const double* rj = P + (long long)j * dp;
    for (int k = j + 1 + gw; k < d; k += nwt) {
      double* rk = P + (long long)k * dp;
      double nj = 0.0, dot = 0.0;
      for (int c = lane; c < dp; c += 32) {
        const double a = __ldcg(rj + c);
        nj += a * a;
        dot += a * __ldcg(rk + c);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        nj += __shfl_xor_sync(0xffffffffu, nj, o);
        dot += __shfl_xor_sync(0xffffffffu, dot, o);
      }
      const double coef = dot / nj;
      for (int c = lane; c < dp; c += 32) __stcg(rk + c, __ldcg(rk + c) - coef * __ldcg(rj + c));
    }
    cluster.sync();
  }
  for (int k = gw; k < d; k += nwt) {
    double* rk = P + (long long)k * dp;
    double nk = 0.0;
    for (int c = lane; c < dp; c += 32) {
      const double a = __ldcg(rk + c);
      nk += a * a;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nk += __shfl_xor_sync(0xffffffffu, nk, o);
    const double inv = 1.0 / sqrt(nk);
    for (int c = lane; c < dp; c += 32) __stcg(rk + c, __ldcg(rk + c) * inv);
  }
}

// ------------------------------------------------------------------ allocation-free variant
// Workspace of rmhmc_eigh_noalloc: one file-scope device array shared by every call on a device.
constexpr size_t kNoAllocDoubles = size_t(1) << 20;  // 8 MiB
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];
constexpr int kMaxDevices = 64;
std::atomic<double*> g_noalloc_ptr[kMaxDevices] = {};
std::mutex g_noalloc_mutex;

// M = A zero-padded to dp x dp, PsiT = I, status = 0 (the workspace keeps the previous call's
// contents, so everything the solver reads is rewritten here).
__global__ void k_noalloc_pack(const double* __restrict__ A, int d, int dp, int n, double* __restrict__ M,
                               double* __restrict__ P, int* __restrict__ status) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n * dp * dp) return;
  const long long c = e / ((long long)dp * dp), r = e % ((long long)dp * dp);
  const int i = (int)(r / dp), j = (int)(r % dp);
  M[e] = (i < d && j < d) ? A[c * d * d + (long long)i * d + j] : 0.0;
  P[e] = (i == j) ? 1.0 : 0.0;
  if (r == 0) status[c] = 0;
}

// lam (n x d) from the padded eigenvalues; Q (n x d x d) with the eigenvectors as columns.
__global__ void k_noalloc_unpack(const double* __restrict__ lamp, const double* __restrict__ P, int d,
                                 int dp, int n, double* __restrict__ lam, double* __restrict__ Q) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n * d * d) return;
  const long long c = e / ((long long)d * d), r = e % ((long long)d * d);
  const int i = (int)(r / d), j = (int)(r % d);
  if (Q) Q[e] = P[c * dp * dp + (long long)j * dp + i];
  if (lam && i == 0) lam[c * d + j] = lamp[c * dp + j];
}

template <typename K, typename... Args>
cudaError_t launch_cluster(K kernel, int n_chains, int C, size_t smem, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(n_chains * C, 1, 1);
  cfg.blockDim = dim3(NW * 32, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

}  // namespace

size_t noalloc_doubles(int n, int dp) {
  const size_t np = (size_t)dp / BL / 2;
  const size_t ints = 2 * (size_t)n + (size_t)n * np;  // status, sweeps, flags
  return 2 * (size_t)n * dp * dp + (size_t)n * dp + 2 * (size_t)n * np * SB * SB + (size_t)n * 64 +
         (ints + 1) / 2 + 4;
}

// CTAs per chain: the largest of 8, 4, 2, 1 that keeps n_chains x cluster within two CTAs per SM
// (a CTA holds 256 threads x 128 registers, half of an SM's register file), so that every SM runs
// two CTAs (16 warps) and the barrier and latency stalls of one hide behind the other.
int jacobi_cluster_size(int n_chains) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 148;
  }
  for (int c = 8; c > 1; c >>= 1)
    if ((long long)n_chains * c <= 2LL * sms) return c;
  return 1;
}

void jacobi_f64(cudaStream_t s, double* M, double* PsiT, double* lam, int dp, int d, int n_chains,
                int rule, double tol, int max_sweeps, int* status, int* sweeps_out, int* sweeps_acc,
                JacobiWork w, int cluster, int sched) {
  const size_t smem = (size_t)NW * WARP_SMEM * sizeof(double);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_jacobi_t<ElemF64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr_set = true;
  }
  launch_cluster(k_jacobi_t<ElemF64>, n_chains, cluster, smem, s, M, PsiT, lam, dp, d, rule, tol, max_sweeps,
                 status, sweeps_out, sweeps_acc, w.V, w.D, w.slots, w.flags, w.tiles, (double*)nullptr,
                 (double*)nullptr, w.crit, sched, (const int*)nullptr);
}

void jacobi_df(cudaStream_t s, double* M, double* PsiT, double* lam, int dp, int d, int n_chains,
               int rule, double tol, int max_sweeps, int* status, int* sweeps_out, int* sweeps_acc,
               JacobiWork w, int cluster, double* pair_scratch_M, double* pair_scratch_P, int sched,
               const int* pre) {
  const size_t smem = (size_t)NW * WARP_SMEM * sizeof(double);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_jacobi_t<ElemDF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr_set = true;
  }
  launch_cluster(k_jacobi_t<ElemDF>, n_chains, cluster, smem, s, M, PsiT, lam, dp, d, rule, tol, max_sweeps,
                 status, sweeps_out, sweeps_acc, w.V, w.D, w.slots, w.flags, w.tiles,
                 reinterpret_cast<float2*>(pair_scratch_M), reinterpret_cast<float2*>(pair_scratch_P), w.crit,
                 sched, pre);
}

void mgs_rows_f64(cudaStream_t s, double* PsiT, int dp, int d, int n_chains, const int* eig_count,
                  int every, int cluster) {
  if (every <= 0) return;
  launch_cluster(k_mgs, n_chains, cluster, 0, s, PsiT, dp, d, eig_count, every);
}

}  // namespace rmhmc

// ------------------------------------------------------------------ C ABI: allocation-free eigen
extern "C" rmhmc_status rmhmc_eigh_noalloc(void* cuda_stream, int n, int d, const double* A_dev,
                                           double* lam_dev, double* Q_dev, double tol, int max_sweeps,
                                           int* sweeps_dev, int* status_dev) {
  using namespace rmhmc;
  if (n < 1 || d < 1 || !A_dev || (!lam_dev && !Q_dev) || !(tol > 0.0) || max_sweeps < 0)
    return RMHMC_EINVAL;
  const int dp = ((d + kJacSB - 1) / kJacSB) * kJacSB;
  if (noalloc_doubles(n, dp) > kNoAllocDoubles) return RMHMC_ESCRATCH;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RMHMC_ECUDA;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // the workspace looked up below is the current device's: a stream of another device is refused
  if (s) {
    int sdev = -1;
    if (cudaStreamGetDevice(s, &sdev) != cudaSuccess) return RMHMC_EINVAL;
    if (sdev != dev) return RMHMC_EINVAL;
  }
  double* base = g_noalloc_ptr[dev].load(std::memory_order_acquire);
  if (!base) {
    // host code cannot use the symbol itself as a device address: look it up once per device
    // (under a lock, so two host threads making their first call together agree)
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    base = g_noalloc_ptr[dev].load(std::memory_order_relaxed);
    if (!base) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return RMHMC_ECUDA;
      base = (double*)p;
      g_noalloc_ptr[dev].store(base, std::memory_order_release);
    }
  }
  const int np = dp / BL / 2;
  double* M = base;
  double* P = M + (size_t)n * dp * dp;
  double* lamp = P + (size_t)n * dp * dp;
  double* V = lamp + (size_t)n * dp;
  double* D = V + (size_t)n * np * SB * SB;
  double* slots = D + (size_t)n * np * SB * SB;
  int* status = (int*)(slots + (size_t)n * 64);
  int* sweeps = status + n;
  int* flags = sweeps + n;
  const long long tot = (long long)n * dp * dp;
  k_noalloc_pack<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(A_dev, d, dp, n, M, P, status);
  const int C = jacobi_cluster_size(n);
  const size_t smem = (size_t)NW * WARP_SMEM * sizeof(double);
  if (cudaFuncSetAttribute(k_jacobi_t<ElemF64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return RMHMC_ECUDA;
  if (launch_cluster(k_jacobi_t<ElemF64>, n, C, smem, s, M, P, lamp, dp, d, (int)RMHMC_JACOBI_RELATIVE, tol,
                     max_sweeps, status,
                     sweeps_dev ? sweeps_dev : sweeps, (int*)nullptr, V, D, slots, flags,
                     (unsigned long long*)nullptr, (double*)nullptr, (double*)nullptr, (float*)nullptr,
                     (int)RMHMC_JACOBI_CYCLIC, (const int*)nullptr) != cudaSuccess)
    return RMHMC_ECUDA;
  const long long out = (long long)n * d * d;
  k_noalloc_unpack<<<(unsigned)((out + 255) / 256), 256, 0, s>>>(lamp, P, d, dp, n, lam_dev, Q_dev);
  if (status_dev && cudaMemcpyAsync(status_dev, status, n * sizeof(int), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return RMHMC_ECUDA;
  return cudaGetLastError() == cudaSuccess ? RMHMC_OK : RMHMC_ECUDA;
}
