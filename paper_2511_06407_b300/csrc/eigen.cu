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

__device__ __forceinline__ void load_v(double* dst, const double* src) {
  const int lane = threadIdx.x & 31;
  for (int e = lane; e < SB * SB; e += 32) dst[(e / SB) * SBP + e % SB] = __ldcg(src + e);
}

__global__ void __launch_bounds__(NW * 32) k_jacobi(double* __restrict__ Mb, double* __restrict__ Pb,
                                                   double* __restrict__ lamb, int dp, int d, int rule,
                                                   double tol,
                                                   int max_sweeps, int* __restrict__ status,
                                                   int* __restrict__ sweeps_out,
                                                   int* __restrict__ sweeps_acc,
                                                   double* __restrict__ Vb, double* __restrict__ Db,
                                                   double* __restrict__ slotsb,
                                                   int* __restrict__ flagsb,
                                                   unsigned long long* __restrict__ tiles) {
  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int chain = blockIdx.x / C;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nb = dp / BL, np = nb / 2;
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
  double* M = Mb + (long long)chain * dp * dp;
  double* P = Pb + (long long)chain * dp * dp;
  double* V = Vb + (long long)chain * np * SB * SB;
  double* D = Db + (long long)chain * np * SB * SB;
  double* slots = slotsb + (long long)chain * 64;
  int* flags = flagsb + (long long)chain * np;
  extern __shared__ double smem[];
  double* ws = smem + warp * WARP_SMEM;
  double* X = ws;
  double* Tt = ws + SB * SBP;
  double* Va = ws + 2 * SB * SBP;
  double* Vq = ws + 3 * SB * SBP;
  __shared__ double red[2][NW];
  __shared__ double cs[NW][3 * SB / 2];  // (c, s, t) of the 8 rotations of a round, per warp
  __shared__ unsigned char sflag[kMaxPairs];  // pair rotated in this round
  __shared__ short sact[kMaxPairs];           // the rotated pairs, in order
  __shared__ int scum[kMaxPairs];             // cumulative active M tiles per column
  __shared__ int snact;

  const int gw = rank * NW + warp, nwt = C * NW;
  const int nct = dp / SB;
  int sweeps = 0;
  bool converged = false;
  double tot0 = 0.0;        // ||M||_F^2 from the first pass
  unsigned int ntile = 0;   // 16 x 16 x 16 tile products this warp executed (phase 2)
  unsigned int nround = 0;  // rounds of 8 rotations this warp applied to a 16 x 16 block (phase 1)
  for (;;) {
    // ---- convergence test. Pass 1: ||M||_F^2 and min_i<d |m_ii|. Pass 2: the worst pair ratio
    //      (pair_ratio) under the chosen rule, with floor = 4 u ||M||_F (rounding level).
    // ||M||_F is invariant under the rotations: summed over M in the first pass only; later
    // passes read the diagonal (a non-finite diagonal entry still poisons tot)
    double tot = 0.0, dmin = 1e308;
    if (sweeps == 0) {
      for (long long e = (long long)rank * blockDim.x + tid; e < (long long)dp * dp;
           e += (long long)C * blockDim.x) {
        const double v = __ldcg(M + e);
        tot = fma(v, v, tot);
        const int i = (int)(e / dp);
        if (i < d && (long long)i * dp + i == e) dmin = fmin(dmin, fabs(v));
      }
    } else {
      for (int i = rank * blockDim.x + tid; i < d; i += C * blockDim.x) {
        const double v = __ldcg(M + (long long)i * dp + i);
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
      __stcg(slots + (sweeps & 1) * 32 + 2 * rank, a);
      __stcg(slots + (sweeps & 1) * 32 + 2 * rank + 1, b);
    }
    cluster.sync();
    tot = 0.0;
    dmin = 1e308;
    for (int r = 0; r < C; ++r) {
      tot += __ldcg(slots + (sweeps & 1) * 32 + 2 * r);
      dmin = fmin(dmin, __ldcg(slots + (sweeps & 1) * 32 + 2 * r + 1));
    }
    if (sweeps == 0) tot0 = tot;
    else if (isfinite(tot)) tot = tot0;
    const double dmin2 = fmax(dmin * dmin, 1e-300);
    const double floor2 = fmax(16.0 * 1.2325951644078310e-32 * tot, 1e-300);  // (4u)^2 ||M||_F^2
    double crit = 0.0, bad = isfinite(tot) ? 0.0 : 1.0;
    for (long long e = (long long)rank * blockDim.x + tid; e < (long long)dp * dp;
         e += (long long)C * blockDim.x) {
      const int j = (int)(e / dp), l = (int)(e % dp);
      if (j >= l) continue;  // M is kept symmetric: the upper triangle decides
      const double v = __ldcg(M + e);
      if (v == 0.0) continue;
      if (!isfinite(v)) bad = 1.0;
      const double djj = __ldcg(M + (long long)j * dp + j), dll = __ldcg(M + (long long)l * dp + l);
      if (pair_unconverged(v, djj, dll, tol * tol, stop_floor2(djj, dll, floor2, rule), rule, dmin2))
        crit = 1.0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      crit = fmax(crit, __shfl_xor_sync(0xffffffffu, crit, o));
      bad = fmax(bad, __shfl_xor_sync(0xffffffffu, bad, o));
    }
    __syncthreads();
    if (lane == 0) { red[0][warp] = crit; red[1][warp] = bad; }
    __syncthreads();
    if (tid == 0) {
      double a = 0.0, b = 0.0;
      for (int w = 0; w < NW; ++w) { a = fmax(a, red[0][w]); b = fmax(b, red[1][w]); }
      __stcg(slots + (sweeps & 1) * 32 + 16 + 2 * rank, a);
      __stcg(slots + (sweeps & 1) * 32 + 16 + 2 * rank + 1, b);
    }
    cluster.sync();
    crit = 0.0;
    bad = 0.0;
    for (int r = 0; r < C; ++r) {
      crit = fmax(crit, __ldcg(slots + (sweeps & 1) * 32 + 16 + 2 * r));
      bad = fmax(bad, __ldcg(slots + (sweeps & 1) * 32 + 16 + 2 * r + 1));
    }
    if (bad != 0.0) break;
    if (crit == 0.0) { converged = true; break; }
    if (sweeps >= max_sweeps) break;
    const double itol2 = 1e-4 * tol * tol;  // inner problems are solved 100x tighter

    for (int r = 0; r < nb - 1; ++r) {
      // ---- phase 1: exact 16 x 16 solves, one warp per block pair
      for (int p = gw; p < np; p += nwt) {
        int I, J;
        circle_pair(r, p, nb, I, J);
        for (int e = lane; e < SB * SB; e += 32) {
          const int a = e / SB, b = e % SB;
          X[a * SBP + b] = __ldcg(M + (long long)gidx(I, J, a) * dp + gidx(I, J, b));
        }
        __syncwarp();
        const bool rot = inner_solve(X, Va, cs[warp], itol2, floor2, rule, dmin2, nround);
        if (rot) {
          for (int e = lane; e < SB * SB; e += 32) {
            const int a = e / SB, b = e % SB;
            __stcg(V + (long long)p * SB * SB + e, Va[a * SBP + b]);
            __stcg(D + (long long)p * SB * SB + e, X[a * SBP + b]);
          }
        }
        if (lane == 0) __stcg(flags + p, rot ? 1 : 0);
        __syncwarp();
      }
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
      // ---- phase 2: apply all rotations to M (P <= Q tiles) and to the rows of Psi^T
      //      over the active jobs only, dealt round-robin to the cluster's warps: the M tiles
      //      (P <= Q) of which P or Q rotated, then the Psi^T row tiles of the rotated pairs
      const int k = scum[np - 1];  // active M tiles
      for (int i = gw; i < k; i += nwt) {
        {
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
          int I1, J1, I2, J2;
          circle_pair(r, Pp, nb, I1, J1);
          circle_pair(r, Q, nb, I2, J2);
          if (Pp == Q) {
            for (int e = lane; e < SB * SB; e += 32) {
              const int a = e / SB, b = e % SB;
              __stcg(M + (long long)gidx(I1, J1, a) * dp + gidx(I1, J1, b), __ldcg(D + (long long)Pp * SB * SB + e));
            }
          } else {
            for (int e = lane; e < SB * SB; e += 32) {
              const int a = e / SB, b = e % SB;
              X[a * SBP + b] = __ldcg(M + (long long)gidx(I1, J1, a) * dp + gidx(I2, J2, b));
            }
            if (fP) load_v(Va, V + (long long)Pp * SB * SB);
            if (fQ) load_v(Vq, V + (long long)Q * SB * SB);
            __syncwarp();
            tile_transform(X, fP ? Va : nullptr, fQ ? Vq : nullptr, Tt, X);
            ntile += (fP ? 1u : 0u) + (fQ ? 1u : 0u);
            const int t = lane >> 1, u0 = (lane & 1) * 8;
#pragma unroll
            for (int j = 0; j < 8; ++j)
              __stcg(M + (long long)gidx(I1, J1, t) * dp + gidx(I2, J2, u0 + j), X[t * SBP + u0 + j]);
#pragma unroll
            for (int j = 0; j < 8; ++j)
              __stcg(M + (long long)gidx(I2, J2, t) * dp + gidx(I1, J1, u0 + j), X[(u0 + j) * SBP + t]);
          }
          __syncwarp();
        }
      }
      const int nPsi = snact * nct;
      for (int j = ((gw - k) % nwt + nwt) % nwt; j < nPsi; j += nwt) {
        const int Pp = sact[j / nct], ct = j % nct;
        int I1, J1;
        circle_pair(r, Pp, nb, I1, J1);
        for (int e = lane; e < SB * SB; e += 32) {
          const int a = e / SB, b = e % SB;
          X[a * SBP + b] = __ldcg(P + (long long)gidx(I1, J1, a) * dp + ct * SB + b);
        }
        load_v(Va, V + (long long)Pp * SB * SB);
        __syncwarp();
        tile_transform(X, Va, nullptr, Tt, X);
        ++ntile;
        const int t = lane >> 1, u0 = (lane & 1) * 8;
#pragma unroll
        for (int j2 = 0; j2 < 8; ++j2)
          __stcg(P + (long long)gidx(I1, J1, t) * dp + ct * SB + u0 + j2, X[t * SBP + u0 + j2]);
        __syncwarp();
      }
      cluster.sync();
    }
    ++sweeps;
  }
  for (int i = rank * blockDim.x + tid; i < dp; i += C * blockDim.x)
    lamb[(long long)chain * dp + i] = __ldcg(M + (long long)i * dp + i);
  if (tiles && lane == 0) {
    if (ntile) atomicAdd(tiles + 2 * chain, (unsigned long long)ntile);
    if (nround) atomicAdd(tiles + 2 * chain + 1, (unsigned long long)nround);
  }
  if (rank == 0 && tid == 0) {
    sweeps_out[chain] = sweeps;
    if (sweeps_acc) sweeps_acc[chain] += sweeps;
    if (!converged) atomicOr(&status[chain], RMHMC_CHAIN_NOTCONV);
  }
}

// ------------------------------------------------------------------ double-float variant
// Mixed precision: the rotations of phase 2 are applied in double-float arithmetic (df.cuh). M and
// Psi^T are held as FP32 pairs in scratch for the whole kernel; the 16 x 16 inner solves (phase 1),
// the stopping test and the conversions stay in FP64.
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

__device__ __forceinline__ float2 ldcg2(const float2* p) { return __ldcg(p); }

__device__ __forceinline__ void load_v_df(float2* dst, const float2* src) {
  const int lane = threadIdx.x & 31;
  for (int e = lane; e < SB * SB; e += 32) dst[(e / SB) * SBP + e % SB] = ldcg2(src + e);
}

// Same algorithm and stopping rule as k_jacobi (the rounding floor uses the double-float unit
// 2^-48); M and Psi^T (double, dp x dp per chain) are converted into the pair buffers Mw, Pw
// (float2, same layout) at entry and back at exit.
__global__ void __launch_bounds__(NW * 32) k_jacobi_df(double* __restrict__ Mb, double* __restrict__ Pb,
                                                      double* __restrict__ lamb, int dp, int d, int rule,
                                                      double tol, int max_sweeps,
                                                      int* __restrict__ status,
                                                      int* __restrict__ sweeps_out,
                                                      int* __restrict__ sweeps_acc,
                                                      double* __restrict__ Vb, double* __restrict__ Db,
                                                      double* __restrict__ slotsb,
                                                      int* __restrict__ flagsb,
                                                      unsigned long long* __restrict__ tiles,
                                                      float2* __restrict__ Mwb, float2* __restrict__ Pwb) {
  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int chain = blockIdx.x / C;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nb = dp / BL, np = nb / 2;
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
  float2* Mw = Mwb + (long long)chain * DD;
  float2* Pw = Pwb + (long long)chain * DD;
  float2* V = (float2*)(Vb + (long long)chain * np * SB * SB);
  float2* D = (float2*)(Db + (long long)chain * np * SB * SB);
  double* slots = slotsb + (long long)chain * 64;
  int* flags = flagsb + (long long)chain * np;
  extern __shared__ double smem[];
  double* ws = smem + warp * WARP_SMEM;
  double* Xd = ws;                    // phase 1 (FP64)
  double* Vd = ws + 2 * SB * SBP;
  float2* X = (float2*)ws;            // phase 2 (pairs), same bytes
  float2* Tt = (float2*)(ws + SB * SBP);
  float2* Va = (float2*)(ws + 2 * SB * SBP);
  float2* Vq = (float2*)(ws + 3 * SB * SBP);
  __shared__ double red[2][NW];
  __shared__ double cs[NW][3 * SB / 2];  // (c, s, t) of the 8 rotations of a round, per warp
  __shared__ unsigned char sflag[kMaxPairs];  // pair rotated in this round
  __shared__ short sact[kMaxPairs];           // the rotated pairs, in order
  __shared__ int scum[kMaxPairs];             // cumulative active M tiles per column
  __shared__ int snact;

  for (long long e = (long long)rank * blockDim.x + tid; e < DD; e += (long long)C * blockDim.x) {
    __stcg(Mw + e, df_split(__ldcg(M + e)));
    __stcg(Pw + e, df_split(__ldcg(P + e)));
  }
  cluster.sync();

  const int gw = rank * NW + warp, nwt = C * NW;
  const int nct = dp / SB;
  int sweeps = 0;
  bool converged = false;
  double tot0 = 0.0;        // ||M||_F^2 from the first pass
  unsigned int ntile = 0;   // 16 x 16 x 16 tile products this warp executed (phase 2)
  unsigned int nround = 0;  // rounds of 8 rotations this warp applied to a 16 x 16 block (phase 1)
  for (;;) {
    double tot = 0.0, dmin = 1e308;
    if (sweeps == 0) {
      for (long long e = (long long)rank * blockDim.x + tid; e < DD; e += (long long)C * blockDim.x) {
        const double v = df_join(ldcg2(Mw + e));
        tot = fma(v, v, tot);
        const int i = (int)(e / dp);
        if (i < d && (long long)i * dp + i == e) dmin = fmin(dmin, fabs(v));
      }
    } else {  // ||M||_F is invariant under the rotations (see k_jacobi)
      for (int i = rank * blockDim.x + tid; i < d; i += C * blockDim.x) {
        const double v = df_join(ldcg2(Mw + (long long)i * dp + i));
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
      __stcg(slots + (sweeps & 1) * 32 + 2 * rank, a);
      __stcg(slots + (sweeps & 1) * 32 + 2 * rank + 1, b);
    }
    cluster.sync();
    tot = 0.0;
    dmin = 1e308;
    for (int r = 0; r < C; ++r) {
      tot += __ldcg(slots + (sweeps & 1) * 32 + 2 * r);
      dmin = fmin(dmin, __ldcg(slots + (sweeps & 1) * 32 + 2 * r + 1));
    }
    if (sweeps == 0) tot0 = tot;
    else if (isfinite(tot)) tot = tot0;
    const double dmin2 = fmax(dmin * dmin, 1e-300);
    const double floor2 = fmax(16.0 * 1.2621774483536189e-29 * tot, 1e-300);  // (4 * 2^-48)^2 ||M||^2
    double crit = 0.0, bad = isfinite(tot) ? 0.0 : 1.0;
    for (long long e = (long long)rank * blockDim.x + tid; e < DD; e += (long long)C * blockDim.x) {
      const int j = (int)(e / dp), l = (int)(e % dp);
      if (j >= l) continue;  // M is kept symmetric: the upper triangle decides
      const double v = df_join(ldcg2(Mw + e));
      if (v == 0.0) continue;
      if (!isfinite(v)) bad = 1.0;
      const double djj = df_join(ldcg2(Mw + (long long)j * dp + j)), dll = df_join(ldcg2(Mw + (long long)l * dp + l));
      if (pair_unconverged(v, djj, dll, tol * tol, stop_floor2(djj, dll, floor2, rule), rule, dmin2))
        crit = 1.0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      crit = fmax(crit, __shfl_xor_sync(0xffffffffu, crit, o));
      bad = fmax(bad, __shfl_xor_sync(0xffffffffu, bad, o));
    }
    __syncthreads();
    if (lane == 0) { red[0][warp] = crit; red[1][warp] = bad; }
    __syncthreads();
    if (tid == 0) {
      double a = 0.0, b = 0.0;
      for (int w = 0; w < NW; ++w) { a = fmax(a, red[0][w]); b = fmax(b, red[1][w]); }
      __stcg(slots + (sweeps & 1) * 32 + 16 + 2 * rank, a);
      __stcg(slots + (sweeps & 1) * 32 + 16 + 2 * rank + 1, b);
    }
    cluster.sync();
    crit = 0.0;
    bad = 0.0;
    for (int r = 0; r < C; ++r) {
      crit = fmax(crit, __ldcg(slots + (sweeps & 1) * 32 + 16 + 2 * r));
      bad = fmax(bad, __ldcg(slots + (sweeps & 1) * 32 + 16 + 2 * r + 1));
    }
    if (bad != 0.0) break;
    if (crit == 0.0) { converged = true; break; }
    if (sweeps >= max_sweeps) break;
    const double itol2 = 1e-4 * tol * tol;

    for (int r = 0; r < nb - 1; ++r) {
      // ---- phase 1 (FP64): exact 16 x 16 solves, one warp per block pair
      for (int p = gw; p < np; p += nwt) {
        int I, J;
        circle_pair(r, p, nb, I, J);
        for (int e = lane; e < SB * SB; e += 32) {
          const int a = e / SB, b = e % SB;
          Xd[a * SBP + b] = df_join(ldcg2(Mw + (long long)gidx(I, J, a) * dp + gidx(I, J, b)));
        }
        __syncwarp();
        const bool rot = inner_solve(Xd, Vd, cs[warp], itol2, floor2, rule, dmin2, nround);
        if (rot) {
          for (int e = lane; e < SB * SB; e += 32) {
            const int a = e / SB, b = e % SB;
            __stcg(V + (long long)p * SB * SB + e, df_split(Vd[a * SBP + b]));
            __stcg(D + (long long)p * SB * SB + e, df_split(Xd[a * SBP + b]));
          }
        }
        if (lane == 0) __stcg(flags + p, rot ? 1 : 0);
        __syncwarp();
      }
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
      // ---- phase 2 (double-float): apply all rotations to M and to the rows of Psi^T
      //      over the active jobs only, dealt round-robin to the cluster's warps: the M tiles
      //      (P <= Q) of which P or Q rotated, then the Psi^T row tiles of the rotated pairs
      const int k = scum[np - 1];  // active M tiles
      for (int i = gw; i < k; i += nwt) {
        {
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
          int I1, J1, I2, J2;
          circle_pair(r, Pp, nb, I1, J1);
          circle_pair(r, Q, nb, I2, J2);
          if (Pp == Q) {
            for (int e = lane; e < SB * SB; e += 32) {
              const int a = e / SB, b = e % SB;
              __stcg(Mw + (long long)gidx(I1, J1, a) * dp + gidx(I1, J1, b), ldcg2(D + (long long)Pp * SB * SB + e));
            }
          } else {
            for (int e = lane; e < SB * SB; e += 32) {
              const int a = e / SB, b = e % SB;
              X[a * SBP + b] = ldcg2(Mw + (long long)gidx(I1, J1, a) * dp + gidx(I2, J2, b));
            }
            if (fP) load_v_df(Va, V + (long long)Pp * SB * SB);
            if (fQ) load_v_df(Vq, V + (long long)Q * SB * SB);
            __syncwarp();
            tile_transform_df(X, fP ? Va : nullptr, fQ ? Vq : nullptr, Tt, X);
            ntile += (fP ? 1u : 0u) + (fQ ? 1u : 0u);
            const int t = lane >> 1, u0 = (lane & 1) * 8;
#pragma unroll
            for (int j = 0; j < 8; ++j)
              __stcg(Mw + (long long)gidx(I1, J1, t) * dp + gidx(I2, J2, u0 + j), X[t * SBP + u0 + j]);
#pragma unroll
            for (int j = 0; j < 8; ++j)
              __stcg(Mw + (long long)gidx(I2, J2, t) * dp + gidx(I1, J1, u0 + j), X[(u0 + j) * SBP + t]);
          }
          __syncwarp();
        }
      }
      const int nPsi = snact * nct;
      for (int j = ((gw - k) % nwt + nwt) % nwt; j < nPsi; j += nwt) {
        const int Pp = sact[j / nct], ct = j % nct;
        int I1, J1;
        circle_pair(r, Pp, nb, I1, J1);
        for (int e = lane; e < SB * SB; e += 32) {
          const int a = e / SB, b = e % SB;
          X[a * SBP + b] = ldcg2(Pw + (long long)gidx(I1, J1, a) * dp + ct * SB + b);
        }
        load_v_df(Va, V + (long long)Pp * SB * SB);
        __syncwarp();
        tile_transform_df(X, Va, nullptr, Tt, X);
        ++ntile;
        const int t = lane >> 1, u0 = (lane & 1) * 8;
#pragma unroll
        for (int j2 = 0; j2 < 8; ++j2)
          __stcg(Pw + (long long)gidx(I1, J1, t) * dp + ct * SB + u0 + j2, X[t * SBP + u0 + j2]);
        __syncwarp();
      }
      cluster.sync();
    }
    ++sweeps;
  }
  for (long long e = (long long)rank * blockDim.x + tid; e < DD; e += (long long)C * blockDim.x) {
    __stcg(M + e, df_join(ldcg2(Mw + e)));
    __stcg(P + e, df_join(ldcg2(Pw + e)));
  }
  for (int i = rank * blockDim.x + tid; i < dp; i += C * blockDim.x)
    lamb[(long long)chain * dp + i] = df_join(ldcg2(Mw + (long long)i * dp + i));
  if (tiles && lane == 0) {
    if (ntile) atomicAdd(tiles + 2 * chain, (unsigned long long)ntile);
    if (nround) atomicAdd(tiles + 2 * chain + 1, (unsigned long long)nround);
  }
  if (rank == 0 && tid == 0) {
    sweeps_out[chain] = sweeps;
    if (sweeps_acc) sweeps_acc[chain] += sweeps;
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
double* g_noalloc_ptr[kMaxDevices] = {};

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
                JacobiWork w, int cluster) {
  const size_t smem = (size_t)NW * WARP_SMEM * sizeof(double);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr_set = true;
  }
  launch_cluster(k_jacobi, n_chains, cluster, smem, s, M, PsiT, lam, dp, d, rule, tol, max_sweeps,
                 status, sweeps_out, sweeps_acc, w.V, w.D, w.slots, w.flags, w.tiles);
}

void jacobi_df(cudaStream_t s, double* M, double* PsiT, double* lam, int dp, int d, int n_chains,
               int rule, double tol, int max_sweeps, int* status, int* sweeps_out, int* sweeps_acc,
               JacobiWork w, int cluster, double* pair_scratch_M, double* pair_scratch_P) {
  const size_t smem = (size_t)NW * WARP_SMEM * sizeof(double);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_jacobi_df, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr_set = true;
  }
  launch_cluster(k_jacobi_df, n_chains, cluster, smem, s, M, PsiT, lam, dp, d, rule, tol, max_sweeps,
                 status, sweeps_out, sweeps_acc, w.V, w.D, w.slots, w.flags, w.tiles,
                 (float2*)pair_scratch_M,
                 (float2*)pair_scratch_P);
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
  if (!g_noalloc_ptr[dev]) {
    // host code cannot use the symbol itself as a device address: look it up once per device
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return RMHMC_ECUDA;
    g_noalloc_ptr[dev] = (double*)p;
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int np = dp / BL / 2;
  double* base = g_noalloc_ptr[dev];
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
  if (cudaFuncSetAttribute(k_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return RMHMC_ECUDA;
  if (launch_cluster(k_jacobi, n, C, smem, s, M, P, lamp, dp, d, (int)RMHMC_JACOBI_RELATIVE, tol,
                     max_sweeps, status,
                     sweeps_dev ? sweeps_dev : sweeps, (int*)nullptr, V, D, slots, flags,
                     (unsigned long long*)nullptr) != cudaSuccess)
    return RMHMC_ECUDA;
  const long long out = (long long)n * d * d;
  k_noalloc_unpack<<<(unsigned)((out + 255) / 256), 256, 0, s>>>(lamp, P, d, dp, n, lam_dev, Q_dev);
  if (status_dev && cudaMemcpyAsync(status_dev, status, n * sizeof(int), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return RMHMC_ECUDA;
  return cudaGetLastError() == cudaSuccess ? RMHMC_OK : RMHMC_ECUDA;
}
