// FP64-accurate batched GEMM on the fifth-generation tensor cores (tcgen05.mma kind::f16, bf16
// operands, FP32 accumulators in tensor memory), by error-free splitting (Ozaki, Ogita, Oishi and
// Rump, "Error-free transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59, 2012).
//
// Splitting. Row r of op(A) (and column j of op(B)) gets the exponent e with max |x| < 2^e. Each
// element becomes the integer N = rint(x 2^(7S - e)) and N is written in balanced base 128 with S
// digits, N = sum_t d_t 128^(S - t), |d_1| <= 128, |d_t| <= 64 (t > 1). Slice t stores
// D_t = d_t 2^(-7(t-1)) in bf16, which is exact (|d_t| <= 256 needs 8 significand bits). Then
// x = 2^(e-7) sum_t D_t up to 2^(e-7S-1), and
//   (op(A) op(B))_ij = 2^(eA_i + eB_j - 14) sum_{t,u} sum_l D_t(A)_il D_u(B)_lj.
// Pairs with t + u <= S + 1 are computed (S (S + 1) / 2 MMA products per K step); the rest lie
// below 2^-7S of the leading term.
// Exact accumulation. All products of one group g = t + u are integer multiples of 2^(-7(g-2)),
// and |sum over the group| <= 2^15 k of those units for g <= 7, so with k <= 512 per launch every
// group g <= 7 sums exactly in an FP32 accumulator (< 2^24 units; group 8 is within one rounding of
// that). Groups 2..8 get one accumulator each; groups >= 9 share one, whose rounding sits ~2^-48
// below the leading term per product. The epilogue adds the accumulators in FP64 (smallest first)
// and scales by the exponents.
//
// Kernel layout (one CTA per 128 x 64 output tile, 320 threads):
//   warp 0   one thread streams the S slices of A (128 rows) and of B (64 rows) for each K step of
//            16 from global memory into a 4-stage shared-memory ring with cp.async.bulk, completion
//            counted on an mbarrier per stage;
//   warp 1   allocates 512 tensor-memory columns; one thread issues the tcgen05.mma of each K step
//            (the S (S + 1) / 2 slice products, up to four per instruction, N <= 256) into the 8
//            accumulators (8 x 64 columns) and releases each stage with tcgen05.commit;
//   warps 2-9 wait for the final commit, read the accumulators with tcgen05.ld (warp w reads lanes
//            32 (w % 4) .., half the columns each), combine them exactly in integers and write
//            alpha C~ + beta C in FP64 through a shared-memory staging tile (coalesced stores).
// The slices are stored in the core-matrix order of the MMA's no-swizzle K-major operand layout
// (8 rows x 16 bytes per core matrix), so each stage is a set of contiguous block copies.
// Every mbarrier wait is bounded (about 2 s of global time): a wait that runs out sets
// RMHMC_CHAIN_TIMEOUT for the batch entry, the CTA still waits (bounded) for its own copies and
// MMAs, writes NaN and frees its tensor memory.
#include <math.h>
#include <stdint.h>

#include "internal.cuh"

namespace rmhmc {

namespace {

constexpr int TC_M = 128;             // output tile rows = MMA M (one TMEM lane per row)
constexpr int TC_N = 64;              // rows of a B-operand tile in the split layout (output columns)
constexpr int TC_K = 16;              // K of one bf16 MMA
constexpr int TC_NACC = 8;            // accumulators: groups 2..8, then one for groups >= 9
// A launch computes output tiles of 128 x NT, NT = 64 (one B-operand tile) or 32 (half of one: the
// finer grid of the tile-width choice); the accumulators take TC_NACC * NT tensor-memory columns.
constexpr int TC_THREADS = 320;        // warp 0 loads, warp 1 issues MMAs, warps 2..9 epilogue
constexpr int TC_KSTEPS_MAX = 32;     // K steps per launch (k <= 512: exact group sums)
constexpr int kExpBad = 0x7fffffff;   // exponent marker of a row holding a non-finite value
constexpr unsigned long long kWaitNs = 2000000000ull;

constexpr int A_SLICE = TC_M * TC_K * 2;  // bytes of one slice of an A stage (4096)
constexpr int B_SLICE = TC_N * TC_K * 2;  // (2048), of which a 32-row half is 1024 contiguous bytes

// NT = 64: one CTA per SM (all 512 tensor-memory columns, a 4-stage ring). NT = 32: two CTAs per SM
// (256 columns each, a ring of at most 3 stages that fits twice in shared memory, an epilogue in
// 8-column chunks to stay within half the register file), so that one CTA's epilogue overlaps the
// other's MMAs.
template <int S, int NT>
struct TcCfg {
  static constexpr int BS = NT * TC_K * 2;  // bytes of one B slice in a stage
  static constexpr int COLS = TC_NACC * NT;  // tensor-memory columns (a power of two >= 32)
  static constexpr int CTAS = NT == 32 ? 2 : 1;  // CTAs per SM
  static constexpr int CW = NT == 32 ? 8 : 16;   // epilogue chunk width (columns)
  static constexpr int STAGE = S * (A_SLICE + BS);
  static constexpr int NST_FIT = (CTAS == 2 ? 111 * 1024 : 226 * 1024) / STAGE;
  static constexpr int NST_MAX = CTAS == 2 ? 3 : 4;
  static constexpr int NST = NST_FIT > NST_MAX ? NST_MAX : NST_FIT;
  static constexpr int BAR_OFF = NST * STAGE;
  static constexpr int SMEM = BAR_OFF + 256;
  static constexpr int NA = S < TC_NACC ? S : TC_NACC;  // accumulators in use
  static_assert(NST >= 2, "at least two pipeline stages");
  static_assert(NT == 64 || NT == 32, "output tile width");
  static_assert(SMEM <= 227 * 1024, "shared memory");
};

// instruction descriptor of tcgen05.mma kind::f16 for an N-column product: FP32 accumulate
// (bits 4-5 = 1), A and B bf16 (bits 7-9 and 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at
// bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t idesc_bf16(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(TC_M >> 4) << 24);
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase of `parity` to complete; false after about limit_ns of global time.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity,
                                          unsigned long long limit_ns = kWaitNs) {
  if (mbar_test(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (true) {
    if (mbar_test(bar, parity)) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes,
                                          uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// shared-memory matrix descriptor, no swizzle, K-major: core matrices of 8 rows x 16 bytes; the
// next core matrix along K is 128 bytes on (leading byte offset), the next 8-row group 256 bytes on
// (stride byte offset); version 1 at bit 46
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)(128 >> 4) << 16) |
         ((uint64_t)(256 >> 4) << 32) | (1ull << 46);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                       uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}

template <int W>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, float (&v)[W]) {
  if constexpr (W == 16) tmem_ld16(taddr, v);
  else tmem_ld8(taddr, v);
}

// ---------------------------------------------------------------- splitting

// e with |x| < 2^e for the largest |x| of a row, from a = the bits of that |x| (the order of
// non-negative doubles is the order of their bit patterns); integer unit only
__device__ __forceinline__ int exponent_of_bits(unsigned long long a) {
  if (a == 0) return 0;
  const int E = (int)(a >> 52);
  if (E == 0) return (63 - __clzll(a)) - 1073;  // subnormal: a 2^-1074
  return E - 1022;                               // 1.f 2^(E-1023) = 0.1f 2^(E-1022)
}

__device__ __forceinline__ void scan_abs(double v, unsigned long long& mx, bool& bad) {
  const unsigned long long a = (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
  if ((a >> 52) == 0x7FF) bad = true;
  else mx = a > mx ? a : mx;
}

// ex[b][r] = exponent of row r of the K-major view (kmaj: X[r * ld + l], else X[l * ld + r]);
// rows R..Rpad-1 get 0. kmaj: one warp per row; otherwise a block covers 32 columns, its 8 warps
// take every 8th l (coalesced 256-byte rows) and combine through shared memory.
__global__ void k_tc_exponents(const double* __restrict__ X, int ld, long long sX, int kmaj, int R,
                               int K, int Rpad, int* __restrict__ ex, const int* __restrict__ mask) {
  const int b = blockIdx.y;
  if (mask && !mask[b]) return;  // entry skipped (uniform per CTA)
  X += b * sX;
  ex += (long long)b * Rpad;
  const int lane = threadIdx.x % 32, wy = threadIdx.x / 32;
  if (kmaj) {
    const int r = blockIdx.x * 8 + wy;
    if (r >= Rpad) return;
    unsigned long long mx = 0;
    bool bad = false;
    if (r < R)
      for (int l = lane; l < K; l += 32) scan_abs(X[(long long)r * ld + l], mx, bad);
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const unsigned long long y = __shfl_xor_sync(0xffffffffu, mx, o);
      mx = y > mx ? y : mx;
    }
    bad = __any_sync(0xffffffffu, bad);
    if (lane == 0) ex[r] = bad ? kExpBad : exponent_of_bits(mx);
  } else {
    __shared__ unsigned long long smx[8][32];
    __shared__ int sbad[8][32];
    const int r = blockIdx.x * 32 + lane;
    unsigned long long mx = 0;
    bool bad = false;
    if (r < R)
      for (int l = wy; l < K; l += 8) scan_abs(X[(long long)l * ld + r], mx, bad);
    smx[wy][lane] = mx;
    sbad[wy][lane] = bad;
    __syncthreads();
    if (wy == 0 && r < Rpad) {
      for (int w = 1; w < 8; ++w) {
        mx = smx[w][lane] > mx ? smx[w][lane] : mx;
        bad = bad || sbad[w][lane];
      }
      ex[r] = bad ? kExpBad : exponent_of_bits(mx);
    }
  }
}

// rint(x 2^sh) as an integer, for |x 2^sh| < 2^63, from the bits of x (integer unit only; ties
// away from zero).
__device__ __forceinline__ long long scaled_integer(double x, int sh) {
  const long long bits = __double_as_longlong(x);
  const int E = (int)((bits >> 52) & 0x7FF);
  long long M = bits & ((1ll << 52) - 1);
  int e2;  // x = +-M 2^e2
  if (E == 0) {
    e2 = -1074;
  } else {
    M |= 1ll << 52;
    e2 = E - 1075;
  }
  const int t = e2 + sh;
  long long n;
  if (t >= 0) n = M << t;  // t <= 10 because the result is below 2^63
  else if (t > -63) n = (M + (1ll << (-t - 1))) >> -t;
  else n = 0;
  return bits < 0 ? -n : n;
}

// One thread per (row r, K step ks, half kc of the step): the 8 elements l = 16 ks + 8 kc + 0..7
// become S slices of 8 bf16 each (one 16-byte row of a core matrix). Per batch entry the slices are
// laid out [r / TR][ks][t][(r % TR) / 8][kc][r % 8][8 elements] for the operand's tile height TR
// (128 rows of A, 64 of B), so everything one pipeline stage of one tile needs (its TR rows, all S
// slices, one K step) is a single contiguous block of S TR 32 bytes.
template <int S>
__global__ void k_tc_split(const double* __restrict__ X, int ld, long long sX, int kmaj, int R,
                           int K, int R8, int KS, int TR8, const int* __restrict__ ex,
                           uint8_t* __restrict__ dig, long long sD, const int* __restrict__ mask) {
  const int b = blockIdx.y;
  if (mask && !mask[b]) return;
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (long long)KS * R8 * 16) return;
  const int ri = (int)(id & 7), kc = (int)((id >> 3) & 1);
  const long long rest = id >> 4;
  const int r8l = (int)(rest % TR8);
  const long long rest2 = rest / TR8;
  const int ks = (int)(rest2 % KS), rt = (int)(rest2 / KS);
  const int r = (rt * TR8 + r8l) * 8 + ri, l0 = ks * TC_K + kc * 8;
  X += b * sX;
  dig += b * sD;
  const int e = ex[(long long)b * R8 * 8 + r];
  const bool row_ok = r < R && e != kExpBad;
  uint32_t w[S][4];
#pragma unroll
  for (int h = 0; h < 8; ++h) {
    const int l = l0 + h;
    long long n = 0;
    if (row_ok && l < K) {
      const double x = kmaj ? X[(long long)r * ld + l] : X[(long long)l * ld + r];
      n = scaled_integer(x, 7 * S - e);  // |x 2^(7S - e)| < 2^(7S) <= 2^63
    }
    int d[S];
#pragma unroll
    for (int t = S - 1; t >= 1; --t) {
      const int dt = (int)(((n + 64) & 127) - 64);  // balanced digit in [-64, 63]
      d[t] = dt;
      n = (n - dt) >> 7;  // exact: n - dt is a multiple of 128
    }
    d[0] = (int)n;  // |d_1| <= 128
#pragma unroll
    for (int t = 0; t < S; ++t) {
      // D_t = d_t 2^(-7t) (0-based t): an exact float, whose upper 16 bits are its bf16 image
      const float f = (float)d[t] * __int_as_float((127 - 7 * t) << 23);
      const uint32_t hb = __float_as_uint(f) >> 16;
      if (h & 1) w[t][h >> 1] |= hb << 16;
      else w[t][h >> 1] = hb;
    }
  }
#pragma unroll
  for (int t = 0; t < S; ++t) {
    const long long off = (((((long long)rt * KS + ks) * S + t) * TR8 + r8l) * 2 + kc) * 128 + ri * 16;
    *reinterpret_cast<uint4*>(dig + off) = make_uint4(w[t][0], w[t][1], w[t][2], w[t][3]);
  }
}

// ---------------------------------------------------------------- the tensor-core GEMM

// v 2^E as a double for |v| < 2^53 (exact), assembled from bits when the result is normal.
__device__ __forceinline__ double int_to_double_pow2(long long v, int E) {
  if (v == 0) return 0.0;
  const unsigned long long a = v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
  const int p = 63 - __clzll(a);  // leading bit, <= 52
  const int be = p + E + 1023;
  if (be <= 0 || be >= 2047) return ldexp((double)v, E);
  const unsigned long long bits = ((unsigned long long)(v < 0) << 63) |
                                  ((unsigned long long)be << 52) |
                                  ((a << (52 - p)) & ((1ull << 52) - 1));
  return __longlong_as_double((long long)bits);
}

struct TcArgs {
  const uint8_t* A;  // slices of op(A), rows = output rows
  long long sA;      // bytes per batch entry
  int RA8;           // padded rows / 8
  const int* eA;     // exponents, eAs per batch entry (0: one entry shared by all)
  long long eAs;
  const uint8_t* B;  // slices of op(B)^T, rows = output columns
  long long sB;
  int RB8;
  const int* eB;
  long long eBs;
  int m, n, KS, ks0, ks1;  // K steps in the split operands, and those of this launch
  double alpha, beta;
  double* C;
  int ldc;
  long long sC;
  int sym;
  int* status;  // per-chain status (may be null); entry b reports to status[b / sdiv]
  int sdiv;
  const int* mask;  // null, or entry b runs only where mask[b] != 0
  unsigned long long wait_ns;  // limit of each bounded wait
  int stall_entry;             // test switch: entry whose loads are never issued (-1: none)
};

template <int S, int NT>
__global__ void __launch_bounds__(TC_THREADS, TcCfg<S, NT>::CTAS) k_gemm_tc(TcArgs a) {
  using Cfg = TcCfg<S, NT>;
  constexpr int NST = Cfg::NST;
  extern __shared__ __align__(1024) uint8_t smem[];
  const int tn = blockIdx.x, tm = blockIdx.y, b = blockIdx.z;
  const int m0 = tm * TC_M, n0 = tn * NT;
  if (a.sym && m0 + TC_M - 1 < n0) return;  // strictly above the diagonal: mirrored by others
  if (a.mask && !a.mask[b]) return;          // entry skipped (before any allocation)
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Cfg::BAR_OFF);
  const uint32_t full0 = smem_addr(bars), empty0 = smem_addr(bars + NST),
                 done = smem_addr(bars + 2 * NST);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * NST + 1);
  __shared__ int failed;
  if (threadIdx.x == 0) {
    failed = 0;
    for (int i = 0; i < NST; ++i) {
      mbar_init(full0 + 8 * i, 1);
      mbar_init(empty0 + 8 * i, 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(tmem_slot)),
                 "r"(Cfg::COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int nk = a.ks1 - a.ks0;

  if (warp == 0) {
    if (lane == 0) {
      const uint8_t* Ab = a.A + b * a.sA;
      const uint8_t* Bb = a.B + b * a.sB;
      int issued = 0;
      // the test switch: for this entry no copy is issued, so the MMA warp's first wait runs out
      // (nothing is in flight, the CTA then frees its tensor memory and returns)
      const int nk_issue = b == a.stall_entry ? 0 : nk;
      for (int it = 0; it < nk_issue; ++it) {
        const int st = it % NST;
        if (it >= NST && !mbar_wait(empty0 + 8 * st, ((it / NST) - 1) & 1, a.wait_ns)) {
          atomicExch(&failed, 1);
          break;
        }
        const uint32_t full = full0 + 8 * st;
        mbar_expect_tx(full, S * (A_SLICE + Cfg::BS));
        const uint32_t sa = smem_addr(smem + st * Cfg::STAGE), sb = sa + S * A_SLICE;
        const long long ks = a.ks0 + it;
        bulk_load(sa, Ab + ((long long)tm * a.KS + ks) * S * A_SLICE, S * A_SLICE, full);
        if (NT == TC_N) {
          bulk_load(sb, Bb + ((long long)tn * a.KS + ks) * S * B_SLICE, S * B_SLICE, full);
        } else {  // the 32-row half (tn % 2) of B tile tn / 2, slice by slice
          const uint8_t* src = Bb + ((long long)(tn >> 1) * a.KS + ks) * S * B_SLICE + (tn & 1) * Cfg::BS;
#pragma unroll
          for (int i = 0; i < S; ++i) bulk_load(sb + i * Cfg::BS, src + i * B_SLICE, Cfg::BS, full);
        }
        issued = it + 1;
      }
      // every issued copy has landed before the CTA may exit (already true unless a wait failed)
      for (int it = issued > NST ? issued - NST : 0; it < issued; ++it)
        if (!mbar_wait(full0 + 8 * (it % NST), (it / NST) & 1, a.wait_ns)) atomicExch(&failed, 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      for (int it = 0; it < nk; ++it) {
        const int st = it % NST;
        if (!mbar_wait(full0 + 8 * st, (it / NST) & 1, a.wait_ns)) {
          atomicExch(&failed, 1);
          break;
        }
        tc_fence_after();
        const uint32_t sa = smem_addr(smem + st * Cfg::STAGE), sb = sa + S * A_SLICE;
        // Accumulator g sits at TMEM column NT g and the B slices follow each other in shared
        // memory, so one MMA with N = NT c multiplies A_i by B_j .. B_(j+c-1) straight into the
        // accumulators of groups i + j .. i + j + c - 1. Pairs past the last separate group go one
        // by one into the shared accumulator. At the first K step the i = 0 products overwrite.
#pragma unroll
        for (int i = 0; i < S; ++i) {
          const uint64_t da = smem_desc(sa + i * A_SLICE);
          const int jmax = (S - 1 - i) < (TC_NACC - 1 - i) ? (S - 1 - i) : (TC_NACC - 1 - i);
          const uint32_t en = (it == 0 && i == 0) ? 0u : 1u;
#pragma unroll
          for (int j0 = 0; j0 <= jmax; j0 += 4) {
            const int c = (jmax - j0 + 1) < 4 ? (jmax - j0 + 1) : 4;
            tc_mma(tmem + (i + j0) * NT, da, smem_desc(sb + j0 * Cfg::BS), idesc_bf16(c * NT), en);
          }
#pragma unroll
          for (int j = jmax + 1; j < S - i; ++j)
            tc_mma(tmem + (TC_NACC - 1) * NT, da, smem_desc(sb + j * Cfg::BS), idesc_bf16(NT), 1u);
        }
        tc_commit(empty0 + 8 * st);  // frees the stage once these MMAs have read it
      }
      tc_commit(done);  // arrives when every MMA issued above has completed
    }
    __syncwarp();
  } else {
    const int ew = warp - 2;    // epilogue warp 0..7
    const int q = warp % 4;     // the TMEM lane quarter this warp may read
    const int half = ew / 4;    // and its half of the tile's NT columns
    int* sec = reinterpret_cast<int*>(smem + Cfg::BAR_OFF - NT * sizeof(int));
    const bool ok = mbar_wait(done, 0, a.wait_ns);
    tc_fence_after();
    // the pipeline stages are free now: column exponents, then one 32 x 17 staging tile per warp
    if (threadIdx.x - 64 < NT) {
      const int col = n0 + threadIdx.x - 64;
      sec[threadIdx.x - 64] = col < a.n ? a.eB[b * a.eBs + col] : 0;
    }
    asm volatile("bar.sync 1, 256;" ::: "memory");  // the eight epilogue warps only
    double* stg = reinterpret_cast<double*>(smem) + ew * 32 * 17;
    const int r = m0 + q * 32 + lane;
    const bool row_in = r < a.m;
    const int er = row_in ? a.eA[b * a.eAs + r] : 0;
    // warp-uniform, since tcgen05.ld is executed by the whole warp
    const bool bad_run = __any_sync(0xffffffffu, !ok || (volatile int&)failed);
    double* Cb = a.C + b * a.sC;
    constexpr int CW = Cfg::CW;
#pragma unroll 1
    for (int cc = 0; cc < NT / 2 / CW; ++cc) {
      const int c = half * (NT / 2 / CW) + cc;  // CW-column chunk of the tile
      // Accumulator g < 7 holds n_g 2^(-7g) with |n_g| < 2^25 exact; the shared one is rounded to
      // units of 2^-49. Exact integers: hi = n_0 2^21 + n_1 2^14 + n_2 2^7 + n_3 (units 2^-21),
      // lo = n_4 2^21 + n_5 2^14 + n_6 2^7 + m (units 2^-49).
      long long hi[CW], lo[CW];
#pragma unroll
      for (int j = 0; j < CW; ++j) hi[j] = lo[j] = 0;
      if (!bad_run) {
#pragma unroll
        for (int g = 0; g < Cfg::NA; ++g) {
          float f[CW];
          tmem_ld<CW>(tmem + ((uint32_t)(q * 32) << 16) + g * NT + c * CW, f);
          const float sc = __int_as_float((127 + (g < TC_NACC - 1 ? 7 * g : 49)) << 23);
#pragma unroll
          for (int j = 0; j < CW; ++j) {
            const long long n = __float2int_rn(f[j] * sc);
            if (g < 4) hi[j] += n << (7 * (3 - g));
            else if (g < TC_NACC - 1) lo[j] += n << (7 * (7 - g));
            else lo[j] += n;
          }
        }
      }
#pragma unroll
      for (int j = 0; j < CW; ++j) {
        const int col = n0 + c * CW + j;
        const int ec = sec[c * CW + j];
        double x;
        if (bad_run || er == kExpBad || ec == kExpBad) {
          x = __longlong_as_double(0x7ff8000000000000ll);
        } else {
          // (hi 2^-21 + lo 2^-49) 2^(er + ec - 14): two exact doubles, one rounding
          const int E = er + ec - 14;
          x = int_to_double_pow2(hi[j], E - 21) + int_to_double_pow2(lo[j], E - 49);
        }
        stg[lane * 17 + j] = (row_in && col < a.n) ? x : 0.0;
      }
      __syncwarp();
      // coalesced: each step writes 32 / CW row segments of CW columns; alpha and beta applied here
#pragma unroll 1
      for (int i = 0; i < CW; ++i) {
        const int rl = (32 / CW) * i + lane / CW, j = lane % CW;
        const int rr = m0 + q * 32 + rl, col = n0 + c * CW + j;
        if (rr < a.m && col < a.n && (!a.sym || col <= rr)) {
          double* cp = Cb + (long long)rr * a.ldc + col;
          double x = a.alpha * stg[rl * 17 + j];
          if (a.beta != 0.0) x += a.beta * *cp;
          *cp = x;
          stg[rl * 17 + j] = x;
        }
      }
      __syncwarp();
      if (a.sym && row_in) {  // mirror: lanes are consecutive rows, so these stores coalesce
#pragma unroll 1
        for (int j = 0; j < CW; ++j) {
          const int col = n0 + c * CW + j;
          if (col < r) Cb[(long long)col * a.ldc + r] = stg[lane * 17 + j];
        }
      }
      __syncwarp();
    }
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && failed && a.status) atomicOr(&a.status[b / a.sdiv], RMHMC_CHAIN_TIMEOUT);
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Cfg::COLS)
                 : "memory");
  }
}

template <int S>
void launch_split(cudaStream_t s, const double* X, int ld, long long sX, bool kmaj, int R, int K,
                  int batch, const TcOperand& op, const int* mask) {
  const long long threads = (long long)op.KS * op.R8 * 16;  // R8 is a multiple of TR8
  dim3 grid((unsigned)((threads + 255) / 256), batch);
  k_tc_split<S><<<grid, 256, 0, s>>>(X, ld, sX, kmaj ? 1 : 0, R, K, op.R8, op.KS, op.TR / 8, op.ex, op.dig,
                                     op.bytes_per_entry, mask);
}

template <int S, int NT>
void launch_gemm(cudaStream_t s, const TcArgs& args, int batch) {
  using Cfg = TcCfg<S, NT>;
  static bool attr[64] = {};  // per device: the shared-memory opt-in is a per-device attribute
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !attr[dev]) {
    cudaFuncSetAttribute(k_gemm_tc<S, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
    if (dev >= 0 && dev < 64) attr[dev] = true;
  }
  dim3 grid((args.n + NT - 1) / NT, (args.m + TC_M - 1) / TC_M, batch);
  k_gemm_tc<S, NT><<<grid, TC_THREADS, Cfg::SMEM, s>>>(args);
}

__global__ void k_scale(double* C, int m, int n, int ldc, long long sC, double beta) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)m * n) return;
  double* c = C + blockIdx.y * sC + (e / n) * ldc + e % n;
  *c = beta == 0.0 ? 0.0 : beta * *c;
}

// The test switch of rmhmc_test_gemm_stall (host side; read at each launch).
int g_stall_entry = -1;
unsigned long long g_wait_ns = kWaitNs;

}  // namespace

int tc_tile_rows(bool b_side) { return b_side ? TC_N : TC_M; }

size_t tc_operand_bytes(int R, int K, int S, int batch, bool b_side) {
  const int TR = tc_tile_rows(b_side);
  const size_t R8 = (size_t)(R + TR - 1) / TR * TR / 8, KS = (K + TC_K - 1) / TC_K;
  const size_t dig = KS * S * R8 * 256, ex = R8 * 8 * sizeof(int);
  return ((dig + 255) / 256 * 256 + (ex + 255) / 256 * 256) * batch;
}

TcOperand tc_operand(void* mem, int R, int K, int S, int batch, bool b_side) {
  TcOperand op;
  op.R = R;
  op.K = K;
  op.S = S;
  op.TR = tc_tile_rows(b_side);
  op.R8 = (R + op.TR - 1) / op.TR * op.TR / 8;
  op.KS = (K + TC_K - 1) / TC_K;
  op.bytes_per_entry = ((long long)op.KS * S * op.R8 * 256 + 255) / 256 * 256;
  op.dig = static_cast<uint8_t*>(mem);
  op.ex = reinterpret_cast<int*>(op.dig + op.bytes_per_entry * batch);
  return op;
}

void tc_split(cudaStream_t s, const double* X, int ld, long long sX, bool kmaj, int batch,
              const TcOperand& op, const int* mask) {
  if (op.R <= 0 || op.K <= 0 || batch <= 0) return;
  const int Rpad = op.R8 * 8;
  if (kmaj)
    k_tc_exponents<<<dim3((Rpad + 7) / 8, batch), 256, 0, s>>>(X, ld, sX, 1, op.R, op.K, Rpad, op.ex, mask);
  else
    k_tc_exponents<<<dim3((Rpad + 31) / 32, batch), 256, 0, s>>>(X, ld, sX, 0, op.R, op.K, Rpad,
                                                                 op.ex, mask);
  switch (op.S) {
    case 6: launch_split<6>(s, X, ld, sX, kmaj, op.R, op.K, batch, op, mask); break;
    case 7: launch_split<7>(s, X, ld, sX, kmaj, op.R, op.K, batch, op, mask); break;
    case 8: launch_split<8>(s, X, ld, sX, kmaj, op.R, op.K, batch, op, mask); break;
    default: launch_split<9>(s, X, ld, sX, kmaj, op.R, op.K, batch, op, mask); break;
  }
}

double gemm_tc_tensor_flops(const TcOperand& A, const TcOperand& B, int batch, bool sym, int nt) {
  nt = nt == 32 ? 32 : TC_N;
  const int tm = (A.R + TC_M - 1) / TC_M, tn = (B.R + nt - 1) / nt;
  long long tiles = 0;  // per batch entry
  for (int i = 0; i < tm; ++i)
    for (int j = 0; j < tn; ++j)
      if (!sym || i * TC_M + TC_M - 1 >= j * nt) ++tiles;
  return (double)tiles * batch * A.KS * (A.S * (A.S + 1) / 2) * 2.0 * TC_M * nt * TC_K;
}

void gemm_tc(cudaStream_t s, const TcOperand& A, const TcOperand& B, double alpha, double beta,
             double* C, int ldc, long long sC, int batch, bool sym, int* status, int sdiv,
             const int* mask, int nt) {
  const int m = A.R, n = B.R, KS = A.KS;
  if (m <= 0 || n <= 0 || batch <= 0) return;
  if (A.TR != TC_M || B.TR != TC_N || B.KS != KS || B.S != A.S) return;  // wrong roles: no launch
  if (KS == 0) {
    const long long mn = (long long)m * n;
    k_scale<<<dim3((unsigned)((mn + 255) / 256), batch), 256, 0, s>>>(C, m, n, ldc, sC, beta);
    return;
  }
  TcArgs a{};
  a.A = A.dig;
  a.sA = A.shared ? 0 : A.bytes_per_entry;
  a.RA8 = A.R8;
  a.eA = A.ex;
  a.eAs = A.shared ? 0 : (long long)A.R8 * 8;
  a.B = B.dig;
  a.sB = B.shared ? 0 : B.bytes_per_entry;
  a.RB8 = B.R8;
  a.eB = B.ex;
  a.eBs = B.shared ? 0 : (long long)B.R8 * 8;
  a.m = m;
  a.n = n;
  a.KS = KS;
  a.alpha = alpha;
  a.C = C;
  a.ldc = ldc;
  a.sC = sC;
  a.sym = sym ? 1 : 0;
  a.status = status;
  a.sdiv = sdiv > 0 ? sdiv : 1;
  a.mask = mask;
  a.wait_ns = g_wait_ns;
  a.stall_entry = g_stall_entry;
  for (int k0 = 0; k0 < KS; k0 += TC_KSTEPS_MAX) {
    a.ks0 = k0;
    a.ks1 = k0 + TC_KSTEPS_MAX < KS ? k0 + TC_KSTEPS_MAX : KS;
    a.beta = k0 == 0 ? beta : 1.0;
    if (nt == 32) {
      switch (A.S) {
        case 6: launch_gemm<6, 32>(s, a, batch); break;
        case 7: launch_gemm<7, 32>(s, a, batch); break;
        case 8: launch_gemm<8, 32>(s, a, batch); break;
        default: launch_gemm<9, 32>(s, a, batch); break;
      }
    } else {
      switch (A.S) {
        case 6: launch_gemm<6, 64>(s, a, batch); break;
        case 7: launch_gemm<7, 64>(s, a, batch); break;
        case 8: launch_gemm<8, 64>(s, a, batch); break;
        default: launch_gemm<9, 64>(s, a, batch); break;
      }
    }
  }
}

}  // namespace rmhmc

extern "C" rmhmc_status rmhmc_gemm_tc(void* cuda_stream, int ta, int tb, int m, int n, int k,
                                      double alpha, const double* A_dev, int lda, long long strideA,
                                      const double* B_dev, int ldb, long long strideB, double beta,
                                      double* C_dev, int ldc, long long strideC, int batch,
                                      int slices, int sym, int* status_dev) {
  using namespace rmhmc;
  if (m < 0 || n < 0 || k < 0 || batch < 0 || slices < 6 || slices > 9) return RMHMC_EINVAL;
  if (sym && m != n) return RMHMC_EINVAL;
  if (m == 0 || n == 0 || batch == 0) return RMHMC_OK;
  if (!C_dev || ldc < n || (k > 0 && (!A_dev || !B_dev))) return RMHMC_EINVAL;
  if (k > 0 && (lda < (ta ? m : k) || ldb < (tb ? k : n))) return RMHMC_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const size_t ba = tc_operand_bytes(m, k, slices, batch, false),
               bb = tc_operand_bytes(n, k, slices, batch, true);
  void* mem = nullptr;
  if (cudaMallocAsync(&mem, ba + bb, s) != cudaSuccess) {
    cudaGetLastError();
    return RMHMC_ENOMEM;
  }
  const TcOperand oa = tc_operand(mem, m, k, slices, batch, false);
  const TcOperand ob = tc_operand(static_cast<char*>(mem) + ba, n, k, slices, batch, true);
  // row i of op(A) is row i of A unless ta; row j of op(B)^T is row j of B when tb
  tc_split(s, A_dev, lda, strideA, !ta, batch, oa);
  tc_split(s, B_dev, ldb, strideB, tb != 0, batch, ob);
  gemm_tc(s, oa, ob, alpha, beta, C_dev, ldc, strideC, batch, sym != 0, status_dev, 1);
  const cudaError_t e = cudaGetLastError();
  cudaFreeAsync(mem, s);
  return e == cudaSuccess ? RMHMC_OK : RMHMC_ECUDA;
}

extern "C" rmhmc_status rmhmc_test_gemm_stall(int entry, double wait_ms) {
  using namespace rmhmc;
  if (entry < 0) {
    g_stall_entry = -1;
    g_wait_ns = kWaitNs;
    return RMHMC_OK;
  }
  if (!(wait_ms >= 1.0 && wait_ms <= 2000.0)) return RMHMC_EINVAL;
  g_stall_entry = entry;
  g_wait_ns = (unsigned long long)(wait_ms * 1e6);
  return RMHMC_OK;
}
