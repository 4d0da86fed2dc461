// Internal declarations shared by the CUDA translation units of librmhmc (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "rmhmc.h"

namespace rmhmc {

// log2 |x| for a finite double, from its exponent field and the FP32 log2 of its significand
// (integer and FP32 operations only; B300's FP64 pipe is 1/64 of its FP32 rate). Zero gives -2000,
// a subnormal the log2 of 2^-1023.
__device__ __forceinline__ float log2_abs(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
  if (b == 0) return -2000.f;
  const int e = (int)(b >> 52) - 1023;
  const float m = __int_as_float(0x3f800000 | (int)((b >> 29) & 0x7fffff));  // significand in [1, 2)
  return (float)e + __log2f(m);
}


constexpr int kMaxN = 1024;       // inputs per problem (FP64 path)
constexpr int kJacBlk = 8;        // Jacobi index block b; a rotated pair of blocks is 16 x 16
constexpr int kJacSB = 2 * kJacBlk;
constexpr int kStatSlots = 32;    // per (chain, kernel) scalar slots

// per (chain, kernel) scalar slot indices (see model kernels)
enum Stat {
  ST_LOGDET = 0,  // log|K|
  ST_FA,          // f . alpha
  ST_AB,          // alpha . beta          (alpha^T D1 alpha)
  ST_AE2,         // alpha . eps2          (alpha^T D2 alpha)
  ST_AE3,         // alpha . eps3          (alpha^T D3 alpha)
  ST_AD,          // alpha . delta         (alpha^T D1 K^-1 D1 alpha ... via delta = D1 gamma)
  ST_GB,          // gamma . beta
  ST_GD,          // gamma . delta
  ST_GE2,         // gamma . eps2
  ST_TRS,         // tr(S)     = <K^-1, D1>
  ST_TRS2,        // tr(S^2)
  ST_TRS3,        // tr(S^3)
  ST_TRR2,        // <K^-1, D2>
  ST_TRR3,        // <K^-1, D3>
  ST_TRSR2,       // <A1, D2> = tr(K^-1 D1 K^-1 D2)
  ST_COUNT
};

struct KernelDev {
  int kind;
  int n_cols;
  int cols[RMHMC_MAX_COLS];
  double jitter;
  double a[2];
  double b[2];
};

struct ModelDev {
  int N, n, P, d, dp, ncov, lik, sample_hypers, n_chains;
  double noise_var;
  const double* X;        // N x ncov
  const double* y;        // N
  const double* u_fixed;  // 2n
  const double* tau;      // n_chains
  KernelDev k[RMHMC_MAX_KERNELS];
};

// The primal (reduced-rank) model: M sinusoidal features per Gaussian-kernel column of Xg, one
// coefficient per linear-kernel column of Xl, a bias; P = M Dg + Dl + 1 coefficients per latent
// function, J functions, then (u_cg, u_sg, u_cl); d = J P + 3.
struct PrimalDev {
  int N, Dg, Dl, M, P, d, dp, lik, n_chains;
  int J, JP;  // latent functions (1 or 2) and J P, the offset of (u_cg, u_sg, u_cl) in q
  double noise_var, L, bias_var, delta;
  double a[3], b[3];
  const double* Xg;   // N x Dg
  const double* Xl;   // N x Dl
  const double* y;    // N
  const double* tau;  // n_chains
};

struct GeomDev {
  int g_kind;
  double alpha;
};

// ---------------------------------------------------------------- linear algebra (linalg.cu)
// Batched FP64 GEMM: C_b = alpha op(A_b) op(B_b) + beta C_b, row-major. op(A) is m x k, op(B) is
// k x n. sym: m == n and the product is symmetric: only tiles on/below the diagonal are computed
// and mirrored. tri: A and B are op()-views of lower-triangular factors with (op(A) op(B))_ij
// summing over k >= max(i, j) only (used for K^-1 = L^-T L^-1).
void gemm_f64(cudaStream_t s, bool ta, bool tb, int m, int n, int k, double alpha, const double* A,
              int lda, long long sA, const double* B, int ldb, long long sB, double beta, double* C,
              int ldc, long long sC, int batch, bool sym, bool tri);
// In-place lower Cholesky of batch N x N matrices (row-major, ld = N); writes log|K| to
// logdet[b * logdet_stride] and sets status bit RMHMC_CHAIN_NOTPD in status[b / per_chain].
// rdiag: batch x 32 doubles of scratch (the reciprocal pivots of one panel).
void cholesky_f64(cudaStream_t s, double* A, int N, int batch, double* logdet, int logdet_stride,
                  int* status, int per_chain, double* rdiag);
// The same with the trailing updates A22 -= L21 L21^T on the tensor cores (gemm_tc, 9 slices); the
// panels (diagonal block and L21 by substitution) stay FP64. tcA / tcB: slices of N x 32 operands.
void cholesky_tc(cudaStream_t s, double* A, int N, int batch, double* logdet, int logdet_stride,
                 int* status, int per_chain, uint8_t* tcA, uint8_t* tcB, double* rdiag);
// t = L^-1 f and a = L^-T t (= K^-1 f) by substitution, per (batch) factor L.
void cholsolve_f64(cudaStream_t s, const double* L, const double* f, double* t, double* a, int N,
                   int batch);
// X = L^-1 (lower triangular) for batch matrices.
void trinv_lower_f64(cudaStream_t s, const double* L, double* X, int N, int batch);
// The same, recursively with the off-diagonal blocks X21 = -X22 (L21 X11) on the tensor cores
// (gemm_tc, 9 slices): tcA / tcB hold the operands' slices (A side and B side, up to N x N), T is
// batch x N x N doubles of scratch (only (N/2 + 16)^2 per matrix used).
void trinv_lower_tc(cudaStream_t s, const double* L, double* X, int N, int batch, uint8_t* tcA,
                    uint8_t* tcB, double* T, int* status, int sdiv);
// y_b = op(A_b) x_b for batch N x N (ld) matrices; row-major.
void gemv_f64(cudaStream_t s, bool ta, int rows, int cols, const double* A, int lda, long long sA,
              const double* x, long long sx, double* y, long long sy, int batch, double alpha,
              double beta);

// ---------------------------------------------------------------- tensor-core GEMM (tcgemm.cu)
// FP64-accurate GEMM on tcgen05 by error-free bf16 slicing. An operand is the K-major view of a
// matrix (R rows, K columns) split into S bf16 slices (6..9) plus one exponent per row, in device
// memory of tc_operand_bytes(R, K, S, batch) bytes placed by tc_operand.
// The slices are laid out for one role: A (tiles of 128 rows, b_side = false) or B (64 rows).
struct TcOperand {
  uint8_t* dig = nullptr;  // slices, bytes_per_entry per batch entry
  int* ex = nullptr;       // row exponents, R8 * 8 per batch entry
  int R = 0, K = 0, S = 0, TR = 0, R8 = 0, KS = 0;
  long long bytes_per_entry = 0;
  bool shared = false;  // one entry read by every batch entry of a product (split with batch 1)
};
int tc_tile_rows(bool b_side);
size_t tc_operand_bytes(int R, int K, int S, int batch, bool b_side);
TcOperand tc_operand(void* mem, int R, int K, int S, int batch, bool b_side);
// Split the K-major view of X (kmaj: row r is X[r * ld + 0..K), else column r, X[0..K) * ld + r).
void tc_split(cudaStream_t s, const double* X, int ld, long long sX, bool kmaj, int batch,
              const TcOperand& op, const int* mask = nullptr);
// C_b = alpha A_b B_b^T + beta C_b (A: m x k rows, B: n x k rows, both split with the same S and
// K); sym: the product is symmetric, written as the mirror of its lower triangle. A bounded wait
// that gives up sets RMHMC_CHAIN_TIMEOUT in status[b / sdiv] (status may be null).
// mask (optional, batch ints): entries with mask[b] == 0 are skipped by the split and the product.
// nt: output tile width, 64 (default) or 32 (twice the tiles, half the columns each; the same
// operands).
void gemm_tc(cudaStream_t s, const TcOperand& A, const TcOperand& B, double alpha, double beta,
             double* C, int ldc, long long sC, int batch, bool sym, int* status, int sdiv,
             const int* mask = nullptr, int nt = 64);
// bf16 tensor-core FLOPs gemm_tc executes for these operands (padded tiles, all slice products).
double gemm_tc_tensor_flops(const TcOperand& A, const TcOperand& B, int batch, bool sym, int nt = 64);

// ---------------------------------------------------------------- eigen (eigen.cu)
// Warm-started block-Jacobi on M (dp x dp per chain, symmetric), rotating PsiT's rows alongside;
// writes lam (dp per chain) and the sweep count; sets RMHMC_CHAIN_NOTCONV on failure. Chains
// whose status is nonzero on entry are skipped.
constexpr int kJacStats = 8;  // counters per chain in JacobiWork::tiles
struct JacobiWork {
  double* V;      // n_chains x (nb/2) x 256
  double* D;      // n_chains x (nb/2) x 256
  double* slots;  // n_chains x 64
  int* flags;     // n_chains x (nb/2): pair rotated in the current round
  unsigned long long* tiles;  // n_chains x kJacStats counters (null = not counted): += 16 x 16 x 16
                              // tile products executed (phase 2), rotation rounds applied to
                              // 16 x 16 blocks (phase 1), outer rounds, 16 x 16 sub-problems solved,
                              // of which rotated, eigen-updates, pre-rotated updates and pairs
  float* crit;    // n_chains x nb x nb: coupling criterion per pair of 8-wide blocks (dynamic schedule)
};
void jacobi_f64(cudaStream_t s, double* M, double* PsiT, double* lam, int dp, int d, int n_chains,
                int rule, double tol, int max_sweeps, int* status, int* sweeps_out, int* sweeps_acc,
                JacobiWork w, int cluster, int sched);
// The same eigen-update with the phase-2 rotations in double-float (FP32 pair) arithmetic;
// pair_scratch_M / pair_scratch_P are n_chains x dp x dp doubles of scratch (used as float2, laid
// out as M and Psi^T). Chains c with pre[c] != 0 (pre may be null) start from the pairs already in
// the scratch (written by the pre-rotation) instead of converting M and Psi^T; every chain ends with
// M, Psi^T and lam written from the pairs.
void jacobi_df(cudaStream_t s, double* M, double* PsiT, double* lam, int dp, int d, int n_chains,
               int rule, double tol, int max_sweeps, int* status, int* sweeps_out, int* sweeps_acc,
               JacobiWork w, int cluster, double* pair_scratch_M, double* pair_scratch_P, int sched,
               const int* pre);
// Modified Gram-Schmidt on the first d rows of PsiT (dp x dp per chain), for chains whose
// eig_count is a positive multiple of every (0 = never).
void mgs_rows_f64(cudaStream_t s, double* PsiT, int dp, int d, int n_chains, const int* eig_count,
                  int every, int cluster);
int jacobi_cluster_size(int n_chains);

// ---------------------------------------------------------------- model kernels (model.cu side)
}  // namespace rmhmc
