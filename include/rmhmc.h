/*
 * rmhmc.h - C ABI of the B300 (sm_103a) SoftAbs-RMHMC library for hierarchical Gaussian-process
 * models (Hayakawa and Asai, "Fast Riemannian-manifold Hamiltonian Monte Carlo for hierarchical
 * Gaussian-process models").
 *
 * Model (Sec. 2.1, Eq. data_likelihood with J = 1, Eq. BMKL, Eq. hpar_prior), dual form:
 *   F = sum_k f_k, f_k ~ N(0, K_k(u_k)) over the N inputs, y_m | F_m ~ Bernoulli(sigmoid(F_m)) or
 *   N(F_m, noise_var); u_k = (log c_k, log theta_k) with theta = exp(u) ~ InvGamma(a, b) per
 *   hyperparameter; tempered posterior P_tau ∝ P(y | F)^tau * prior (Sec. "MC integration for BME").
 *   Position q = (f_1[0:N], ..., f_n[0:N], u_1[0:2], ..., u_n[0:2]), d = nN + 2n
 *   (d = nN when the hyperparameters are held fixed).
 *   Kernels:  SE      k = c (exp(-|x - x'|^2 / (2 theta^2)) + jitter [same sample])
 *             LINEAR  k = c (x . x' + theta + jitter [same sample])
 *             OVERLAP k = c (exp(-#mismatching columns / theta) + jitter [same sample])
 * Sampler (Sec. 2.2, Algorithm 1): Hamiltonian of Eq. Hamiltonian with the soft-absolute metric
 *   G = Psi g(Lambda) Psi^T of the Hessian H = Psi Lambda Psi^T; generalized leapfrog of
 *   Eq. leapfrog with n_fp fixed-point iterations for each implicit half; gradient terms through
 *   the Betancourt contractions W1, W2 (Eq. d3_transform, Eq. Betancourt_formula); eigenvectors
 *   carried across substeps by warm-started Jacobi (Sec. 2.4).
 *
 * Conventions
 *   - Every pointer argument is owned by the caller. Arguments named *_dev are device pointers
 *     (e.g. torch CUDA tensors) on the device that was current at rmhmc_init_model; *_host are
 *     host pointers. Arrays are row-major, float64 unless stated, chain-major (n_chains x ...).
 *   - The model owns its device copies, per-chain state and workspaces until rmhmc_free_model.
 *   - Calls enqueue work on the stream given at init and return without synchronising, except
 *     where stated; read outputs after synchronising that stream.
 *   - The return value is the call-level status. Per-chain numerical failures (a kernel matrix
 *     that is not positive definite, a non-finite value, Jacobi that did not converge) never abort
 *     a call: they are reported per chain in status_dev and, inside rmhmc_sample, make the
 *     proposal rejected.
 */
#ifndef RMHMC_H
#define RMHMC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RMHMC_OK = 0,
  RMHMC_EINVAL = 1,     /* bad argument (sizes, kinds, null pointers) */
  RMHMC_ENOMEM = 2,     /* device allocation failed */
  RMHMC_ECUDA = 3,      /* a CUDA runtime call failed */
  RMHMC_ENOTCONV = 4,   /* per chain: Jacobi did not reach the tolerance within max_sweeps */
  RMHMC_ENONFINITE = 5, /* per chain: a non-finite Hamiltonian or position */
  RMHMC_ETIMEOUT = 6,   /* a bounded device-side wait gave up */
  RMHMC_ENOTIMPL = 7,   /* option not implemented in this build */
  RMHMC_ENOTPD = 8,     /* per chain: a kernel matrix lost positive definiteness (Cholesky) */
  RMHMC_ESCRATCH = 9    /* rmhmc_eigh_noalloc: the batch does not fit its fixed workspace */
} rmhmc_status;

/* per-chain status bits written to status_dev / chain_status_dev (0 = healthy) */
#define RMHMC_CHAIN_NOTPD 1
#define RMHMC_CHAIN_NOTCONV 2
#define RMHMC_CHAIN_NONFINITE 4
#define RMHMC_CHAIN_TIMEOUT 8   /* a bounded device-side wait gave up (results of that call invalid) */

typedef enum {
  RMHMC_LIK_BERNOULLI_LOGIT = 0,
  RMHMC_LIK_GAUSSIAN = 1,
  RMHMC_LIK_MEANVAR = 2  /* primal model with J = 2 only: y ~ N(F_1, delta + exp F_2) (Example 1) */
} rmhmc_lik;
typedef enum { RMHMC_K_SE = 0, RMHMC_K_LINEAR = 1, RMHMC_K_OVERLAP = 2 } rmhmc_kernel_kind;
typedef enum { RMHMC_G_COTH = 0, RMHMC_G_SQRT = 1 } rmhmc_gkind;
typedef enum { RMHMC_FP64 = 0, RMHMC_MIXED = 1 } rmhmc_precision;
/* Jacobi stopping rules (u = 2^-53, floor = 4 u ||M||_F, d_min = min_i |m_ii|): sweeps continue
 * while some pair j != l has
 *   METRIC:   |m_jl| > max(zeta |m_jj m_ll| / d_min, floor)  -- first-order error of G^-1, W1, W2
 *             and log|G| below zeta relative; eigenvalues inside near-degenerate clusters are
 *             left mixed (the metric is insensitive to that), which saves most sweeps
 *   RELATIVE: |m_jl| > max(zeta sqrt(|m_jj m_ll|), floor)   -- every eigenpair resolved */
typedef enum { RMHMC_JACOBI_METRIC = 0, RMHMC_JACOBI_RELATIVE = 1 } rmhmc_jacobi_rule;
/* Order of the Jacobi rotations (Sec. 2.4's Jacobi; the same stopping rule either way):
 *   CYCLIC:  round-robin sweeps, every pair of 8-wide index blocks once per sweep;
 *   DYNAMIC: each round pairs the blocks greedily by their largest remaining coupling (under the
 *            stopping rule) and solves only the pairs above the tolerance, which after a warm
 *            start is a few per round; sweeps are then reported as rounds / (blocks - 1).
 * The order applies to warm eigen-updates; a cold start (rmhmc_set_state, or every update of the
 * static ablation, eigen_start = 1) always takes the cyclic order. */
typedef enum { RMHMC_JACOBI_CYCLIC = 0, RMHMC_JACOBI_DYNAMIC = 1 } rmhmc_jacobi_schedule;

#define RMHMC_MAX_COLS 16
#define RMHMC_MAX_KERNELS 3

/* One GP component (Eq. BMKL): kernel kind, the input columns it reads, the jitter and the
 * InvGamma(a, b) hyperpriors (Eq. hpar_prior) on (c, theta). */
typedef struct {
  int kind;                   /* rmhmc_kernel_kind */
  int n_cols;                 /* 1..RMHMC_MAX_COLS */
  int cols[RMHMC_MAX_COLS];   /* column indices into X */
  double jitter;              /* > 0; K = c (K~ + jitter I) */
  double prior_a[2];          /* shape of InvGamma on (c, theta) */
  double prior_b[2];          /* scale of InvGamma on (c, theta) */
} rmhmc_kernel_desc;

/* The data and model. X, y, kernels and u_fixed are host pointers, read during
 * rmhmc_init_model only. */
typedef struct {
  int N;                        /* number of inputs, 1..1024 */
  int n_cov;                    /* columns of X */
  const double* X;              /* host, N x n_cov */
  const double* y;              /* host, N (0/1 for Bernoulli) */
  int lik;                      /* rmhmc_lik */
  double noise_var;             /* Gaussian likelihood variance */
  int n_kernels;                /* 1..RMHMC_MAX_KERNELS */
  const rmhmc_kernel_desc* kernels;
  int sample_hypers;            /* 1: q includes u; 0: u held at u_fixed */
  const double* u_fixed;        /* host, 2 n_kernels, used when sample_hypers == 0 */
} rmhmc_model_desc;

/* Integrator and geometry settings. The geometry fields (g_kind, alpha, jacobi_tol, max_sweeps,
 * reorth_every, precision, jacobi_rule, eigen_start) must be the same in every call on a model as in
 * rmhmc_set_state. */
typedef struct {
  double eps;          /* leapfrog step size (Eq. leapfrog) */
  int n_leapfrog;      /* leapfrogs per MH proposal (C in Algorithm 1) */
  int n_fp;            /* fixed-point iterations for each implicit half-step, >= 1 */
  int g_kind;          /* rmhmc_gkind: g = l coth(alpha l) or sqrt(1/alpha^2 + l^2) */
  double alpha;        /* soft-abs sharpness (kappa = 1 / alpha for the sqrt map) */
  double jacobi_tol;   /* zeta, the tolerance of Sec. 2.4 (see jacobi_rule for how it is applied) */
  int max_sweeps;      /* Jacobi sweep limit per eigen-update */
  int reorth_every;    /* Gram-Schmidt of Psi every this many eigen-updates (Sec. 2.4); 0 = never */
  int precision;       /* rmhmc_precision: FP64, or MIXED = the Jacobi rotations in double-float
                          (FP32 pairs, ~48-bit significand), and the K^-1 algebra (K^-1 = L^-T L^-1,
                          K^-1 dK and its products) and the d x d products M = Psi^T H Psi and
                          W = Psi C Psi^T on the tensor cores (rmhmc_gemm_tc with 9 and 7 slices);
                          Cholesky, L^-1, H, log|G| and the Hamiltonian stay FP64 */
  int jacobi_rule;     /* rmhmc_jacobi_rule: when M = Psi^T H Psi counts as diagonal */
  int eigen_start;     /* 0: warm start from the previous Psi (dynamic, Sec. 2.4); 1: cold start
                          from Psi = I at every eigen-update (the static ablation of Sec. 3.1) */
} rmhmc_integrator;

typedef struct rmhmc_model rmhmc_model;

/* Validate the description, copy X, y and the kernel descriptors to the device and allocate the
 * per-chain state for n_chains chains (positions, momenta, eigenvectors, workspaces).
 * tau_host: n_chains inverse temperatures in (0, 1] (NULL = all 1). cuda_stream: a cudaStream_t
 * (NULL = legacy default stream). On success *out owns the device memory.
 * Errors: EINVAL (bad sizes/kinds), ENOMEM, ECUDA. */
rmhmc_status rmhmc_init_model(const rmhmc_model_desc* desc, int n_chains, const double* tau_host,
                              void* cuda_stream, rmhmc_model** out);

/* Device bytes rmhmc_init_model would allocate for desc and n_chains (every buffer, each rounded
 * to 256 bytes), without allocating: what an admission controller budgets HBM with. The arrays
 * in desc are not read (only the sizes and kinds). Errors: EINVAL. */
rmhmc_status rmhmc_plan_bytes(const rmhmc_model_desc* desc, int n_chains, size_t* bytes);

/* The primal (reduced-rank) model of the paper's experiments (Sec. 2.1 Eq. Solin_representation,
 * the reduced-rank appendix, Sec. 2.5): every covariate column of Xg has a one-dimensional
 * Gaussian kernel represented by M sinusoidal features phi_m(x) = sin(pi m (x + L) / (2L))
 * (m = 1..M) with coefficients a_km ~ N(0, c_g V_m(s_g)), V_m(s) = sqrt(pi s)
 * exp(-pi^2 m^2 s / (16 L^2)) (the spectral density of exp(-r^2/s) at pi m / (2L)); every column
 * of Xl has a linear kernel, a_l ~ N(0, c_l); a bias b ~ N(0, bias_var); one shared (c_g, s_g) for
 * the Gaussian kernels and one c_l for the linear ones, each ~ InvGamma(prior_a, prior_b) and
 * sampled as u = log(theta). F_i = sum_km a_km phi_m(Xg_ik) + sum_l a_l Xl_il + b, and the
 * likelihood is lik on (F_i, y_i) tempered by tau. Coordinates q = (a_km (k-major, m fastest),
 * a_l, b, u_cg, u_sg, u_cl): d = M n_gauss + n_linear + 4 (= 30 D + 4 for Sec. 2.5). With J = 2
 * (Example 1 of Sec. 2.1, the covariate-dependent mean and variance of Sec. 2.6) there are two
 * functions F_1, F_2 on the same features with y_i ~ N(F_1i, delta + exp F_2i): q = (coefficients
 * of F_1, coefficients of F_2, u_cg, u_sg, u_cl), d = 2 P + 3 with P = M n_gauss + n_linear + 1.
 * Host arrays are read during rmhmc_init_primal only. */
typedef struct {
  int N;                        /* number of samples, >= 1 */
  int n_gauss;                  /* columns of Xg (Gaussian kernels), >= 0 */
  int n_linear;                 /* columns of Xl (linear kernels), >= 0 */
  const double* Xg;             /* host, N x n_gauss (NULL if n_gauss == 0) */
  const double* Xl;             /* host, N x n_linear (NULL if n_linear == 0) */
  const double* y;              /* host, N (0/1 for Bernoulli) */
  int lik;                      /* rmhmc_lik */
  double noise_var;             /* Gaussian likelihood variance */
  int M;                        /* features per Gaussian kernel, >= 1 */
  double L;                     /* half-width of the feature domain [-L, L], > 0 */
  double bias_var;              /* Sigma, the prior variance of b, > 0 */
  double prior_a[3];            /* InvGamma shapes for (c_g, s_g, c_l) */
  double prior_b[3];            /* InvGamma scales for (c_g, s_g, c_l) */
  int J;                        /* latent functions: 1, or 2 for the mean/variance model (lik must
                                   then be RMHMC_LIK_MEANVAR); each has its own coefficients on the
                                   same features, all share (c_g, s_g, c_l) */
  double delta;                 /* J = 2: the fixed variance floor, >= 0 */
} rmhmc_primal_desc;

/* As rmhmc_init_model, for the primal model; the returned model works with every other call of
 * this header. Errors: EINVAL (bad sizes, d > 4096, N > 2^20), ENOMEM, ECUDA. */
rmhmc_status rmhmc_init_primal(const rmhmc_primal_desc* desc, int n_chains, const double* tau_host,
                               void* cuda_stream, rmhmc_model** out);
/* As rmhmc_plan_bytes, for the primal model. */
rmhmc_status rmhmc_plan_bytes_primal(const rmhmc_primal_desc* desc, int n_chains, size_t* bytes);

/* Set every chain's position (q_dev: n_chains x d) and momentum (p_dev: n_chains x d, may be
 * NULL = zero) and evaluate the geometry there: U, its gradient, Hessian (Eq. d_Hamiltonian
 * derivatives), a cold-start Jacobi eigendecomposition from Psi = I (Sec. 2.4), and the
 * third-derivative operator of Sec. 2.3. Errors: EINVAL, ECUDA. */
rmhmc_status rmhmc_set_state(rmhmc_model* m, const rmhmc_integrator* integ, const double* q_dev,
                             const double* p_dev);

/* Advance every chain by n_steps generalized leapfrogs (Eq. leapfrog) from the model's state,
 * then copy the state out. p_in_dev (n_chains x d, may be NULL): momenta to start from instead of
 * the model's current ones (the geometry depends on q only, so nothing is recomputed). Outputs:
 * q_dev, p_dev (n_chains x d), H_dev (n_chains, Eq. Hamiltonian at the end), status_dev
 * (n_chains ints, RMHMC_CHAIN_* bits seen since rmhmc_set_state or the last Algorithm 1 iteration;
 * RMHMC_CHAIN_NONFINITE when the chain's q, p, U or, if H_dev is given, H is not finite at the
 * end); each may be NULL. Errors: EINVAL, ECUDA. */
rmhmc_status rmhmc_leapfrog(rmhmc_model* m, const rmhmc_integrator* integ, int n_steps,
                            const double* p_in_dev, double* q_dev, double* p_dev, double* H_dev,
                            int* status_dev);

/* Algorithm 1 for n_burn + n_iter iterations from the model's state: momentum p = G^{1/2} z with
 * z from Philox4x64-10 (key (seed, chain), counter (block, iteration, 0, 0)), n_leapfrog
 * leapfrogs, Metropolis-Hastings with r from counter (0, iteration, 1, 0) (accept iff
 * log r < H0 - H1). Iteration numbers continue across calls on the same model. The last n_iter
 * iterations are recorded: q_samples_dev (n_iter x n_chains x d), logp_dev (n_iter x n_chains,
 * log P_tau(q) = -U(q)), loglik_dev (n_iter x n_chains, the untempered log-likelihood
 * ln P(y | F), the integrand of thermodynamic integration for the model evidence), accept_dev
 * (n_iter x n_chains ints), sweeps_dev (n_iter x n_chains ints,
 * Jacobi sweeps in that iteration's trajectory), chain_status_dev (n_chains ints, OR of the
 * RMHMC_CHAIN_* bits seen). Any output pointer may be NULL. The host enqueues iteration by
 * iteration; the call returns after enqueueing. Errors: EINVAL, ECUDA. */
rmhmc_status rmhmc_sample(rmhmc_model* m, const rmhmc_integrator* integ, int n_iter, int n_burn,
                          uint64_t seed, double* q_samples_dev, double* logp_dev,
                          double* loglik_dev, int* accept_dev, int* sweeps_dev,
                          int* chain_status_dev);

/* Copy out the geometry at the current state (for checks and diagnostics): U_dev (n_chains),
 * dU_dev (n_chains x d), hess_dev (n_chains x d x d, Hessian of U), lam_dev (n_chains x d,
 * eigenvalues in the solver's order), G_dev (n_chains x d x d, the soft-abs metric), sweeps_dev
 * (n_chains ints, sweeps of the last eigen-update). Any pointer may be NULL. */
rmhmc_status rmhmc_geometry(rmhmc_model* m, double* U_dev, double* dU_dev, double* hess_dev,
                            double* lam_dev, double* G_dev, int* sweeps_dev);

/* At the current position and a given momentum p_dev (n_chains x d): dHdq_dev = dH/dq
 * (dU + 1/2 tr(W2 dH_i) - 1/2 tr(W1 dH_i), Eq. Betancourt_formula with the sign of the derivative
 * of Eq. Hamiltonian), Ginv_p_dev = G^-1 p = dH/dp, H_dev = Eq. Hamiltonian. NULL skips an output. */
rmhmc_status rmhmc_hamiltonian_grad(rmhmc_model* m, const double* p_dev, double* dHdq_dev,
                                    double* Ginv_p_dev, double* H_dev);

/* ---------------------------------------------------------------- uneven batches (one graph)
 * A batch advances several models of different sizes (N, kernels, chains) together: the first
 * rmhmc_batch_leapfrog captures one generalized leapfrog of every model into a single CUDA graph
 * (each model's kernels on its own stream, forked from and joined back to the batch stream with
 * events, so models overlap on the GPU) and every call replays it n_steps times with one graph
 * launch per leapfrog; the graph is re-captured when eps or n_fp change. cuda_stream must be a
 * created stream (the legacy default stream cannot be captured); every model needs its own
 * non-default stream (distinct from cuda_stream), a state (rmhmc_set_state) and profiling off.
 * The models stay usable on their own; rmhmc_batch_free does not free them.
 * Errors: EINVAL (bad arguments, shared or default streams, no state), ECUDA (capture failed). */
typedef struct rmhmc_batch rmhmc_batch;
rmhmc_status rmhmc_batch_create(rmhmc_model* const* models, int n_models, void* cuda_stream,
                                rmhmc_batch** out);
rmhmc_status rmhmc_batch_leapfrog(rmhmc_batch* b, const rmhmc_integrator* integ, int n_steps);
void rmhmc_batch_free(rmhmc_batch* b);

/* Serving (continuous batching of sampling jobs on one GPU). A server owns one scheduler thread
 * on `device`. rmhmc_server_submit deep-copies a job (its model description, tau and initial state
 * are host data read during the call) and queues it with its footprint: rmhmc_plan_bytes (or
 * rmhmc_plan_bytes_primal) plus the server's per-job buffers. The scheduler admits queued jobs in
 * submission order while the head of the queue fits in what is left of hbm_budget_bytes, gives each
 * admitted job its own model and non-blocking CUDA stream, sets the state (q0, or zero) and keeps
 * `depth` one-iteration rmhmc_sample calls in flight per job; jobs of different sizes run
 * concurrently and their kernels overlap. It notices completion by event queries, releases a
 * finished job's model and stream at once and returns its bytes to the budget, so new jobs are
 * admitted while others run. The results are those of one rmhmc_sample(n_iter, n_burn, seed) call
 * on the job's model (iteration numbers continue across the one-iteration calls), and a job's
 * results do not depend on what else is running. Outputs go to the caller's device buffers, which
 * must stay valid until the job is done (state RMHMC_JOB_DONE or RMHMC_JOB_FAILED). Calls are
 * thread-safe; times are seconds since rmhmc_server_create. */
typedef struct rmhmc_server rmhmc_server;
typedef enum {
  RMHMC_JOB_QUEUED = 0,
  RMHMC_JOB_RUNNING = 1,
  RMHMC_JOB_DONE = 2,
  RMHMC_JOB_FAILED = 3  /* the model could not be created or a call failed: see job_error */
} rmhmc_job_state;
typedef struct {
  const rmhmc_model_desc* model;   /* dual model (host), or NULL */
  const rmhmc_primal_desc* primal; /* primal model (host), or NULL: exactly one of the two */
  int n_chains;
  const double* tau_host;          /* n_chains inverse temperatures, NULL = all 1 */
  const double* q0_host;           /* n_chains x d initial positions, NULL = zero */
  rmhmc_integrator integ;
  int n_iter;                      /* recorded iterations */
  int n_burn;                      /* burn-in iterations before them */
  uint64_t seed;
  double* q_samples_dev;           /* n_iter x n_chains x d, or NULL */
  double* logp_dev;                /* n_iter x n_chains, or NULL */
  int* accept_dev;                 /* n_iter x n_chains, or NULL */
  int* chain_status_dev;           /* n_chains: OR of the RMHMC_CHAIN_* bits of every iteration, or NULL */
  double* loglik_dev;              /* n_iter x n_chains untempered ln P(y | F) per sample (the
                                      thermodynamic-integration input of the BME appendix), or NULL */
} rmhmc_job_desc;
/* depth >= 1: iterations in flight per job. Errors: EINVAL. */
rmhmc_status rmhmc_server_create(int device, size_t hbm_budget_bytes, int depth, rmhmc_server** out);
/* Queue a job; *job_id receives its id. Errors: EINVAL (bad description, or a footprint larger than
 * the whole budget). */
rmhmc_status rmhmc_server_submit(rmhmc_server* s, const rmhmc_job_desc* job, int* job_id);
/* A job's state (rmhmc_job_state), its error (RMHMC_OK unless FAILED) and, in times_host[3], its
 * submission, admission and finish times (-1 until they happen); each output may be NULL. */
rmhmc_status rmhmc_server_poll(rmhmc_server* s, int job_id, int* state, rmhmc_status* job_error,
                               double* times_host);
/* Block until the job (job_id >= 0) or every submitted job (job_id = -1) has finished, or until
 * timeout_s seconds have passed (timeout_s < 0: no limit; then ETIMEOUT). */
rmhmc_status rmhmc_server_wait(rmhmc_server* s, int job_id, double timeout_s);
/* The server's clock, running and queued job counts, the most jobs ever resident at once and the
 * bytes of the budget in use; each output may be NULL. */
rmhmc_status rmhmc_server_stats(rmhmc_server* s, double* now_s, int* n_active, int* max_active,
                                int* n_queued, size_t* bytes_in_use);
/* Finish every submitted job, stop the scheduler and free the server. NULL is a no-op. */
void rmhmc_server_destroy(rmhmc_server* s);

/* Autotuner (not part of the method's arithmetic): chooses the model's Jacobi cluster size (CTAs
 * per chain: 1, 2, 4 or 8) and rotation schedule (rmhmc_jacobi_schedule) by timing generalized
 * leapfrogs (integ's eps and n_fp; integ's geometry fields must match the state's; two timed after
 * one untimed, from the model's current state) of each combination (cluster sizes whose CTAs
 * would not all be resident at two per SM are skipped), then, in the RMHMC_MIXED form, the output tile width
 * of its tensor-core GEMMs (128 x 64 or 128 x 32 tiles) with the best of those, then the first-order
 * pre-rotation on or off (rmhmc_set_prerotation), keeping the fastest at each step.
 * The state is then restored: q, p and the eigenbasis as before, the geometry re-evaluated at q
 * (U, dU and the Hessian are recomputed exactly; the basis is already converged there). Without it
 * a model uses the cyclic schedule, the largest cluster that keeps two CTAs per SM, 64-column
 * tiles and the pre-rotation. Synchronises the stream; needs a state. *cluster_out, *sched_out,
 * *tile_out and *prerot_out (each may be NULL) receive the choice. */
rmhmc_status rmhmc_autotune(rmhmc_model* m, const rmhmc_integrator* integ, int* cluster_out,
                            int* sched_out, int* tile_out, int* prerot_out);
/* Set the output tile width of the model's tensor-core GEMMs (64 or 32 columns, else EINVAL). */
rmhmc_status rmhmc_set_gemm_tile(rmhmc_model* m, int nt);
/* A new non-blocking CUDA stream on the current device (for batches of many models: each model of
 * a batch needs a stream of its own, and a framework's stream pool may hand out the same stream
 * twice), and its release (after the work on it is done). Errors: EINVAL, ECUDA. */
rmhmc_status rmhmc_stream_create(void** stream_out);
rmhmc_status rmhmc_stream_destroy(void* stream);
/* First-order pre-rotation of warm eigen-updates in the RMHMC_MIXED form (on by default; enable 0
 * or 1, else EINVAL). After a warm start M = Psi^T H Psi is diagonal up to small couplings: every
 * pair (j, l) that fails the Jacobi stopping rule gets the angle x / 2, x = 2 m_jl / (m_ll - m_jj)
 * (atan(x) / 2 to FP32 rounding), which zeroes its coupling to first order; with the skew matrix A
 * of these angles, X = I + A + A^2 / 2 + A^3 / 6 + A^4 / 24 (exp(A) to fourth order, orthogonal up
 * to A^6 / 72) is applied as M <- X^T M X and Psi <- Psi X from the lists of A's nonzeros (the
 * first- and second-order terms in double-float pairs), and the double-float Jacobi then starts
 * from the result, checks the stopping rule and rotates whatever is left. Pairs with |x| > 2e-5
 * (nearly equal diagonal entries) are left to the Jacobi; a chain takes it only when
 * ||A||_F <= 1e-3 (so that A^6 / 72 is below 1e-19); cold starts, matrices of more than 1701
 * (padded) rows and the FP64 path use the Jacobi alone. Not part of the paper's method, which this
 * accelerates: the eigen-update's result still satisfies the same stopping rule. */
rmhmc_status rmhmc_set_prerotation(rmhmc_model* m, int enable);
/* Set the Jacobi cluster size (1, 2, 4, 8, or 0 for the default) and rotation schedule directly. */
rmhmc_status rmhmc_set_jacobi(rmhmc_model* m, int cluster, int sched);

/* Kernel-level profile (for measurement; not part of the method). While enabled, every kernel
 * launch of the model is bracketed by CUDA events on the model's stream and counted in one of
 * RMHMC_PROF_NCAT categories (names from rmhmc_profile_category), with the algorithmic FLOPs of
 * the work it must do (GEMM 2mnk on the unpadded sizes, halved for symmetric outputs; for the
 * tensor-core GEMMs of the mixed form, category "gemm_tc", the bf16 tensor FLOPs executed: every
 * slice product of every 128 x 64 tile computed, padding included; Cholesky
 * and triangular inverse N^3/3; Jacobi 2 * 16^3 per 16 x 16 x 16 rotation-tile product executed,
 * tiles skipped because both rotations were the identity not counted, plus 1952 per round of 8
 * rotations applied inside a 16 x 16 sub-problem; the pre-rotation's kernels, category
 * "prerotation": 2 flops per double-float multiply-add of its first- and second-order products,
 * 24 dp per pre-rotated pair). rmhmc_profile(m, 1)
 * resets and starts, rmhmc_profile(m, 0) stops. rmhmc_profile_read synchronises the stream and
 * writes per-category milliseconds, FLOPs and launch counts (host arrays of RMHMC_PROF_NCAT). */
#define RMHMC_PROF_NCAT 11
rmhmc_status rmhmc_profile(rmhmc_model* m, int enable);
rmhmc_status rmhmc_profile_read(rmhmc_model* m, double* ms_host, double* flops_host,
                                long long* launches_host);
const char* rmhmc_profile_category(int i);
/* Work counters of the eigen-update (Sec. 2.4's Jacobi), summed over the model's chains since the
 * last rmhmc_profile(m, 1) (or model creation): counters_host[0..7] = 16 x 16 x 16 rotation-tile
 * products of phase 2, rotation rounds applied inside 16 x 16 sub-problems, outer rounds (parallel
 * steps of the block Jacobi), 16 x 16 sub-problems solved, of which rotated, eigen-updates,
 * eigen-updates that took the first-order pre-rotation, pairs it rotated.
 * Counted whether or not profiling is on (the autotuner's trial runs excepted). Synchronises the
 * stream. */
rmhmc_status rmhmc_jacobi_counters(rmhmc_model* m, long long* counters_host);

/* Measure this GPU's FP64 FMA throughput (a roofline denominator, not part of the method): runs a
 * dependent-chain DFMA kernel on every SM for about ms_target milliseconds on cuda_stream and writes
 * the achieved TFLOP/s (2 flops per FMA) to *tflops_host. Synchronises the stream. */
rmhmc_status rmhmc_fp64_peak(void* cuda_stream, int ms_target, double* tflops_host);
/* The same for FP32 FFMA. */
rmhmc_status rmhmc_fp32_peak(void* cuda_stream, int ms_target, double* tflops_host);
/* The same for the double-float multiply-add (the Dot2 step of the RMHMC_MIXED kernels: FP32
 * two-product and two-sum with a compensation word), 2 flops per step: the denominator of the
 * double-float Jacobi. */
rmhmc_status rmhmc_df_peak(void* cuda_stream, int ms_target, double* tflops_host);

/* Allocation-free eigendecomposition of a batch of symmetric matrices, for callers that cannot
 * allocate device memory (e.g. code running inside another framework's memory pool or arena, a
 * plug-in whose host forbids cudaMalloc, or a real-time loop that must not hit the allocator).
 * The paper has no counterpart: it is this library's cold-start block-Jacobi (the solver inside
 * rmhmc_set_state) with its workspace in a fixed, file-scope device array of 8 MiB
 * (1,048,576 doubles) that every GPU loading the library keeps until the process exits.
 * A_dev (n x d x d, read only) holds symmetric matrices; outputs lam_dev (n x d, eigenvalues in
 * the solver's order) and/or Q_dev (n x d x d, eigenvectors as columns, A = Q diag(lam) Q^T);
 * tol and max_sweeps as in rmhmc_integrator (jacobi_tol, max_sweeps; the RELATIVE rule, so every
 * eigenpair is resolved); sweeps_dev and status_dev
 * (n ints each, RMHMC_CHAIN_NOTCONV on failure) may be NULL. With dp = d rounded up to a multiple
 * of 16, the batch must satisfy 2 n dp^2 + n dp + 512 n dp/16 + 64 n + O(n dp/16) <= 1,048,576
 * doubles (e.g. n = 64 at d = 64, n = 1 at d = 700); larger batches return RMHMC_ESCRATCH
 * without touching the GPU. No device memory is allocated or freed by the call. The array itself
 * is committed on a device when the library's device code is loaded there, which under lazy module
 * loading (CUDA_MODULE_LOADING=LAZY, the default) can be this entry point's first call: a caller
 * budgeting memory inside an arena should make one warm-up call before taking its measure. The
 * first call on a device looks up the array's device address (cudaGetSymbolAddress, once per
 * device, safe from several host threads), so make that first call before any stream capture.
 * cuda_stream must belong to the current device (else RMHMC_EINVAL): the workspace used is the
 * current device's. All calls share the one array and it keeps the previous call's contents (every
 * value the solver reads is rewritten first); calls that overlap on the GPU, from two streams or
 * two threads, race on it and must be serialised by the caller. Enqueued on cuda_stream. */
rmhmc_status rmhmc_eigh_noalloc(void* cuda_stream, int n, int d, const double* A_dev,
                                double* lam_dev, double* Q_dev, double tol, int max_sweeps,
                                int* sweeps_dev, int* status_dev);

/* Batched FP64-accurate GEMM on the tensor cores (tcgen05, bf16 operands, FP32 accumulators in
 * tensor memory), the contraction engine of the RMHMC_MIXED path (K^-1 algebra, Psi^T H Psi and
 * Psi C Psi^T of Sec. 2.3-2.4), exposed for direct use and testing:
 *   C_b = alpha op(A_b) op(B_b) + beta C_b,  b < batch,
 * row-major; op(A) is m x k (A_dev + b strideA, A^T when ta), op(B) is k x n (B^T when tb), C is
 * m x n with leading dimension ldc. Method: error-free splitting (Ozaki, Ogita, Oishi and Rump,
 * Numer. Algorithms 59, 2012): every row of op(A) and column of op(B) is scaled by a power of two
 * and cut into `slices` bf16 numbers of 7 bits each (the first 8); the slice products whose
 * weights sum to at most slices + 1 are formed on the tensor cores with exact FP32 group sums (k is
 * processed 512 at a time), and combined in FP64. Error: about 2^(-7 slices) k max|row of op(A)|
 * max|column of op(B)| plus FP64 rounding of the result; slices = 9 (63 bits) is at or below
 * FP64 GEMM rounding, 7 about 2^-49. slices: 6..9. sym (m == n): the product is known to be
 * symmetric; only its lower triangle is computed and mirrored. A row or column holding a
 * non-finite value gives NaN in the corresponding row or column of C. Scratch of
 * about 2 (m + n) k slices bytes (rows padded to 128) is taken with cudaMallocAsync on cuda_stream
 * and released the same way; ENOMEM if that fails. status_dev (batch ints, may be NULL) receives
 * RMHMC_CHAIN_TIMEOUT for an entry whose bounded device wait gave up. Enqueued on cuda_stream. */
rmhmc_status rmhmc_gemm_tc(void* cuda_stream, int ta, int tb, int m, int n, int k, double alpha,
                           const double* A_dev, int lda, long long strideA, const double* B_dev,
                           int ldb, long long strideB, double beta, double* C_dev, int ldc,
                           long long strideC, int batch, int slices, int sym, int* status_dev);

/* Test switch of the bounded device waits (failure detection; the paper has no counterpart).
 * Every wait of the tensor-core GEMM (the pipeline's mbarriers) gives up after a time limit, marks
 * the batch entry RMHMC_CHAIN_TIMEOUT in status_dev, writes NaN for that entry and lets the kernel
 * free its tensor memory and return, so the context stays usable. To exercise that path without a
 * fault: entry >= 0 makes every later GEMM launch issue no copy for batch entry `entry` (nothing is
 * then in flight for it and its first wait runs out) and sets every wait's limit to wait_ms
 * (1..2000 ms, else RMHMC_EINVAL); entry < 0 restores normal operation (no stall, the ~2 s limit).
 * Off by default; host-side state of the process, read when a GEMM is enqueued. */
rmhmc_status rmhmc_test_gemm_stall(int entry, double wait_ms);

/* Dimension d of q, and number of chains. */
int rmhmc_dim(const rmhmc_model* m);
int rmhmc_n_chains(const rmhmc_model* m);

/* Release the model's device memory (synchronises its stream first). NULL is a no-op. */
void rmhmc_free_model(rmhmc_model* m);

/* Static string for a status code. */
const char* rmhmc_status_string(rmhmc_status s);

/* Library build identifier, e.g. "rmhmc sm_103a fp64". */
const char* rmhmc_version(void);

#ifdef __cplusplus
}
#endif
#endif /* RMHMC_H */
