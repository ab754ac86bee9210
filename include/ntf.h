/*
 * ntf.h -- C ABI of the GB300 library for ADMoM non-negative CP factorization (NTF).
 *
 * Method: Liavas & Sidiropoulos, "Parallel Algorithms for Constrained Tensor Factorization
 * via Alternating Direction Method of Multipliers" (arXiv 1409.2383).  For an N-way dense
 * tensor X (N = 3 or 4) and rank R the library computes, per factor n,
 *
 *   M_n = X^(n) (Khatri-Rao of the other factors)               Sec. IV-A item 1
 *   G_n = Hadamard product of the other factors' Grams         Sec. IV-A item 2
 *   A   = (M_n + rho At - Y) (G_n + rho I)^{-1}                 eq. (ADMM_NTF_ALS_C)
 *   At  = (A + Y / rho)_+ ,  Y = Y + rho (A - At)               eq. (ADMoM_NTF)
 *
 * the residuals of Sec. IV-C, the penalty rule of Sec. IV-D and the relative
 * factorization error of Sec. VI-A.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Layout: the tensor is row-major [I_1, ..., I_N] (last index fastest).  Every factor,
 *   auxiliary, dual and MTTKRP matrix is row-major [I_n, R] FP32.  Gram, coefficient and
 *   Cholesky matrices are row-major [R, R] FP64.
 * - Memory: pointers named d_* are device pointers owned by the caller and only borrowed
 *   for the duration of the call (the tensor: for the life of the context).  The context
 *   owns its workspace, allocated in ntf_create and freed in ntf_destroy.  Arrays of
 *   pointers (``const float* const* d_factors``) are host arrays of N device pointers.
 *   Every array pointer must be a multiple of its element size (FP32: 4, BF16: 2, FP64: 8
 *   bytes); otherwise the call returns NTF_ERR_INVALID_ARG before any launch.
 * - Streams: every call is enqueued on the stream given to ntf_create and returns without
 *   waiting, except where a host result is returned (stats, rel_err, norms), in which case
 *   the call synchronizes that stream.
 * - Errors: a status code; nothing is thrown across the ABI.  Argument errors are detected
 *   on the host before any launch (NTF_ERR_INVALID_ARG).  Numerical failures found on the
 *   device (a non-positive Cholesky pivot, a non-finite residual) are recorded in the
 *   context and returned by the next synchronizing call or by ntf_sync.  ntf_last_error()
 *   gives a message for the calling thread's most recent failure.  A context stays usable
 *   after any error.
 * - Limits: 3 <= N <= 4, 1 <= R <= 64, 1 <= I_n <= 2^30, and each half of the tensor's
 *   matrix views below 2^31 entries (ntf_create).
 */
#ifndef NTF_H
#define NTF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ntf_ctx ntf_ctx;

typedef enum {
  NTF_OK = 0,
  NTF_ERR_INVALID_ARG = 1,   /* bad size, null pointer, unknown mode            */
  NTF_ERR_CUDA = 2,          /* a CUDA runtime call failed                       */
  NTF_ERR_OOM = 3,           /* workspace allocation failed                      */
  NTF_ERR_NOT_SPD = 4,       /* Cholesky of G + rho I met a non-positive pivot   */
  NTF_ERR_NONFINITE = 5,     /* a residual norm or the fit is NaN / Inf          */
  NTF_ERR_NOT_CONVERGED = 6, /* ntf_run hit its iteration limit                  */
  NTF_ERR_TIMEOUT = 7,       /* a bounded device-side wait gave up               */
  NTF_ERR_UNSUPPORTED = 8    /* valid request this build does not implement      */
} ntf_status;

/* Storage type of the tensor; arithmetic is FP32 accumulation either way. */
typedef enum { NTF_F32 = 0, NTF_BF16 = 1 } ntf_dtype;

/* Which factors feed the Khatri-Rao products and Grams of the later updates.
 * PRIMAL: the unconstrained A^{k+1} (eq. ADMM_NTF_ALS_C as printed).
 * AUX:    the non-negative auxiliaries At^{k+1}. */
typedef enum { NTF_KR_PRIMAL = 0, NTF_KR_AUX = 1 } ntf_kr_source;

/* ADAPTIVE: rho per factor, adapted once per outer iteration by eq. (varying_penalty_rule).
 * TRACE:    rho = trace(G_n)/R, recomputed at every factor update.
 * FIXED:    rho stays at the value set by ntf_set_rho (default rho0). */
typedef enum { NTF_RHO_ADAPTIVE = 0, NTF_RHO_TRACE = 1, NTF_RHO_FIXED = 2 } ntf_rho_policy;

/* Engine of the two MTTKRP contractions.  TENSOR: tcgen05 tensor cores fed by TMA (needs
 * R <= 64 and 16-byte aligned tensor rows, else ntf_create fails with NTF_ERR_UNSUPPORTED);
 * SIMT: FP32 FMA kernels (any shape); AUTO: TENSOR where it applies, else SIMT.  Both keep
 * FP32 accuracy: the tensor-core path multiplies BF16 tensor entries by a 3-part BF16 split
 * of the Khatri-Rao operand, or FP32 entries as TF32 hi/lo pairs (three MMAs per step). */
typedef enum { NTF_CONTRACT_AUTO = 0, NTF_CONTRACT_TENSOR = 1, NTF_CONTRACT_SIMT = 2 } ntf_contraction;

typedef struct {
  int inner_iters;   /* L >= 1: update/projection/dual repetitions per factor (paper: 1) */
  int kr_source;     /* ntf_kr_source                                                    */
  int rho_policy;    /* ntf_rho_policy                                                   */
  double rho0;       /* initial penalty (paper: 1)                                       */
  double mu;         /* penalty rule parameters (paper: 8, 4, 2), Sec. VI-A               */
  double tau_incr;
  double tau_decr;
  double eps_abs;    /* stopping tolerances of Sec. IV-C (paper: 1e-4, 1e-4)            */
  double eps_rel;
  int contraction;   /* ntf_contraction (default AUTO)                                   */
  /* KKT stopping rule of ntf_run (eq. KKT_NTF; default 0 = not used): the run stops at a
   * checked iteration where every factor's last update has kkt_dual <= kkt_dual_tol and
   * kkt_comp <= kkt_comp_tol (a tolerance of 0 leaves that measure untested; see
   * ntf_update_stats for the measures). */
  double kkt_dual_tol;
  double kkt_comp_tol;
  /* Factor 0's second tree level (Sec. IV-A: the MTTKRP finished from the shared
   * contraction) formed in that contraction's epilogue instead of a separate pass over its
   * [I_1 I_2, R] intermediate; applies to the tensor-core engine with one contraction chunk,
   * R <= 32 and I_2 >= 32.  0 (default): where it applies and the intermediate is at least
   * half the L2 size; 1: wherever it applies; -1: never.  Results equal to rounding. */
  int fuse_level;
  /* Copies of the tensor kept on the device for the tensor-core engine, made once by
   * ntf_create and owned by the context (ntf_profile.tensor_copy_bytes reports their size):
   * (a) a transposed copy (X[P, Q] stored as [Q, P], rows padded to 16-byte multiples), on
   * which the second contraction X^T W (Sec. IV-A) runs as a row-major product: for FP32
   * storage the operand split then needs no transpose in shared memory; (b) a copy of the
   * first contraction's view with rows padded to 16-byte multiples, where the tensor's rows
   * are not (the tensor-memory copies need that pitch).  A 3-way tensor whose trailing extent
   * makes unaligned rows then uses the view X[I_1, I_2 I_3] for both contractions (the
   * smaller padding).  0 (default): a copy is made where it takes at most half the free
   * device memory: the padded copy and the transposed one wherever the tensor's own rows do
   * not allow the tensor-core path, and the transposed one also for FP32 storage, and for
   * BF16 storage when the product is not cut into chunks along P, the rank is 17..32 and the
   * Khatri-Rao table is streamed (P > 448): the cases where the row-major product measured
   * faster than the M-contiguous one; 1: both wherever they apply, any size; -1: never (the
   * FMA kernels take what the tensor cores cannot).  Results are equal to rounding either
   * way. */
  int tensor_copy;
} ntf_params;

/* Per-factor residuals of one update (Sec. IV-C), all Frobenius norms, and the KKT measures
 * of the factor's non-negative least-squares problem at the new auxiliary At (eq. KKT_NTF:
 * with the other factors fixed the factor solves min_{At >= 0} 1/2 ||X^(n) - At K^T||^2, whose
 * gradient is g = At G - M, G the coefficient matrix without rho and M the MTTKRP; the
 * optimality conditions are At >= 0, g >= 0, At (*) g = 0).  Scaled with s_x = max |At| and
 * s_g = max |G| s_x + max |M| (FP32 arithmetic for g, so values below about R 2^-24 are
 * rounding):
 *   kkt_neg_x = max(0, -min At) / s_x                  (0: At is projected)
 *   kkt_dual  = max(0, max(-g)) / s_g                  (dual feasibility)
 *   kkt_comp  = sum |At (*) g| / (I_n R s_x s_g)       (complementarity) */
typedef struct {
  double primal_res; /* ||A - At||                                   */
  double dual_res;   /* rho ||At_after - At_before||                 */
  double norm_A;
  double norm_At;
  double norm_Y;
  double rho;        /* penalty used by this update                  */
  double kkt_neg_x;
  double kkt_dual;
  double kkt_comp;
} ntf_update_stats;

typedef struct {
  int iters;          /* outer iterations executed                          */
  int converged;      /* 1 if the residual test held for every factor       */
  int reached_target; /* 1 if rel_err <= target_rfe was observed            */
  int kkt_met;        /* 1 if the KKT tolerances held for every factor      */
  double rel_err;     /* relative error of the auxiliaries at the end       */
  double kkt_dual;    /* largest kkt_dual over the factors of the last      */
  double kkt_comp;    /* checked iteration (likewise kkt_comp)              */
} ntf_run_stats;

/* Fill *p with the paper's settings (paper_mode != 0: L=1, PRIMAL, ADAPTIVE, rho0=1,
 * mu=8, tau=4/2, eps=1e-4) or with the fixed-penalty inner-loop form (paper_mode == 0:
 * L=5, AUX, TRACE, same stopping tolerances).  Never fails. */
void ntf_default_params(ntf_params* p, int paper_mode);

/* Create a context for a tensor of the given order, dims[order] and rank.  d_tensor
 * (dtype NTF_F32 or NTF_BF16, row-major) must stay valid and unchanged until
 * ntf_destroy.  stream: a cudaStream_t (NULL = legacy default stream).  Computes ||X||^2
 * once (synchronizes).  On failure *out is NULL.  Errors: NTF_ERR_INVALID_ARG for an order
 * outside [3, 4], a rank outside [1, 64], a dim outside [1, 2^30], an unknown dtype, a null
 * tensor or invalid params; NTF_ERR_UNSUPPORTED if a half of the tensor's matrix views
 * (I_1 I_2 and the remaining dims; for 3-way tensors also I_1 and I_2 I_3) reaches 2^31
 * entries; all of these before any CUDA call. */
ntf_status ntf_create(ntf_ctx** out, int order, const int64_t* dims, int rank, int dtype,
                      const void* d_tensor, const ntf_params* p, void* stream);

/* Free the workspace.  Accepts NULL. */
ntf_status ntf_destroy(ntf_ctx* ctx);

/* ||X||_F^2 of the tensor, FP64 accumulation (computed at creation). */
ntf_status ntf_tensor_norm2(ntf_ctx* ctx, double* out);

/* MTTKRP of Sec. IV-A item 1: d_M[I_mode, R] = X^(mode) (Khatri-Rao of d_factors[m],
 * m != mode).  Streams the tensor from device memory once.  d_factors[mode] is ignored
 * (may be NULL). */
ntf_status ntf_mttkrp(ntf_ctx* ctx, int mode, const float* const* d_factors, float* d_M);

/* Gram F^T F (FP64 accumulation) of factor d_F [I_mode, R]; stored in the context as the
 * Gram of factor `mode` (used by later ntf_system / ntf_admm_update calls) and, if d_G is
 * not NULL, also written to d_G [R, R]. */
ntf_status ntf_gram(ntf_ctx* ctx, int mode, const float* d_F, double* d_G);

/* Coefficient matrix of eq. (ADMM_NTF_ALS_C) from the stored Grams (Sec. IV-A item 2):
 * d_H = Hadamard_{m != mode} Gram_m + rho I and its lower Cholesky factor d_L (each may be
 * NULL), rho chosen by the penalty policy.  Synchronizes and reports NTF_ERR_NOT_SPD. */
ntf_status ntf_system(ntf_ctx* ctx, int mode, double* d_H, double* d_L, double* rho_out);

/* One factor update (eq. ADMM_NTF_ALS_C then eq. ADMoM_NTF, repeated inner_iters times,
 * with the coefficient matrix factored once): reads d_M and the stored Grams, updates
 * d_A (primal, output only), d_At and d_Y in place, then refreshes the stored Gram of
 * factor `mode` from the Khatri-Rao source (d_A or d_At) and, under the ADAPTIVE policy,
 * applies the penalty rule to this factor's rho.  stats (host, may be NULL): residuals of
 * Sec. IV-C; when given, the call synchronizes. */
ntf_status ntf_admm_update(ntf_ctx* ctx, int mode, const float* d_M, float* d_A, float* d_At,
                           float* d_Y, ntf_update_stats* stats);

/* Structural constraint of a factor's auxiliary (Sec. IV-E; the constraint set of the
 * projection in eq. ADMoM_NTF):
 *   NTF_CONSTRAINT_NONNEG  (default) At >= 0: the projection (.)_+ of eq. ADMoM_NTF;
 *   NTF_CONSTRAINT_BOX     lo <= At <= hi entrywise (hi may be +inf): the projection clamps;
 *   NTF_CONSTRAINT_SPARSE  At >= 0 with at most max_nonzeros nonzero entries in the whole
 *                          factor (eq. g_new_def): the projection keeps the max_nonzeros
 *                          largest positive entries of A + Y / rho (ties: lower flat index
 *                          first) and zeroes the rest.  Its inner iterations run as separate
 *                          launches (a selection over all rows per iteration).
 * Applies to the later ntf_admm_update and ntf_run calls of that factor.  The KKT measures of
 * ntf_update_stats are those of the non-negative problem whatever the constraint.  Errors:
 * NTF_ERR_INVALID_ARG for an unknown kind, lo > hi or a NaN bound, max_nonzeros < 0;
 * NTF_ERR_UNSUPPORTED for the sparsity constraint when I_mode R >= 2^32. */
typedef enum {
  NTF_CONSTRAINT_NONNEG = 0,
  NTF_CONSTRAINT_BOX = 1,
  NTF_CONSTRAINT_SPARSE = 2
} ntf_constraint;
ntf_status ntf_set_constraint(ntf_ctx* ctx, int mode, int kind, double lo, double hi,
                              int64_t max_nonzeros);

/* Penalty of factor `mode` (used by ADAPTIVE and FIXED policies). */
ntf_status ntf_set_rho(ntf_ctx* ctx, int mode, double rho);
ntf_status ntf_get_rho(ntf_ctx* ctx, int mode, double* rho);

/* Relative factorization error ||X - [F_1..F_N]||_F / ||X||_F of Sec. VI-A, evaluated as
 * sqrt(||X||^2 - 2 <M_N, F_N> + 1^T (Hadamard of all Grams) 1) / ||X|| with one MTTKRP of
 * the last factor (one tensor pass).  Does not touch the stored Grams.  Synchronizes. */
ntf_status ntf_fit(ntf_ctx* ctx, const float* const* d_factors, double* rel_err);

/* The same error by explicit reconstruction: ||X - [F_1..F_N]||_F^2 summed entry by entry
 * (FP32 model values, FP64 sums) over one tensor pass, with R multiply-adds per entry.  The
 * identity above subtracts terms of size ||X||^2, so an error e ||X||^2 of <M_N, F_N> (the FP32
 * contraction's rounding, about 1e-6 relative) moves the squared error by 2e ||X||^2: at low
 * noise (errors near 1e-3) this call is the accurate one.  Synchronizes. */
ntf_status ntf_fit_explicit(ntf_ctx* ctx, const float* const* d_factors, double* rel_err);

/* Same, from a last-factor MTTKRP the caller already has (no tensor pass).  Uses the
 * stored Grams, which must be those of d_F_last and of the factors d_M_last was formed
 * with.  Synchronizes. */
ntf_status ntf_fit_from_mttkrp(ntf_ctx* ctx, const float* d_M_last, const float* d_F_last,
                               double* rel_err);

/* Whole factorization: outer iterations of eq. (ADMoM_NTF) in Gauss-Seidel order starting
 * from the given state (d_A, d_At, d_Y: host arrays of N device pointers, updated in
 * place), until the residual test of Sec. IV-C holds for every factor (if eps_abs or
 * eps_rel > 0), rel_err <= target_rfe (if target_rfe > 0), the KKT tolerances of the params
 * hold for every factor (if kkt_dual_tol or kkt_comp_tol > 0) -- each tested every
 * check_every iterations -- or max_outer iterations.  Grams are (re)initialised from the Khatri-Rao
 * source factors first.  rfe_hist (host, may be NULL, length max_outer) receives the error
 * after every checked iteration (NaN elsewhere).  Returns NTF_ERR_NOT_CONVERGED if
 * max_outer was reached without meeting a requested criterion (out is still filled).
 * The stopping rules are evaluated on the device; the call enqueues the next iteration
 * before it reads the previous one's outcome, so one iteration more may be enqueued than
 * run: its kernels find the run stopped and leave the state as it is (the state, iteration
 * count and error are those of stopping at the first checked iteration that met a rule).
 * The call may return while that iteration's kernels still drain on the context's stream;
 * work enqueued on that stream afterwards (or ntf_sync) is ordered after them. */
ntf_status ntf_run(ntf_ctx* ctx, float* const* d_A, float* const* d_At, float* const* d_Y,
                   int max_outer, double target_rfe, int check_every, double* rfe_hist,
                   ntf_run_stats* out);

/* Device-time accounting of the two tensor contractions inside ntf_run (the dominant
 * kernels): CUDA events are recorded around each contraction launch on the context's
 * stream and read back at every check of ntf_run.  Counters restart at enable. */
typedef struct {
  int64_t sweeps;             /* outer iterations run while profiling was on            */
  int64_t kernel_launches;    /* library kernels launched by those sweeps               */
  int64_t contractions[2];    /* timed launches: [0] X * KR_right, [1] X^T * KR_left     */
  double contraction_ms[2];   /* summed device time of those launches, milliseconds     */
  double contraction_bytes[2];/* tensor bytes each such launch reads (algorithmic)      */
  int64_t ws_rows_considered; /* warm start: rows offered a prediction                  */
  int64_t ws_rows_accepted;   /* warm start: rows whose prediction the judge kept       */
  int64_t tensor_copy_bytes;  /* device bytes of the transposed tensor copy (0: none;
                               * params.tensor_copy), on which [1] then runs             */
} ntf_profile;

ntf_status ntf_profile_enable(ntf_ctx* ctx, int enable);
ntf_status ntf_profile_get(ntf_ctx* ctx, ntf_profile* out);

/* Sweep trace.  With tracing on, every step of an outer iteration (first and second
 * contraction, second tree level of each MTTKRP, warm start, rows, reductions, coefficient
 * systems) is bracketed by CUDA events on the stream that runs it, inside the recorded CUDA
 * graph as well.  ntf_trace_get (synchronizes) returns, for the last outer iteration of the
 * last ntf_run, each step's start and end in microseconds from the start of that iteration,
 * in enqueue order; *n_entries = the number of steps (at most max_entries are written).
 * stream: 0 = the context's stream, 1 = the second-contraction stream, 2 = the side stream of
 * the MTTKRP second levels and the first system.  mode: the factor the step serves. */
typedef struct {
  char name[24];
  int stream;
  int mode;
  double start_us;
  double end_us;
} ntf_trace_entry;

ntf_status ntf_trace_enable(ntf_ctx* ctx, int enable);
ntf_status ntf_trace_get(ntf_ctx* ctx, ntf_trace_entry* out, int max_entries, int* n_entries);

/* Synchronize the context's stream; return (and clear) a deferred device-side error. */
ntf_status ntf_sync(ntf_ctx* ctx);

/* Failure detection.  Every device-side wait of the library's kernels (the mbarrier rings
 * between the roles of the tensor-core contractions) is bounded: a wait that has not ended
 * after 2 s sets the timeout bit of the context's device status word; the kernel's roles then
 * leave their loops, wait (again bounded) for their copies in flight, free their tensor memory
 * and return, and the next call that reads the status (ntf_sync, ntf_run, ntf_mttkrp, ...)
 * returns NTF_ERR_TIMEOUT and clears it; the context stays usable.  ntf_watchdog_check runs
 * that bounded wait on the context's stream on an mbarrier that nothing completes, with the
 * limit limit_ms (0 < limit_ms <= 2000), and returns what ntf_sync then reports:
 * NTF_ERR_TIMEOUT when the wait gave up as it must.  A status already pending before the
 * call is returned first (and the check is not run); NTF_ERR_INVALID_ARG for a null context
 * or a limit out of range. */
ntf_status ntf_watchdog_check(ntf_ctx* ctx, double limit_ms);

/* ---------------------------------------------------------------------------------------
 * Learned warm start (not in the paper; an addition evaluated against the plain method).
 * With the other factors fixed each row of a factor solves the non-negative least squares
 * min_{x >= 0} 1/2 x^T G x - m^T x (G: coefficient matrix of eq. ADMM_NTF_ALS_C without rho,
 * m: MTTKRP row), whose solution x* and dual y* = m - G x* satisfy eq. (KKT_NTF).  The network
 * maps [vec(G/s) ; m/s ; z], s = trace(G)/R, z = (G + s I)^{-1} m (the first primal iterate of
 * the row's ADMM from zero, eq. ADMM_NTF_ALS_C), to [x* ; y* / s]: layers R^2+2R -> H -> H ->
 * 2R with the exact GELU, BF16 weights in every product (FP32 master copies, FP32
 * accumulation).  Parameters are one flat FP32 array in the order W1 [H, R^2+2R], b1 [H],
 * W2 [H, H], b2 [H], W3 [2R, H], b3 [2R] (row-major), of ntf_mlp_param_count(R, H) floats.
 * Batches: `groups` normalised coefficient matrices d_Gn [groups, R^2] (G/s), CSR offsets
 * d_offsets [groups + 1] (device ints; the rows of group g are offsets[g] .. offsets[g+1]-1)
 * and per-row inputs d_mrows [rows, 2R] ([m/s ; z]); targets [rows, 2R].  All calls run on the
 * stream given at creation.  Inside a factor update (ntf_attach_warmstart) z is formed with
 * the update's own (G + rho I)^{-1}, which is (G + s I)^{-1} under the trace penalty policy. */
typedef struct ntf_mlp ntf_mlp;

/* Number of floats in the parameter array (-1 for an invalid rank / width). */
int64_t ntf_mlp_param_count(int rank, int hidden);

/* Create a network from host parameters (copied); workspaces for up to max_rows rows and
 * max_groups coefficient matrices per call.  Adam moments start at zero. */
ntf_status ntf_mlp_create(ntf_mlp** out, int rank, int hidden, const float* h_params,
                          int max_rows, int max_groups, void* stream);
ntf_status ntf_mlp_destroy(ntf_mlp* net);

/* Copy the FP32 master parameters to host memory (synchronizes). */
ntf_status ntf_mlp_get_params(ntf_mlp* net, float* h_params);

/* d_out [rows, 2R] = network output for the batch. */
ntf_status ntf_mlp_forward(ntf_mlp* net, const float* d_Gn, const int* d_offsets, int groups,
                           const float* d_mrows, int rows, float* d_out);

/* Mean-squared-error gradient of the batch against d_targets; if apply != 0 one Adam step
 * (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr).  loss (host, may be NULL: the call
 * then does not synchronize) receives the batch loss; d_grad_out (device, may be NULL) the
 * gradient in the parameter layout. */
ntf_status ntf_mlp_train_step(ntf_mlp* net, const float* d_Gn, const int* d_offsets, int groups,
                              const float* d_mrows, const float* d_targets, int rows, float lr,
                              int apply, double* loss, float* d_grad_out);
const char* ntf_mlp_last_error(void);

/* Use `net` (same rank, max_rows >= the largest tensor extent) to warm-start factor updates:
 * before the inner iterations each row is offered the network's (max(0, x), min(0, s y))
 * and keeps it in place of the carried-over (At, Y) row only if it is better on both
 * counts -- a smaller row objective 1/2 x^T G x - m^T x (the row's share of the fit) and a
 * smaller KKT natural residual ||min(x, G x - m)||; the plain iterations then refine either
 * way.  sweeps >= 1: the network is consulted in the first `sweeps` outer iterations of
 * each ntf_run call (the cold start, where it helps); sweeps = 0: in every iteration.
 * ntf_admm_update consults it whenever attached.  net = NULL detaches.  The context does
 * not own the network. */
ntf_status ntf_attach_warmstart(ntf_ctx* ctx, ntf_mlp* net, int sweeps);

/* Training rows of the warm-start network from one factor update (the inputs the update's own
 * warm start forms): with the stored Grams and the penalty policy, the factor's coefficient
 * system is built as ntf_admm_update builds it; then, with s = trace(G)/R,
 *   d_Gn      [R, R]    = G / s                         (G: the coefficient matrix, no rho)
 *   d_mrows   [I, 2R]   = [m / s ; z],  z = (G + rho I)^{-1} m, per MTTKRP row m of d_M
 *   d_targets [I, 2R]   = [At ; Y / s]  from d_At, d_Y  (optional: NULL skips it)
 * and *s_out = s (host).  Under the trace policy rho = s, so z = (G + s I)^{-1} m, the first
 * primal iterate of the row's ADMM from zero (eq. ADMM_NTF_ALS_C).  Device arrays are
 * caller-owned, FP32 row-major; I = dims[mode].  Synchronizes; NTF_ERR_NOT_SPD if the system
 * failed. */
ntf_status ntf_warmstart_rows(ntf_ctx* ctx, int mode, const float* d_M, const float* d_At,
                              const float* d_Y, float* d_Gn, float* d_mrows, float* d_targets,
                              double* s_out);

/* MTTKRP that allocates nothing.  The paper has no counterpart: this entry point exists for
 * callers that cannot call cudaMalloc on their call path -- services that reserve all
 * device memory at start-up and treat any later allocation as a failure, or host code where
 * the device-wide synchronization an allocation may cause is not acceptable.  It computes
 * exactly what ntf_mttkrp computes (d_M[I_mode, R] = X^(mode) times the Khatri-Rao product
 * of d_factors[m], m != mode; same layouts; d_factors is a host array of `order` device
 * pointers, d_factors[mode] ignored) without a context: its scratch memory (split-K partial
 * sums and the contraction intermediate) is one static 32 MiB device array that every GPU
 * loading this library holds until the process exits.
 * - The first call on each device looks up that array's device address (cudaGetSymbolAddress
 *   with the device current) and caches it.  With CUDA's lazy module loading (the default)
 *   that lookup is also when the 32 MiB array is placed in device memory, so make the first
 *   call on each device before any stream capture and before the caller reserves the
 *   device's memory; alternatively set CUDA_MODULE_LOADING=EAGER, which places the array when
 *   the library is loaded.
 * - d_tensor, d_M and the used d_factors must be device memory of the current device (checked
 *   with cudaPointerGetAttributes before any launch: NTF_ERR_INVALID_ARG otherwise, e.g. for
 *   host memory or another device's memory).
 * - All calls on a device share the array and it keeps the last call's contents (nothing in
 *   it needs to start at zero).  Calls whose work overlaps on the GPU -- on different streams
 *   or from different threads -- race on it; serialize them.
 * - NTF_ERR_INVALID_ARG, before any launch, if an argument is invalid or if the scratch the
 *   mode needs exceeds the 32 MiB maximum: the contraction intermediate of the mode's group
 *   (I_1 I_2 R floats for modes 1-2, I_2 I_3 R floats for mode 3 of a 3-way tensor; I_1 I_2 R
 *   or I_3 I_4 R floats for a 4-way tensor) plus a Khatri-Rao table of the other group.
 *   Partial sums that would not fit beside them are avoided by not splitting the contraction.
 * - NTF_ERR_UNSUPPORTED, before any CUDA call, under the size limit of ntf_create (a half
 *   of the tensor's matrix views with 2^31 or more entries).
 * - Never calls cudaMalloc, cudaFree or any allocating routine.  Asynchronous on `stream`. */
ntf_status ntf_mttkrp_noalloc(int order, const int64_t* dims, int rank, int dtype,
                              const void* d_tensor, int mode, const float* const* d_factors,
                              float* d_M, void* stream);

/* ---------------------------------------------------------------------------------------
 * Sparse tensors (the sparse case of Sec. IV-A: with n nonzeros the MTTKRP costs 3nF flops
 * for a 3-way tensor and never forms the Khatri-Rao matrix).  A tensor given in coordinate
 * form -- d_idx [nnz, order] int32 (row-major: the order indices of each nonzero, each in
 * [0, dims[m])), d_vals [nnz] FP32, duplicates allowed (they add up) -- is laid out once by
 * ntf_sptensor_create: for every mode, the nonzeros sorted by that mode's index (a stable
 * radix sort on the device) with row offsets.  The layout is owned by the object (about
 * (order + 1) * order * 4 + 28 bytes per nonzero of device memory, allocated at creation;
 * the inputs are not referenced afterwards).  Calls run on the stream given at creation;
 * ntf_sptensor_create synchronizes it. */
typedef struct ntf_sptensor ntf_sptensor;

/* Errors: NTF_ERR_INVALID_ARG for an order outside [3, 4], a dim outside [1, 2^30], nnz
 * outside [1, 2^31), a null or misaligned pointer; NTF_ERR_OOM.  Indices outside the dims are
 * not checked (the caller's contract). */
ntf_status ntf_sptensor_create(ntf_sptensor** out, int order, const int64_t* dims, int64_t nnz,
                               const int32_t* d_idx, const float* d_vals, void* stream);
ntf_status ntf_sptensor_destroy(ntf_sptensor* sp);

/* d_M [I_mode, R] = MTTKRP of mode `mode` (FP32 products and sums, a fixed summation order):
 * row i is the sum over the nonzeros with i_mode = i of v prod_{m != mode} F_m[i_m, :]
 * (d_factors: host array of order device pointers [I_m, R], d_factors[mode] ignored).
 * Asynchronous. */
ntf_status ntf_sptensor_mttkrp(ntf_sptensor* sp, int mode, int rank,
                               const float* const* d_factors, float* d_M);
int64_t ntf_sptensor_nnz(const ntf_sptensor* sp);
const char* ntf_sptensor_last_error(void);

/* FP32 -> BF16 storage conversion (round to nearest even), n elements, on `stream`.  d_out:
 * device memory.  d_in: device memory, or page-locked host memory that the device addresses
 * directly (cudaHostAlloc / cudaMallocHost under unified addressing): the kernel then reads
 * it over the host link, so that the copy to the device and the conversion are one pass that
 * writes half the bytes. */
ntf_status ntf_to_bf16(const float* d_in, uint16_t* d_out, int64_t n, void* stream);

const char* ntf_status_string(ntf_status s);
const char* ntf_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* NTF_H */
