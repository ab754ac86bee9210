// Internal declarations of the GB300 NTF library: context, device control block, launch
// helpers.  Not part of the ABI (include/ntf.h is).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <atomic>

#include "ntf.h"

namespace ntf {

constexpr int kMaxOrder = 4;

// The persistent tensor-core contractions hold most of every SM's shared memory and run in
// the SM configuration with the largest shared-memory carve-out.  A kernel that runs beside
// them (the factor updates, reductions, coefficient systems and second tree levels of a sweep)
// asks for that configuration too, so that its CTAs can be placed on an SM next to a
// contraction CTA instead of waiting for one to exit.  Set once per kernel and device; a
// refusal only loses the hint, and its error is cleared.
template <auto kKernel>
inline void prefer_shared_carveout() {
  static std::atomic<unsigned long long> done{0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return;
  }
  const unsigned long long bit = 1ull << (dev & 63);
  if (done.load(std::memory_order_relaxed) & bit) return;
  if (cudaFuncSetAttribute(reinterpret_cast<const void*>(kKernel),
                           cudaFuncAttributePreferredSharedMemoryCarveout,
                           cudaSharedmemCarveoutMaxShared) == cudaSuccess)
    done.fetch_or(bit, std::memory_order_relaxed);
  else
    (void)cudaGetLastError();
}

// Records the calling thread's last-error message (returned by ntf_last_error) and returns s.
ntf_status record_error(ntf_status s, const char* fmt, ...);

// Entry idx of a split Khatri-Rao table of the tensor-core contractions (parts n apart):
// BF16, W = w1 + w2 + w3 with w1 = bf16(W), w2 = bf16(W - w1), w3 = bf16(W - w1 - w2) (each
// remainder exact in FP32); FP32 (TF32 operands), W = wh + wl, wh = W truncated to TF32,
// wl = W - wh (exact).
__device__ __forceinline__ void split_store(void* W, int64_t n, int64_t idx, float w,
                                            bool bf16) {
  if (bf16) {
    __nv_bfloat16* o = static_cast<__nv_bfloat16*>(W);
    const __nv_bfloat16 b1 = __float2bfloat16_rn(w);
    const float r1 = w - __bfloat162float(b1);
    const __nv_bfloat16 b2 = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(b2);
    o[idx] = b1;
    o[n + idx] = b2;
    o[2 * n + idx] = __float2bfloat16_rn(r2);
  } else {
    float* o = static_cast<float*>(W);
    const float hi = __uint_as_float(__float_as_uint(w) & 0xFFFFE000u);
    o[idx] = hi;
    o[n + idx] = w - hi;
  }
}
constexpr int kMaxRank = 64;
constexpr int kNumSM = 152;  // used only to size grids; the real count is queried at create

// A group of consecutive modes whose factors are combined into Khatri-Rao rows.  Row q of
// the group's Khatri-Rao table decomposes with the LAST mode fastest, matching the
// row-major tensor layout: q = ((i_0 * dim_1) + i_1) * dim_2 + i_2.
struct Group {
  const float* F[3];
  int dim[3];
  int n;
};

// Deferred device-side error bits.
enum : int { kStNotSpd = 1, kStNonFinite = 2, kStTimeout = 4 };

// Outcome of one sweep of ntf_run, written by the last factor's reduction into host-mapped
// memory (slot = sweep & 1), so that the host reads it without a copy on the stream.
struct SweepSnap {
  int sweep;       // sweeps finished in the run, this one included
  int status;      // kSt* bits at the end of the sweep
  int stop;        // 1: fit target reached, 2: residual criteria of Sec. IV-C met,
                   // 4: KKT tolerances of eq. (KKT_NTF) met
  int pad;
  double rel_err;
  double kkt_dual;  // largest scaled dual infeasibility over the factors of the sweep
  double kkt_comp;  // largest scaled complementarity over the factors of the sweep
};

// Small device-resident control block: penalties, residual norms and fit terms live here so
// that a whole sweep runs without host round trips.
struct Ctrl {
  double rho[kMaxOrder];          // penalty per factor (adaptive / fixed policies)
  double stats[kMaxOrder][8];     // primal, dual, |A|, |At|, |Y|, rho used, -, -
  // KKT measures of each factor's last update (eq. KKT_NTF, scaled): negativity of At, dual
  // infeasibility, complementarity; [3]: max |G| of the coefficient matrix (set by the system)
  double kkt[kMaxOrder][4];
  double fit_inner;               // <M_N, F_N>
  double fit_gram;                // 1^T (Hadamard of all Grams) 1
  double rel_err;
  double x_norm2;
  int status;                     // kSt* bits
  int bad[kMaxOrder];             // 1 if the last system of factor n was not SPD
  int pad[3];
  unsigned long long ws_rows[2];  // warm start: rows considered, rows that took the prediction
  unsigned int red_count[kMaxOrder];  // CTAs of the running rows kernel that have finished
  unsigned int sys_count;             // CTAs of the running reduce-and-system kernel finished
  // Run control (ntf_run): at a checked sweep the last factor's reduction decides whether the
  // run stops there; the rows, reductions and systems of every later sweep then return at once
  // (the host enqueues a sweep before it reads the outcome of the previous one).
  int stop;                // read by the sweep kernels
  int stop_next;           // decided by the running sweep; moved to stop by the last CTA
  int sweep;               // sweeps finished in the current run
  int use_tgt, use_res, check_every, max_outer;
  double target_rfe, eps_rel;
  double res_base[kMaxOrder];  // sqrt(I_m R) eps_abs
  double kkt_dual_tol, kkt_comp_tol;  // KKT stopping rule (0: that measure is not tested)
  int use_kkt, pad2;
};

// ------------------------------------------------------------------ kernel launchers
// mttkrp.cu
struct GemmPlan {
  int tiles;          // CTAs along the output rows (64 per tile)
  int chunks;         // CTAs along the contraction range (> 1: partial sums)
  int64_t chunk_len;  // contraction elements per chunk
  bool vec16;         // 16-byte cp.async staging possible
};

int round_rp(int R);
int64_t kr_rows_padded(int64_t K);
GemmPlan plan_gemm_n(int64_t P, int64_t Q, int dtype, const void* X, int num_sms);
GemmPlan plan_gemm_t(int64_t P, int64_t Q, int dtype, const void* X, int num_sms);
// W[K_pad, RP] = Khatri-Rao rows of the group (zero padding)
cudaError_t launch_kr_table(const Group& g, int64_t K, int R, float* W, cudaStream_t st);
// out (or partial[chunks]) [P, R] = X[P, Q] * W[Q, R]
cudaError_t launch_gemm_n(const void* X, int dtype, int64_t P, int64_t Q, int R, const float* W,
                          const GemmPlan& plan, float* out_or_partial, cudaStream_t st);
// out (or partial[chunks]) [Q, R] = X[P, Q]^T * W[P, R]
cudaError_t launch_gemm_t(const void* X, int dtype, int64_t P, int64_t Q, int R, const float* W,
                          const GemmPlan& plan, float* out_or_partial, cudaStream_t st);
// out[n] = sum_s partial[s * n + i]
// y[Q, P] = x[P, Q]^T for elements of es = 2 or 4 bytes (the transposed tensor copy), rows of
// y ldy >= P elements apart (0: P).
cudaError_t launch_transpose(const void* x, int es, int64_t P, int64_t Q, void* y,
                             cudaStream_t st, int64_t ldy = 0);
// y[P, 0..Q) = x[P, Q], rows of y ldy >= Q elements apart, the rest of each row zero (the
// padded tensor copy).
cudaError_t launch_pad_rows(const void* x, int es, int64_t P, int64_t Q, void* y, int64_t ldy,
                            cudaStream_t st);

cudaError_t launch_sum_splits(const float* partial, int splits, int64_t n, float* out,
                              cudaStream_t st);
// T[Ia, Ib, R]:  fast: out[a, r] = sum_b T[a, b, r] F[b, r];  slow: out[b, r] = sum_a T F[a, r]
cudaError_t launch_post_fast(const float* T, int64_t Ia, int64_t Ib, int R, const float* F,
                             float* out, cudaStream_t st);
int post_slow_splits(int64_t Ia, int64_t Ib, int R, int num_sms);
cudaError_t launch_post_slow(const float* T, int64_t Ia, int64_t Ib, int R, const float* F,
                             int splits, float* partial, float* out, cudaStream_t st);
// Vectorised variants (post4_ok: float4 for R % 4 == 0 and 16-byte aligned T, F, out; else
// float2 for even R <= 64 and 8-byte alignment); slow: splits of the reduced range with
// partials [splits, Ib, R] and per-b-block counters (zeroed, left zeroed)
bool post4_ok(int R, const void* T, const void* F, const void* out);
cudaError_t launch_post_fast4(const float* T, int64_t Ia, int64_t Ib, int R, const float* F,
                              float* out, cudaStream_t st);
// The last step of the second tree level formed in a GEMM-N epilogue (umma::Args::post_*):
// out[a, r] = sum over the 32-row groups g holding rows of a, in increasing g, of
// part[g][a - 32 g / Ib][r]  (Ib >= 32).
cudaError_t launch_post_part(const float* part, int64_t Ia, int64_t Ib, int R, float* out,
                             cudaStream_t st);
int post_slow4_splits(int64_t Ia, int64_t Ib, int R, int num_sms);
int64_t post_slow4_blocks(int64_t Ib, int R);
cudaError_t launch_post_slow4(const float* T, int64_t Ia, int64_t Ib, int R, const float* F,
                              int splits, float* partial, unsigned* count, float* out,
                              cudaStream_t st);
cudaError_t launch_norm2(const void* X, int dtype, int64_t n, double* partial, int blocks,
                         double* out, cudaStream_t st);
cudaError_t launch_to_bf16(const float* in, uint16_t* out, int64_t n, cudaStream_t st);

// umma_host.cu / umma_{bf16,f32}.cu: tensor-core contractions (tcgen05 + TMA).
namespace umma {
struct Args {
  int64_t M;          // output rows
  int64_t K;          // contraction length
  int64_t chunk_len;  // contraction elements per K-chunk (a multiple of 64)
  int R;              // output columns written (R <= N)
  int tiles;          // ceil(M / 128)
  int chunks;         // K-chunks (> 1: out holds chunk partial sums [chunks][M][R])
  float* out;
  int* err;           // device status word: kStTimeout is or-ed in on a timeout
  unsigned* sched;    // [2] work-item counter and finished-CTA counter (zero between launches)
  const int* skip;    // nonzero flag (read once per CTA): no work; may be null
  // GEMM-N with one K-chunk: the leading mode's second tree level formed in the epilogue.
  // Output row p = a Ib + b contributes out[p] * post_F[b] to mode a's MTTKRP row; per group
  // of 32 rows g, post_part[g][0..1][0..R) hold the sums over its rows of the first and the
  // second value of a it meets (post_Ib >= 32).  post_F null: off.
  const float* post_F;
  int64_t post_Ib;
  float* post_part;
};
}  // namespace umma

struct UmmaPlan {
  bool on = false;
  bool transposed = false;  // GEMM-T (X^T W) rather than GEMM-N (X W)
  bool f32 = false;         // FP32 storage (TF32 split) rather than BF16
  bool wres = false;        // BF16: whole split table resident in shared memory
  int N = 0;                // MMA N: R rounded up to a multiple of 16
  int splits = 0;           // parts of the W table (3 BF16 or 2 TF32)
  int grid = 0;             // persistent CTAs
  int64_t K_pad = 0;        // W table row length (multiple of 64)
  umma::Args args{};        // out and err are set at launch
  CUtensorMap tx{}, tw{};
};
// Plans the contraction of X viewed as [P, Q] (GEMM-T when transposed) with the split W table
// at Wsplit (umma_wsplit_bytes bytes); ld is the row pitch of X in elements (0: Q).  Returns
// false (plan.on = false) when the shape or alignment does not admit the tensor-core path.
bool umma_plan(UmmaPlan* plan, bool transposed, int dtype, const void* X, int64_t P, int64_t Q,
               int R, void* Wsplit, int num_sms, int64_t ld = 0);
size_t umma_wsplit_bytes(int64_t K, int R, int dtype);
cudaError_t launch_kr_split(const Group& g, const UmmaPlan& plan, int R, void* Wsplit,
                            cudaStream_t st);
// sched: 2 device counters owned by the caller, zero before the first launch (each launch
// leaves them zero); launches sharing a counter pair must not overlap
cudaError_t launch_umma(const UmmaPlan& plan, float* out, int* err, unsigned* sched,
                        const int* skip, cudaStream_t st, const float* post_F = nullptr,
                        int64_t post_Ib = 0, float* post_part = nullptr);
// The contractions' bounded mbarrier wait, on a barrier that nothing completes: ors
// kStTimeout into *err after limit_ns.
cudaError_t launch_wait_check(int* err, uint64_t limit_ns, cudaStream_t st);

// admm.cu
cudaError_t launch_gram(const float* F, int64_t I, int R, double* G, cudaStream_t st);
cudaError_t launch_system(const double* grams, int N, int mode, int R, int rho_policy,
                          Ctrl* ctrl, double* H, double* L, cudaStream_t st);
int fit_blocks(int64_t I, int R);
// relative error by explicit reconstruction into ctrl->rel_err (partial: max_blocks doubles)
cudaError_t launch_fit_explicit(const void* X, int dtype, int N, const int64_t* dims,
                                const float* const* F, int R, double* partial, int max_blocks,
                                Ctrl* ctrl, cudaStream_t st);
cudaError_t launch_fit(const float* M, const float* F, int64_t I, int R, const double* grams,
                       int N, double* partial, Ctrl* ctrl, cudaStream_t st);

// update.cu: one factor update in three launches -- system (FP64 coefficient matrix, its
// Cholesky factor and inverse), rows (the inner iterations), reduce (Gram, residuals, fit).
struct UpdateCall {
  const double* grams;
  double* sys;
  const float* M;
  float* A;
  float* At;
  float* Y;
  Ctrl* ctrl;
  double* gram_part;
  double* scal_part;
  double* gram_out;
  SweepSnap* snap;  // a sweep of ntf_run: its outcome slots (host-mapped), else null
  // the split Khatri-Rao table of the contraction that this factor alone forms (3-way
  // tensors), written by the rows kernel from the new rows; null: none
  void* wsplit;
  int64_t ws_kpad;  // table row length
  int ws_n;         // rows per part
  bool ws_bf16;
  int64_t I;
  int N, mode, R, inner, rho_policy;
  bool kr_aux, want_fit;
  double mu, tau_incr, tau_decr;
  // projection of the auxiliary (Sec. IV-E): onto the box [box_lo, box_hi] (the default
  // [0, inf) is the non-negative orthant); the at-most-c-nonzeros projection runs its inner
  // iterations in sparse_proj.cu and the rows kernel then only forms the partial sums
  // (tail_only, with the auxiliary before the update in t_before)
  float box_lo = 0.0f, box_hi = HUGE_VALF;
  bool tail_only = false;
  const float* t_before = nullptr;
};
int update_blocks(int64_t I);
int update_scalars();
size_t update_sys_bytes(int N, int R);
cudaError_t launch_update_system(const UpdateCall& u, cudaStream_t st);
cudaError_t launch_update_rows(const UpdateCall& u, cudaStream_t st);
// no-op when the rows kernel reduces its own partials (update_fused)
cudaError_t launch_update_reduce(const UpdateCall& u, cudaStream_t st);
bool update_fused(const UpdateCall& u);
// reduction of u's factor, then (in its last CTA) the coefficient system of `next`'s factor;
// only for !update_fused(u)
cudaError_t launch_update_reduce_system(const UpdateCall& u, const UpdateCall& next,
                                        cudaStream_t st);
cudaError_t launch_update(const UpdateCall& u, cudaStream_t st);

// mlp.cu: warm-start network (parameter layout, forward, backward, Adam) and its use
struct MlpShape {
  int R, H, P, Din, Dout;  // P: per-row input width (2R)
  int64_t oW1, ob1, oW2, ob2, oW3, ob3, count;  // offsets into the flat parameter array
};
MlpShape mlp_shape(int R, int H);
cudaError_t mlp_group_terms(const MlpShape& s, const __nv_bfloat16* pb, const float* Gn,
                            int groups, float* hG, cudaStream_t st);
cudaError_t mlp_forward_rows(const MlpShape& s, const float* p, const __nv_bfloat16* pb,
                             const float* hG, const int* row_group, const float* mrows, int rows,
                             float* z1, float* h1, float* z2, float* h2, float* out,
                             cudaStream_t st);
cudaError_t mlp_backward(const MlpShape& s, const __nv_bfloat16* pb, const float* Gn,
                         const int* offs, int groups, const int* all_offs, const float* mrows,
                         int rows, const float* T, const float* z1, const float* h1,
                         const float* z2, const float* h2, const float* out, float* d_out,
                         float* d_h2, float* d_h1, float* gsum, float* grad, double* loss_part,
                         double* loss, cudaStream_t st);
cudaError_t mlp_adam(const MlpShape& s, float* p, const float* grad, float* m, float* v,
                     __nv_bfloat16* pb, float lr, int step, cudaStream_t st);
cudaError_t mlp_row_groups(const int* offs, int groups, int* row_group, cudaStream_t st);
cudaError_t mlp_refresh_bf16(const MlpShape& s, const float* p, __nv_bfloat16* pb, cudaStream_t st);
cudaError_t ws_prepare(const float* G, const float* Hinv, const float* M, int R, int64_t I,
                       float* Gn, float* mrows, float* s_out, cudaStream_t st);
// out [I, 2R] = [At ; Y / s] (training targets; s read from the device)
cudaError_t ws_targets(const float* At, const float* Y, const float* s_ptr, int R, int64_t I,
                       float* out, cudaStream_t st);
cudaError_t ws_judge(const float* out, const float* G, const float* M, const float* s_ptr,
                     float* At, float* Y, int64_t I, int R, unsigned long long* counters,
                     cudaStream_t st);
// The whole warm start of a factor (inputs, network, judge) in one kernel, when the hidden
// width and shared memory allow (ws_fused_ok); the computation of ws_prepare + forward +
// ws_judge with other summation orders in the products.
bool ws_fused_ok(const MlpShape& s);
cudaError_t ws_fused(const MlpShape& s, const float* p, const __nv_bfloat16* pb, float* hG,
                     const float* G, const float* Hinv, const float* M, float* At, float* Y,
                     int64_t I, unsigned long long* counters, cudaStream_t st);
// update.cu: FP32 coefficient matrix (no rho) and FP32 (G + rho I)^{-1} of factor `mode` in
// its system slot
const float* update_sys_h32(const double* sys, int mode, int R);
const float* update_sys_hinv32(const double* sys, int mode, int R);
// FP64 (G + rho I)^{-1} of factor `mode` (written by the sweep-operator system: the policies
// other than trace, and the trace policy for small R)
const double* update_sys_hinv64(const double* sys, int mode, int R);

// sparse_proj.cu: the inner iterations of a factor update whose auxiliary is projected onto
// the non-negative matrices with at most c nonzeros (Sec. IV-E): copies At to t_before, then
// per inner iteration the primal step, the selection of the c largest entries (V [I, R] and
// sel [2] scratch) and the projection and dual step; the rows kernel then runs with tail_only
int sparse_inner_launches(int inner);
cudaError_t launch_sparse_inner(const UpdateCall& u, int64_t c, float* V, float* t_before,
                                unsigned* sel, cudaStream_t st);

// mlp_api.cu: warm start of a factor update by an attached network
cudaError_t mlp_warm_start(ntf_mlp* n, const double* sys, int mode, const float* M, float* At,
                           float* Y, int64_t I, unsigned long long* counters, cudaStream_t st);
int mlp_rank(const ntf_mlp* n);
int mlp_ws_launches(const ntf_mlp* n);  // kernels one mlp_warm_start launches
int mlp_max_rows(const ntf_mlp* n);

}  // namespace ntf
