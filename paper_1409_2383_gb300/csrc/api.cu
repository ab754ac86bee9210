// C ABI of the NTF library (include/ntf.h): context management, argument checking, the
// per-step entry points and the native outer-iteration driver.
//
// Tensor passes per outer iteration.  Factors 1..s_R are updated from one contraction
// T_R = X[P_R, Q_R] * KR(factors s_R+1..N) (P_R = I_1..I_{s_R}), the remaining factors from
// one contraction T_L = X[P_L, Q_L]^T * KR(factors 1..s_L) (s_L <= s_R); s_R = 2, s_L = 1 for
// N = 3 and s_R = s_L = 2 for N = 4, so that each Khatri-Rao operand of a 3-way tensor is a
// single factor and no contraction range needs splitting -- except for skewed 3-way shapes
// whose last extent does not give 16-byte rows (then s_R = 1 and both passes view X as
// [I_1, I_2 I_3], for the tensor cores).  Gauss-Seidel order (eq.
// ADMM_NTF_ALS_C) is respected: T_R only involves factors that are not updated before the
// factors it serves, and T_L only involves factors already updated.  So a sweep reads the
// tensor twice, whatever N is, and every M_n equals the MTTKRP of its definition up to
// summation order.
#include <cmath>
#include <cstddef>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "ntf_internal.cuh"

using ntf::Ctrl;
using ntf::GemmPlan;
using ntf::Group;

struct ntf_ctx {
  int N = 0, R = 0, dtype = 0, num_sms = 0;
  int s_R = 0, s_L = 0;           // split points of the two contractions
  int64_t dims[ntf::kMaxOrder] = {0, 0, 0, 0};
  int64_t P_R = 0, Q_R = 0, P_L = 0, Q_L = 0, numel = 0, max_dim = 0;
  const void* X = nullptr;
  cudaStream_t st = nullptr;
  ntf_params prm{};
  GemmPlan pn{}, pt{};
  ntf::UmmaPlan un{}, ut{};      // tensor-core plans of the two contractions (on: used)
  void* Xt = nullptr;            // the transposed copy of the tensor (params.tensor_copy)
  void* Xp = nullptr;            // the row-padded copy of X[P_R, Q_R] (params.tensor_copy)
  int64_t copy_bytes = 0;        // device bytes of both copies
  int post_split_left = 1, post_split_right = 1;
  int post4_split_left = 1, post4_split_right = 1;   // vectorised second level (R % 4 == 0)
  unsigned* post_count = nullptr;  // per-b-block counters of the vectorised slow level
  unsigned* umma_sched = nullptr;  // [4] work counters of the two tensor-core contractions
  int64_t post_count_right = 0;    // offset of the right group's counters
  // workspace: every device buffer below is carved from arena[0] (sized before the
  // tensor-core plans) or arena[1] (the partial sums, sized by the plans)
  void* arena[2] = {nullptr, nullptr};
  float* partial = nullptr;      // partial sums of the first contraction and of the posts
  float* partial_b = nullptr;    // partial sums of the second contraction (its own stream)
  // factor 0's second tree level formed in the first contraction's epilogue (tensor cores,
  // one K-chunk, N <= 32, s_R >= 2, I_1 >= 32): per-32-row-group sums [ceil(P_R / 32), 2, R],
  // and whether the last enqueued first contraction wrote them for the next factor-0 level
  float* fpart = nullptr;
  bool fpart_ready = false;
  float* TR = nullptr;           // [P_R, R]
  float* TL = nullptr;           // [Q_L, R]
  float* W = nullptr;            // Khatri-Rao table of the first contraction [K_pad, RP]
  float* W_b = nullptr;          // Khatri-Rao table of the second contraction
  void* Wu = nullptr;            // split Khatri-Rao tables of the tensor-core contractions
  void* Wu_b = nullptr;
  // side streams of a sweep: B runs the second contraction, C the coefficient systems
  cudaStream_t sB = nullptr, sC = nullptr;
  cudaEvent_t ev_start = nullptr, ev_tl = nullptr, ev_b = nullptr, ev_c = nullptr;
  cudaEvent_t ev_sys[ntf::kMaxOrder] = {}, ev_rows[ntf::kMaxOrder] = {},
              ev_red[ntf::kMaxOrder] = {}, ev_post[ntf::kMaxOrder] = {};
  float* Mbuf = nullptr;         // [max_dim, R]
  double* grams = nullptr;       // [N, R, R] stored Grams
  double* grams_tmp = nullptr;   // [N, R, R] for ntf_fit
  double* chol = nullptr;        // [N, R, R]
  double* sys = nullptr;         // per-factor H^{-1} (FP64, FP32) and H (FP32)
  double* gram_part = nullptr;   // [update blocks, R (R + 1) / 2] per-CTA Gram partials
  double* scal_part = nullptr;   // [update blocks, 8] per-CTA residual / fit partial sums
  double* fit_part = nullptr;    // [64]
  double* dpart = nullptr;       // [1024] misc FP64 partials
  Ctrl* d_ctrl = nullptr;
  Ctrl* h_ctrl = nullptr;        // pinned
  double x_norm2 = 0.0;
  // structural constraint of each factor's auxiliary (Sec. IV-E; ntf_set_constraint)
  int cons_kind[ntf::kMaxOrder] = {};
  float cons_lo[ntf::kMaxOrder] = {}, cons_hi[ntf::kMaxOrder] = {};
  int64_t cons_c[ntf::kMaxOrder] = {};
  float* sp_V = nullptr;         // [max_dim, R] scratch of the sparsity projection
  float* sp_tb = nullptr;        // [max_dim, R] the auxiliary before a sparse-projected update
  unsigned* sp_sel = nullptr;    // [2] its selection
  ntf_mlp* ws = nullptr;         // attached warm-start network (not owned)
  int ws_sweeps = 0;             // consult it in the first ws_sweeps iterations of a run (0: all)
  bool ws_now = true;            // whether the sweep being enqueued consults it
  // Recorded sweeps: slot 0 without, slot 1 with the warm-start network.
  struct SweepGraph {
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;          // kept for the event-node updates of a replay
    cudaGraphNode_t prof_node[2][2] = {};  // profiling event records [contraction][start, end]
    const void* key[3 * ntf::kMaxOrder] = {};
    int launches = 0;            // kernels in the recorded sweep
    bool prof = false;           // whether it holds profiling events
    bool trace = false;          // whether it holds trace events
    ntf_mlp* ws = nullptr;       // warm-start network recorded in it
  } graphs[2];
  bool swept_eagerly = false;    // one eager sweep has set every kernel attribute
  // tracing: begin/end events of every step of the last enqueued sweep
  static constexpr int kTraceMax = 48;
  bool trace = false;
  cudaEvent_t tr_origin = nullptr;
  cudaEvent_t tr_ev[2 * kTraceMax] = {};
  struct TraceInfo {
    const char* name;
    int stream, mode;
  } tr_info[kTraceMax] = {};
  int tr_n = 0;
  // profiling: events around the two contractions, one set per sweep parity (a sweep is
  // enqueued before the previous one is read back)
  bool prof = false;
  int prof_par = 0;
  cudaEvent_t ev[2][2][2] = {};  // [parity][contraction][start, end]
  bool ev_pending[2][2] = {};
  // outcome of the sweeps of ntf_run (host-mapped, two slots) and their completion events
  ntf::SweepSnap* h_snap = nullptr;
  ntf::SweepSnap* d_snap = nullptr;
  cudaEvent_t ev_sweep[2] = {};
  int64_t launches = 0;          // kernel launches enqueued (counted at enqueue time)
  ntf_profile pr{};
};

namespace {

thread_local std::string g_last_error;

ntf_status fail(ntf_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

#define NTF_CUDA(call)                                                                  \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail(e_ == cudaErrorMemoryAllocation ? NTF_ERR_OOM : NTF_ERR_CUDA,         \
                  "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

#define NTF_TRY(expr)             \
  do {                            \
    ntf_status s_ = (expr);       \
    if (s_ != NTF_OK) return s_;  \
  } while (0)

ntf_status check_mode(const ntf_ctx* c, int mode) {
  if (!c) return fail(NTF_ERR_INVALID_ARG, "null context");
  if (mode < 0 || mode >= c->N) return fail(NTF_ERR_INVALID_ARG, "mode %d out of range", mode);
  return NTF_OK;
}

// Device arrays are read with loads of their element type (at least): a pointer that is not
// a multiple of its element size is refused before any launch.
bool misaligned(const void* p, size_t elem) { return reinterpret_cast<uintptr_t>(p) % elem != 0; }

ntf_status check_params(const ntf_params* p) {
  if (!p) return fail(NTF_ERR_INVALID_ARG, "null params");
  if (p->inner_iters < 1) return fail(NTF_ERR_INVALID_ARG, "inner_iters must be >= 1");
  if (p->kr_source != NTF_KR_PRIMAL && p->kr_source != NTF_KR_AUX)
    return fail(NTF_ERR_INVALID_ARG, "unknown kr_source %d", p->kr_source);
  if (p->rho_policy < NTF_RHO_ADAPTIVE || p->rho_policy > NTF_RHO_FIXED)
    return fail(NTF_ERR_INVALID_ARG, "unknown rho_policy %d", p->rho_policy);
  if (!(p->rho0 > 0.0) || !std::isfinite(p->rho0))
    return fail(NTF_ERR_INVALID_ARG, "rho0 must be positive");
  if (p->rho_policy == NTF_RHO_ADAPTIVE &&
      (!(p->mu > 1.0) || !(p->tau_incr > 1.0) || !(p->tau_decr > 1.0)))
    return fail(NTF_ERR_INVALID_ARG, "penalty rule needs mu, tau_incr, tau_decr > 1");
  if (p->eps_abs < 0.0 || p->eps_rel < 0.0)
    return fail(NTF_ERR_INVALID_ARG, "negative stopping tolerance");
  if (p->contraction < NTF_CONTRACT_AUTO || p->contraction > NTF_CONTRACT_SIMT)
    return fail(NTF_ERR_INVALID_ARG, "unknown contraction engine %d", p->contraction);
  if (p->fuse_level < -1 || p->fuse_level > 1)
    return fail(NTF_ERR_INVALID_ARG, "fuse_level must be -1, 0 or 1, not %d", p->fuse_level);
  if (p->tensor_copy < -1 || p->tensor_copy > 1)
    return fail(NTF_ERR_INVALID_ARG, "tensor_copy must be -1, 0 or 1, not %d", p->tensor_copy);
  if (!(p->kkt_dual_tol >= 0.0) || !(p->kkt_comp_tol >= 0.0))
    return fail(NTF_ERR_INVALID_ARG, "negative KKT tolerance");
  return NTF_OK;
}

Group make_group(const ntf_ctx* c, int first, int count, const float* const* F) {
  Group g{};
  g.n = count;
  for (int j = 0; j < count; ++j) {
    g.F[j] = F[first + j];
    g.dim[j] = static_cast<int>(c->dims[first + j]);
  }
  return g;
}

ntf_status read_ctrl(ntf_ctx* c) {
  NTF_CUDA(cudaMemcpyAsync(c->h_ctrl, c->d_ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, c->st));
  NTF_CUDA(cudaStreamSynchronize(c->st));
  return NTF_OK;
}

// Return and clear the deferred device status (h_ctrl must be fresh).
ntf_status take_status(ntf_ctx* c) {
  const int st = c->h_ctrl->status;
  if (!st) return NTF_OK;
  c->h_ctrl->status = 0;
  NTF_CUDA(cudaMemsetAsync(&c->d_ctrl->status, 0, sizeof(int), c->st));
  if (st & ntf::kStNotSpd)
    return fail(NTF_ERR_NOT_SPD, "Cholesky of G + rho I met a non-positive pivot");
  if (st & ntf::kStNonFinite) return fail(NTF_ERR_NONFINITE, "non-finite residual or fit");
  return fail(NTF_ERR_TIMEOUT, "device-side wait gave up");
}

// Events around contraction k when profiling (recorded into the graph when capturing).
// While the stream is being captured the record must become a graph node of its own
// (external event record), so that every replay records the event.
ntf_status prof_mark(ntf_ctx* c, int k, int which, cudaStream_t st) {
  if (!c->prof) return NTF_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  NTF_CUDA(cudaStreamIsCapturing(st, &cs));
  if (cs == cudaStreamCaptureStatusActive)
    NTF_CUDA(cudaEventRecordWithFlags(c->ev[c->prof_par][k][which], st, cudaEventRecordExternal));
  else
    NTF_CUDA(cudaEventRecord(c->ev[c->prof_par][k][which], st));
  if (which == 1) c->ev_pending[c->prof_par][k] = true;
  return NTF_OK;
}

// Record event `ev` on `st` (as a graph node of its own while the stream is captured).
ntf_status record_any(cudaEvent_t ev, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  NTF_CUDA(cudaStreamIsCapturing(st, &cs));
  if (cs == cudaStreamCaptureStatusActive)
    NTF_CUDA(cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal));
  else
    NTF_CUDA(cudaEventRecord(ev, st));
  return NTF_OK;
}

// Trace step bracket: returns the slot (or -1 when not tracing).
int trace_begin(ntf_ctx* c, const char* name, int mode, int sid, cudaStream_t st) {
  if (!c->trace || c->tr_n >= ntf_ctx::kTraceMax) return -1;
  const int i = c->tr_n++;
  c->tr_info[i] = {name, sid, mode};
  if (record_any(c->tr_ev[2 * i], st) != NTF_OK) return -1;
  return i;
}
ntf_status trace_end(ntf_ctx* c, int i, cudaStream_t st) {
  if (i < 0) return NTF_OK;
  return record_any(c->tr_ev[2 * i + 1], st);
}

// T_R[P_R, R] = X[P_R, Q_R] * KR(factors s_R..N-1), on stream st (table_ready: the split
// table was written by the last factor's rows kernel)
ntf_status contract_right(ntf_ctx* c, const float* const* F, float* dst, cudaStream_t st,
                          bool table_ready = false, bool fuse0 = false) {
  const Group g = make_group(c, c->s_R, c->N - c->s_R, F);
  c->fpart_ready = false;
  if (c->un.on) {
    if (!table_ready) {
      NTF_CUDA(ntf::launch_kr_split(g, c->un, c->R, c->Wu, st));
      c->launches += 1;
    }
    const int chunks = c->un.args.chunks;
    float* out = chunks > 1 ? c->partial : dst;
    NTF_TRY(prof_mark(c, 0, 0, st));
    // factor 0's second tree level in the epilogue when factor 0's MTTKRP follows
    const bool fz = fuse0 && c->fpart != nullptr;
    NTF_CUDA(ntf::launch_umma(c->un, out, &c->d_ctrl->status, c->umma_sched, &c->d_ctrl->stop,
                              st, fz ? F[1] : nullptr, fz ? c->dims[1] : 0,
                              fz ? c->fpart : nullptr));
    c->fpart_ready = fz;
    NTF_TRY(prof_mark(c, 0, 1, st));
    c->launches += 1;
    if (chunks > 1) {
      NTF_CUDA(ntf::launch_sum_splits(c->partial, chunks, c->P_R * c->R, dst, st));
      c->launches += 1;
    }
    return NTF_OK;
  }
  NTF_CUDA(ntf::launch_kr_table(g, c->Q_R, c->R, c->W, st));
  float* out = c->pn.chunks > 1 ? c->partial : dst;
  NTF_TRY(prof_mark(c, 0, 0, st));
  NTF_CUDA(ntf::launch_gemm_n(c->X, c->dtype, c->P_R, c->Q_R, c->R, c->W, c->pn, out, st));
  NTF_TRY(prof_mark(c, 0, 1, st));
  c->launches += 2;
  if (c->pn.chunks > 1) {
    NTF_CUDA(ntf::launch_sum_splits(c->partial, c->pn.chunks, c->P_R * c->R, dst, st));
    c->launches += 1;
  }
  return NTF_OK;
}

// T_L[Q_L, R] = X[P_L, Q_L]^T * KR(factors 0..s_L-1), on stream st (table_ready: the split
// table was written by factor 0's rows kernel)
ntf_status contract_left(ntf_ctx* c, const float* const* F, float* dst, cudaStream_t st,
                         bool table_ready = false) {
  const Group g = make_group(c, 0, c->s_L, F);
  if (c->ut.on) {
    if (!table_ready) {
      NTF_CUDA(ntf::launch_kr_split(g, c->ut, c->R, c->Wu_b, st));
      c->launches += 1;
    }
    const int chunks = c->ut.args.chunks;
    float* out = chunks > 1 ? c->partial_b : dst;
    NTF_TRY(prof_mark(c, 1, 0, st));
    NTF_CUDA(ntf::launch_umma(c->ut, out, &c->d_ctrl->status, c->umma_sched + 2,
                              &c->d_ctrl->stop, st));
    NTF_TRY(prof_mark(c, 1, 1, st));
    c->launches += 1;
    if (chunks > 1) {
      NTF_CUDA(ntf::launch_sum_splits(c->partial_b, chunks, c->Q_L * c->R, dst, st));
      c->launches += 1;
    }
    return NTF_OK;
  }
  NTF_CUDA(ntf::launch_kr_table(g, c->P_L, c->R, c->W_b, st));
  float* out = c->pt.chunks > 1 ? c->partial_b : dst;
  NTF_TRY(prof_mark(c, 1, 0, st));
  NTF_CUDA(ntf::launch_gemm_t(c->X, c->dtype, c->P_L, c->Q_L, c->R, c->W_b, c->pt, out, st));
  NTF_TRY(prof_mark(c, 1, 1, st));
  c->launches += 2;
  if (c->pt.chunks > 1) {
    NTF_CUDA(ntf::launch_sum_splits(c->partial_b, c->pt.chunks, c->Q_L * c->R, dst, st));
    c->launches += 1;
  }
  return NTF_OK;
}

// After a host synchronisation: add the device time of the last recorded contractions.
// (par: the parity set of a sweep that has completed; -1: both sets, after a full sync)
void prof_collect(ntf_ctx* c, int par = -1) {
  if (!c->prof) return;
  for (int q = 0; q < 2; ++q) {
    if (par >= 0 && q != par) continue;
    for (int k = 0; k < 2; ++k) {
      if (!c->ev_pending[q][k]) continue;
      c->ev_pending[q][k] = false;
      float ms = 0.0f;
      if (cudaEventElapsedTime(&ms, c->ev[q][k][0], c->ev[q][k][1]) == cudaSuccess) {
        c->pr.contractions[k] += 1;
        c->pr.contraction_ms[k] += ms;
      } else {
        (void)cudaGetLastError();  // not recorded: leave no stale error behind
      }
    }
  }
}

// Second tree level: M of `mode` from the group's contraction T (group of 1 or 2 modes).
ntf_status finish_mode(ntf_ctx* c, int mode, const float* T, const float* const* F, float* M,
                       cudaStream_t st) {
  const bool left = mode < c->s_R;
  const int first = left ? 0 : c->s_L;
  const int count = left ? c->s_R : c->N - c->s_L;
  if (count == 1) {
    if (T != M)
      NTF_CUDA(cudaMemcpyAsync(M, T, c->dims[mode] * c->R * sizeof(float),
                               cudaMemcpyDeviceToDevice, st));
    return NTF_OK;
  }
  const int64_t Ia = c->dims[first], Ib = c->dims[first + 1];
  if (mode == first && left && c->fpart_ready) {
    // the contraction's epilogue formed the group sums: only their sum per row remains
    NTF_CUDA(ntf::launch_post_part(c->fpart, Ia, Ib, c->R, M, st));
    c->fpart_ready = false;
    c->launches += 1;
  } else if (mode == first) {
    if (ntf::post4_ok(c->R, T, F[first + 1], M))
      NTF_CUDA(ntf::launch_post_fast4(T, Ia, Ib, c->R, F[first + 1], M, st));
    else
      NTF_CUDA(ntf::launch_post_fast(T, Ia, Ib, c->R, F[first + 1], M, st));
    c->launches += 1;
  } else if (ntf::post4_ok(c->R, T, F[first], M)) {
    const int sp = left ? c->post4_split_left : c->post4_split_right;
    NTF_CUDA(ntf::launch_post_slow4(T, Ia, Ib, c->R, F[first], sp, c->partial,
                                    c->post_count + (left ? 0 : c->post_count_right), M, st));
    c->launches += 1;
  } else {
    const int sp = left ? c->post_split_left : c->post_split_right;
    NTF_CUDA(ntf::launch_post_slow(T, Ia, Ib, c->R, F[first], sp, c->partial, M, st));
    c->launches += sp > 1 ? 2 : 1;
  }
  return NTF_OK;
}

ntf::UpdateCall make_call(ntf_ctx* c, int mode, const float* M, float* A, float* At, float* Y,
                          bool want_fit) {
  ntf::UpdateCall u{};
  const int R = c->R;
  u.grams = c->grams;
  u.sys = c->sys;
  u.M = M;
  u.A = A;
  u.At = At;
  u.Y = Y;
  u.ctrl = c->d_ctrl;
  u.gram_part = c->gram_part;
  u.scal_part = c->scal_part;
  u.gram_out = c->grams + static_cast<int64_t>(mode) * R * R;
  u.I = c->dims[mode];
  u.N = c->N;
  u.mode = mode;
  u.R = R;
  u.inner = c->prm.inner_iters;
  u.rho_policy = c->prm.rho_policy;
  u.kr_aux = c->prm.kr_source == NTF_KR_AUX;
  u.want_fit = want_fit;
  u.mu = c->prm.mu;
  u.tau_incr = c->prm.tau_incr;
  u.tau_decr = c->prm.tau_decr;
  u.box_lo = c->cons_lo[mode];
  u.box_hi = c->cons_hi[mode];
  return u;
}

// The rows of a factor update (the inner iterations and the update's partial sums); under
// the sparsity constraint the inner iterations run as separate launches first.
ntf_status launch_rows(ntf_ctx* c, const ntf::UpdateCall& u, cudaStream_t st) {
  if (c->cons_kind[u.mode] == NTF_CONSTRAINT_SPARSE) {
    NTF_CUDA(ntf::launch_sparse_inner(u, c->cons_c[u.mode], c->sp_V, c->sp_tb, c->sp_sel, st));
    c->launches += ntf::sparse_inner_launches(u.inner);
    ntf::UpdateCall t = u;
    t.tail_only = true;
    t.t_before = c->sp_tb;
    NTF_CUDA(ntf::launch_update_rows(t, st));
    return NTF_OK;
  }
  NTF_CUDA(ntf::launch_update_rows(u, st));
  return NTF_OK;
}

ntf_status warm_start(ntf_ctx* c, int mode, const float* M, float* At, float* Y,
                      cudaStream_t st) {
  if (!c->ws || !c->ws_now) return NTF_OK;
  NTF_CUDA(ntf::mlp_warm_start(c->ws, c->sys, mode, M, At, Y, c->dims[mode],
                               c->d_ctrl->ws_rows, st));
  c->launches += ntf::mlp_ws_launches(c->ws);
  return NTF_OK;
}

ntf_status enqueue_update(ntf_ctx* c, int mode, const float* M, float* A, float* At, float* Y,
                          bool want_fit) {
  const ntf::UpdateCall u = make_call(c, mode, M, A, At, Y, want_fit);
  NTF_CUDA(ntf::launch_update_system(u, c->st));
  NTF_TRY(warm_start(c, mode, M, At, Y, c->st));
  NTF_TRY(launch_rows(c, u, c->st));
  NTF_CUDA(ntf::launch_update_reduce(u, c->st));
  c->launches += ntf::update_fused(u) ? 2 : 3;
  return NTF_OK;
}

// Factor 0's MTTKRP: the first contraction (T_R) and its second tree level, on stream st.
ntf_status enqueue_lead(ntf_ctx* c, const float* const* src, cudaStream_t st, int sid,
                        bool table_ready = false) {
  const float* T = c->s_R == 1 ? c->Mbuf : c->TR;
  int t = trace_begin(c, "contract_right", 0, sid, st);
  NTF_TRY(contract_right(c, src, const_cast<float*>(T), st, table_ready, true));
  NTF_TRY(trace_end(c, t, st));
  t = trace_begin(c, "mttkrp_level2", 0, sid, st);
  NTF_TRY(finish_mode(c, 0, T, src, c->Mbuf, st));
  NTF_TRY(trace_end(c, t, st));
  return NTF_OK;
}

// What every sweep expects at its start: factor 0's coefficient system and MTTKRP (the system
// on the side stream next to the contraction).  Each sweep leaves the same for the next one.
ntf_status enqueue_prologue(ntf_ctx* c, float* const* A, float* const* At, float* const* Y) {
  const float* const* src = c->prm.kr_source == NTF_KR_AUX ? At : A;
  cudaStream_t sa = c->st, sc = c->sC;
  NTF_CUDA(cudaEventRecord(c->ev_start, sa));
  NTF_CUDA(cudaStreamWaitEvent(sc, c->ev_start, 0));
  NTF_CUDA(ntf::launch_update_system(make_call(c, 0, c->Mbuf, A[0], At[0], Y[0], false), sc));
  NTF_CUDA(cudaEventRecord(c->ev_sys[0], sc));
  c->launches += 1;
  NTF_TRY(enqueue_lead(c, src, sa, 0));
  NTF_CUDA(cudaStreamWaitEvent(sa, c->ev_sys[0], 0));
  return NTF_OK;
}

// One outer iteration in Gauss-Seidel order with two tensor passes, from factor 0's system
// and MTTKRP (left by the prologue or the previous sweep).  Three streams: the main stream A
// runs every factor's rows, reductions and coefficient systems; B runs the second
// contraction as soon as the factors it needs are updated and, after the last factor's rows,
// the next sweep's first contraction and factor 0's MTTKRP; C forms the next factor's MTTKRP
// from its contraction (second tree level) while A reduces the current factor's update and,
// in the same kernel, builds the next factor's coefficient system (after the last factor:
// factor 0's, for the next sweep).  The last factor's update also forms the fit terms.
ntf_status enqueue_sweep(ntf_ctx* c, float* const* A, float* const* At, float* const* Y) {
  const float* const* src = c->prm.kr_source == NTF_KR_AUX ? At : A;
  cudaStream_t sa = c->st, sb = c->sB, sc = c->sC;
  c->tr_n = 0;
  if (c->trace) NTF_TRY(record_any(c->tr_origin, sa));
  NTF_CUDA(cudaEventRecord(c->ev_start, sa));
  NTF_CUDA(cudaStreamWaitEvent(sb, c->ev_start, 0));
  NTF_CUDA(cudaStreamWaitEvent(sc, c->ev_start, 0));
  const float* T = c->s_R == 1 ? c->Mbuf : c->TR;
  int t = -1;
  for (int m = 0; m < c->N; ++m) {
    ntf::UpdateCall u = make_call(c, m, c->Mbuf, A[m], At[m], Y[m], m == c->N - 1);
    if (m + 1 == c->N) u.snap = c->d_snap;     // the sweep's outcome and stopping decision
    // A contraction whose Khatri-Rao operand is this factor alone (3-way tensors: the second
    // contraction after factor 0, the next sweep's first after the last factor) takes its
    // split table from this factor's rows kernel instead of a separate launch.
    const ntf::UmmaPlan* tp = m == 0 && c->s_L == 1 && c->ut.on ? &c->ut
                              : m + 1 == c->N && c->N - c->s_R == 1 && c->un.on ? &c->un
                                                                                : nullptr;
    if (tp) {
      u.wsplit = tp == &c->ut ? c->Wu_b : c->Wu;
      u.ws_kpad = tp->K_pad;
      u.ws_n = tp->N;
      u.ws_bf16 = !tp->f32;
    }
    const bool fused = ntf::update_fused(u);  // the rows kernel reduces by itself
    if (m > 0) NTF_CUDA(cudaStreamWaitEvent(sa, c->ev_post[m], 0));
    if (c->ws && c->ws_now) {
      t = trace_begin(c, "warm_start", m, 0, sa);
      NTF_TRY(warm_start(c, m, c->Mbuf, At[m], Y[m], sa));
      NTF_TRY(trace_end(c, t, sa));
    }
    t = trace_begin(c, "rows", m, 0, sa);
    NTF_TRY(launch_rows(c, u, sa));
    NTF_TRY(trace_end(c, t, sa));
    NTF_CUDA(cudaEventRecord(c->ev_rows[m], sa));
    c->launches += 1;
    if (m == c->s_L - 1) {
      // B: the second contraction, as soon as factors 0..s_L-1 are updated (enqueued before
      // any stream waits for it in this sweep)
      NTF_CUDA(cudaStreamWaitEvent(sb, c->ev_rows[m], 0));
      t = trace_begin(c, "contract_left", c->s_R, 1, sb);
      NTF_TRY(contract_left(c, src, c->TL, sb, m == 0 && c->s_L == 1 && c->ut.on));
      NTF_TRY(trace_end(c, t, sb));
      NTF_CUDA(cudaEventRecord(c->ev_tl, sb));
    }
    if (m + 1 == c->N) {
      // B: the next sweep's factor-0 MTTKRP (needs the last factor updated; T_R and the
      // MTTKRP buffer are free once this factor's rows have run)
      NTF_CUDA(cudaStreamWaitEvent(sb, c->ev_rows[m], 0));
      NTF_TRY(enqueue_lead(c, src, sb, 1, c->N - c->s_R == 1 && c->un.on));
    }
    // A: this factor's reduction, then the next factor's coefficient system (after the last
    // factor, factor 0's for the next sweep)
    const int n = m + 1 < c->N ? m + 1 : 0;
    const ntf::UpdateCall un = make_call(c, n, c->Mbuf, A[n], At[n], Y[n], false);
    t = trace_begin(c, fused ? "system" : "reduce+system", n, 0, sa);
    if (fused) NTF_CUDA(ntf::launch_update_system(un, sa));
    else NTF_CUDA(ntf::launch_update_reduce_system(u, un, sa));
    NTF_TRY(trace_end(c, t, sa));
    c->launches += 1;
    if (m + 1 < c->N) {
      // C: the next factor's MTTKRP, next to A's reduction (needs factor m updated; the right
      // group needs T_L, enqueued above in this or an earlier iteration of this sweep)
      NTF_CUDA(cudaStreamWaitEvent(sc, c->ev_rows[m], 0));
      if (n >= c->s_R) NTF_CUDA(cudaStreamWaitEvent(sc, c->ev_tl, 0));
      t = trace_begin(c, "mttkrp_level2", n, 2, sc);
      NTF_TRY(finish_mode(c, n, n < c->s_R ? T : c->TL, src, c->Mbuf, sc));
      NTF_TRY(trace_end(c, t, sc));
      NTF_CUDA(cudaEventRecord(c->ev_post[n], sc));
    }
  }
  NTF_CUDA(cudaEventRecord(c->ev_b, sb));
  NTF_CUDA(cudaEventRecord(c->ev_c, sc));
  NTF_CUDA(cudaStreamWaitEvent(sa, c->ev_b, 0));
  NTF_CUDA(cudaStreamWaitEvent(sa, c->ev_c, 0));
  return NTF_OK;
}

// Page-locked, device-mapped control blocks (the host mirror of Ctrl followed by the two
// sweep-outcome slots): allocating and freeing page-locked memory is slow, so blocks of
// destroyed contexts are kept for the next ones (portable: a context on another device of
// the process may take a block over).
constexpr size_t kPinnedBytes =
    ((sizeof(Ctrl) + 63) / 64) * 64 + 2 * sizeof(ntf::SweepSnap);
std::mutex g_pinned_mu;
std::vector<void*> g_pinned_free;

cudaError_t pinned_acquire(void** p) {
  {
    std::lock_guard<std::mutex> lock(g_pinned_mu);
    if (!g_pinned_free.empty()) {
      *p = g_pinned_free.back();
      g_pinned_free.pop_back();
      return cudaSuccess;
    }
  }
  return cudaHostAlloc(p, kPinnedBytes, cudaHostAllocMapped | cudaHostAllocPortable);
}
void pinned_release(void* p) {
  std::lock_guard<std::mutex> lock(g_pinned_mu);
  g_pinned_free.push_back(p);
}

// Offsets of the buffers carved from one arena (256-byte aligned).
struct Carver {
  size_t off = 0;
  size_t take(size_t bytes) {
    const size_t o = off;
    off += (std::max<size_t>(bytes, 16) + 255) / 256 * 256;
    return o;
  }
};

// The profiling event records of a recorded sweep, so that each replay can be given the
// event set of its parity.
ntf_status find_prof_nodes(ntf_ctx* c, cudaGraph_t gr, ntf_ctx::SweepGraph& g) {
  for (auto& k : g.prof_node) k[0] = k[1] = nullptr;
  if (!c->prof) return NTF_OK;
  size_t n = 0;
  NTF_CUDA(cudaGraphGetNodes(gr, nullptr, &n));
  std::vector<cudaGraphNode_t> nodes(n);
  NTF_CUDA(cudaGraphGetNodes(gr, nodes.data(), &n));
  for (cudaGraphNode_t nd : nodes) {
    cudaGraphNodeType t;
    NTF_CUDA(cudaGraphNodeGetType(nd, &t));
    if (t != cudaGraphNodeTypeEventRecord) continue;
    cudaEvent_t e = nullptr;
    NTF_CUDA(cudaGraphEventRecordNodeGetEvent(nd, &e));
    for (int k = 0; k < 2; ++k)
      for (int w = 0; w < 2; ++w)
        if (e == c->ev[c->prof_par][k][w]) g.prof_node[k][w] = nd;
  }
  return NTF_OK;
}

// Replay a recorded sweep on the context's stream (profiling events of parity c->prof_par).
ntf_status launch_graph(ntf_ctx* c, ntf_ctx::SweepGraph& g) {
  if (g.prof)
    for (int k = 0; k < 2; ++k) {
      for (int w = 0; w < 2; ++w)
        if (g.prof_node[k][w])
          NTF_CUDA(cudaGraphExecEventRecordNodeSetEvent(g.exec, g.prof_node[k][w],
                                                        c->ev[c->prof_par][k][w]));
      if (g.prof_node[k][1]) c->ev_pending[c->prof_par][k] = true;
    }
  NTF_CUDA(cudaGraphLaunch(g.exec, c->st));
  c->launches += g.launches;
  return NTF_OK;
}

void free_ctx(ntf_ctx* c) {
  if (!c) return;
  for (auto& g : c->graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
  }
  for (cudaEvent_t e : {c->ev_start, c->ev_tl, c->ev_b, c->ev_c})
    if (e) cudaEventDestroy(e);
  for (int m = 0; m < ntf::kMaxOrder; ++m)
    for (cudaEvent_t e : {c->ev_sys[m], c->ev_rows[m], c->ev_red[m], c->ev_post[m]})
      if (e) cudaEventDestroy(e);
  if (c->sB) cudaStreamDestroy(c->sB);
  if (c->sC) cudaStreamDestroy(c->sC);
  for (auto& set : c->ev)
    for (auto& pair : set)
      for (auto& e : pair)
        if (e) cudaEventDestroy(e);
  if (c->tr_origin) cudaEventDestroy(c->tr_origin);
  for (cudaEvent_t e : c->tr_ev)
    if (e) cudaEventDestroy(e);
  cudaFree(c->arena[0]);
  cudaFree(c->arena[1]);
  cudaFree(c->Xt);
  cudaFree(c->Xp);
  if (c->h_ctrl) pinned_release(c->h_ctrl);
  for (cudaEvent_t e : c->ev_sweep)
    if (e) cudaEventDestroy(e);
  delete c;
}

}  // namespace

ntf_status ntf::record_error(ntf_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

extern "C" {

void ntf_default_params(ntf_params* p, int paper_mode) {
  if (!p) return;
  p->inner_iters = paper_mode ? 1 : 5;
  p->kr_source = paper_mode ? NTF_KR_PRIMAL : NTF_KR_AUX;
  p->rho_policy = paper_mode ? NTF_RHO_ADAPTIVE : NTF_RHO_TRACE;
  p->rho0 = 1.0;
  p->mu = 8.0;
  p->tau_incr = 4.0;
  p->tau_decr = 2.0;
  p->eps_abs = 1e-4;
  p->eps_rel = 1e-4;
  p->contraction = NTF_CONTRACT_AUTO;
  p->kkt_dual_tol = 0.0;
  p->kkt_comp_tol = 0.0;
  p->fuse_level = 0;
  p->tensor_copy = 0;
}

const char* ntf_status_string(ntf_status s) {
  switch (s) {
    case NTF_OK: return "ok";
    case NTF_ERR_INVALID_ARG: return "invalid argument";
    case NTF_ERR_CUDA: return "CUDA error";
    case NTF_ERR_OOM: return "out of device memory";
    case NTF_ERR_NOT_SPD: return "coefficient matrix not positive definite";
    case NTF_ERR_NONFINITE: return "non-finite value";
    case NTF_ERR_NOT_CONVERGED: return "not converged";
    case NTF_ERR_TIMEOUT: return "device wait timed out";
    case NTF_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

const char* ntf_last_error(void) { return g_last_error.c_str(); }

ntf_status ntf_create(ntf_ctx** out, int order, const int64_t* dims, int rank, int dtype,
                      const void* d_tensor, const ntf_params* p, void* stream) {
  if (!out) return fail(NTF_ERR_INVALID_ARG, "null output pointer");
  *out = nullptr;
  if (order < 3 || order > ntf::kMaxOrder)
    return fail(NTF_ERR_INVALID_ARG, "order %d not in [3, %d]", order, ntf::kMaxOrder);
  if (!dims) return fail(NTF_ERR_INVALID_ARG, "null dims");
  if (rank < 1 || rank > ntf::kMaxRank)
    return fail(NTF_ERR_INVALID_ARG, "rank %d not in [1, %d]", rank, ntf::kMaxRank);
  if (dtype != NTF_F32 && dtype != NTF_BF16) return fail(NTF_ERR_INVALID_ARG, "unknown dtype");
  if (!d_tensor) return fail(NTF_ERR_INVALID_ARG, "null tensor");
  if (misaligned(d_tensor, dtype == NTF_BF16 ? 2 : 4))
    return fail(NTF_ERR_INVALID_ARG, "tensor pointer not aligned to its element size");
  NTF_TRY(check_params(p));
  for (int m = 0; m < order; ++m)
    if (dims[m] < 1 || dims[m] > (int64_t{1} << 30))
      return fail(NTF_ERR_INVALID_ARG, "dims[%d] = %lld out of range", m, (long long)dims[m]);

  ntf_ctx* c = new ntf_ctx();
  c->N = order;
  c->R = rank;
  c->dtype = dtype;
  c->X = d_tensor;
  c->st = static_cast<cudaStream_t>(stream);
  c->prm = *p;
  c->s_R = 2;
  c->s_L = order == 3 ? 1 : 2;
  // each half is a product of at most two dims (<= 2^60), so nothing here overflows; the
  // tensor's size is formed only once both halves are known to be below 2^31 (checked on both
  // matrix views, whichever split the passes use)
  c->P_R = c->P_L = c->Q_R = c->Q_L = 1;
  for (int m = 0; m < order; ++m) {
    c->dims[m] = dims[m];
    c->max_dim = std::max(c->max_dim, dims[m]);
    (m < c->s_R ? c->P_R : c->Q_R) *= dims[m];
    (m < c->s_L ? c->P_L : c->Q_L) *= dims[m];
  }
  if (c->P_R >= (int64_t{1} << 31) || c->Q_R >= (int64_t{1} << 31) ||
      c->P_L >= (int64_t{1} << 31) || c->Q_L >= (int64_t{1} << 31)) {
    delete c;
    return fail(NTF_ERR_UNSUPPORTED, "tensor halves must each have < 2^31 entries");
  }
  // Skewed 3-way shapes (the paper's I x 50 x 50): when the rows of X[I_1 I_2, I_3] are not
  // 16-byte multiples (TMA needs that pitch), both passes use the second view (s_R = 1: factor
  // 1 from X[I_1, I_2 I_3] KR(factors 2, 3), the others from its transpose as before): its
  // rows are 16-byte multiples, or, when they are not either, a row-padded copy of it wastes
  // a smaller fraction than one of X[I_1 I_2, I_3] (params.tensor_copy), so that both
  // contractions run on the tensor cores.
  if (order == 3 && p->contraction != NTF_CONTRACT_SIMT) {
    const int64_t es = dtype == NTF_BF16 ? 2 : 4;
    const bool last_ok = (dims[2] * es) % 16 == 0, pair_ok = (dims[1] * dims[2] * es) % 16 == 0;
    if (!last_ok && (pair_ok || p->tensor_copy != -1)) {
      c->s_R = 1;
      c->P_R = dims[0];
      c->Q_R = dims[1] * dims[2];
    }
  }
  c->numel = c->P_R * c->Q_R;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev);
  int l2_bytes = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&l2_bytes, cudaDevAttrL2CacheSize, dev);
  if (e != cudaSuccess) {
    delete c;
    return fail(NTF_ERR_CUDA, "no CUDA device: %s", cudaGetErrorString(e));
  }
  const int R = rank;
  c->pn = ntf::plan_gemm_n(c->P_R, c->Q_R, dtype, d_tensor, c->num_sms);
  c->pt = ntf::plan_gemm_t(c->P_L, c->Q_L, dtype, d_tensor, c->num_sms);
  int64_t part = 0, part_b = 0;
  if (c->pn.chunks > 1) part = std::max<int64_t>(part, c->pn.chunks * c->P_R * R);
  if (c->pt.chunks > 1) part_b = c->pt.chunks * c->Q_L * R;
  if (c->s_R == 2) {
    c->post_split_left = ntf::post_slow_splits(dims[0], dims[1], R, c->num_sms);
    part = std::max<int64_t>(part, c->post_split_left * dims[1] * R);
  }
  if (order - c->s_L == 2) {
    c->post_split_right = ntf::post_slow_splits(dims[c->s_L], dims[c->s_L + 1], R, c->num_sms);
    part = std::max<int64_t>(part, c->post_split_right * dims[c->s_L + 1] * R);
  }
  int64_t post_counts = 0;
  if (R % 4 == 0 || (R % 2 == 0 && R <= 64)) {  // the vectorised levels (float4 or float2)
    if (c->s_R == 2) {
      c->post4_split_left = ntf::post_slow4_splits(dims[0], dims[1], R, c->num_sms);
      part = std::max<int64_t>(part, c->post4_split_left * dims[1] * R);
      post_counts += ntf::post_slow4_blocks(dims[1], R);
    }
    c->post_count_right = post_counts;
    if (order - c->s_L == 2) {
      c->post4_split_right =
          ntf::post_slow4_splits(dims[c->s_L], dims[c->s_L + 1], R, c->num_sms);
      part = std::max<int64_t>(part, c->post4_split_right * dims[c->s_L + 1] * R);
      post_counts += ntf::post_slow4_blocks(dims[c->s_L + 1], R);
    }
  }
  const int64_t w_rows = ntf::kr_rows_padded(c->Q_R), w_rows_b = ntf::kr_rows_padded(c->P_L);
  const int64_t RR = static_cast<int64_t>(R) * R;
  const int upd_blocks = ntf::update_blocks(c->max_dim);
  // arena 0: every buffer whose size is known before the tensor-core plans (whose tensor maps
  // need the split tables' addresses)
  const bool tc = p->contraction != NTF_CONTRACT_SIMT;
  const size_t wu_bytes = tc ? ntf::umma_wsplit_bytes(c->Q_R, R, dtype) : 0;
  const size_t wub_bytes = tc ? ntf::umma_wsplit_bytes(c->P_L, R, dtype) : 0;
  Carver a0;
  const size_t oTR = a0.take(c->P_R * R * sizeof(float));
  const size_t oTL = a0.take(c->Q_L * R * sizeof(float));
  const size_t oW = a0.take(w_rows * ntf::round_rp(R) * sizeof(float));
  const size_t oWb = a0.take(w_rows_b * ntf::round_rp(R) * sizeof(float));
  const size_t oWu = a0.take(wu_bytes), oWub = a0.take(wub_bytes);
  const size_t oPC = a0.take((post_counts + 1) * sizeof(unsigned));
  const size_t oUS = a0.take(4 * sizeof(unsigned));
  const size_t oM = a0.take(c->max_dim * R * sizeof(float));
  const size_t oG = a0.take(order * RR * sizeof(double));
  const size_t oGt = a0.take(order * RR * sizeof(double));
  const size_t oCh = a0.take(order * RR * sizeof(double));
  const size_t oSys = a0.take(ntf::update_sys_bytes(order, R));
  const size_t oGp = a0.take(upd_blocks * RR * sizeof(double));
  const size_t oSp = a0.take(upd_blocks * ntf::update_scalars() * sizeof(double));
  const size_t oFp = a0.take(64 * sizeof(double));
  const size_t oDp = a0.take(1024 * sizeof(double));
  const size_t oCtl = a0.take(sizeof(Ctrl));
  const size_t oSpV = a0.take(c->max_dim * R * sizeof(float));
  const size_t oSpT = a0.take(c->max_dim * R * sizeof(float));
  const size_t oSpS = a0.take(2 * sizeof(unsigned));
  e = cudaMalloc(&c->arena[0], a0.off);
  if (e == cudaSuccess) {
    char* b = static_cast<char*>(c->arena[0]);
    c->TR = reinterpret_cast<float*>(b + oTR);
    c->TL = reinterpret_cast<float*>(b + oTL);
    c->W = reinterpret_cast<float*>(b + oW);
    c->W_b = reinterpret_cast<float*>(b + oWb);
    if (tc) {
      c->Wu = b + oWu;
      c->Wu_b = b + oWub;
    }
    c->post_count = reinterpret_cast<unsigned*>(b + oPC);
    c->umma_sched = reinterpret_cast<unsigned*>(b + oUS);
    c->Mbuf = reinterpret_cast<float*>(b + oM);
    c->grams = reinterpret_cast<double*>(b + oG);
    c->grams_tmp = reinterpret_cast<double*>(b + oGt);
    c->chol = reinterpret_cast<double*>(b + oCh);
    c->sys = reinterpret_cast<double*>(b + oSys);
    c->gram_part = reinterpret_cast<double*>(b + oGp);
    c->scal_part = reinterpret_cast<double*>(b + oSp);
    c->fit_part = reinterpret_cast<double*>(b + oFp);
    c->dpart = reinterpret_cast<double*>(b + oDp);
    c->d_ctrl = reinterpret_cast<Ctrl*>(b + oCtl);
    c->sp_V = reinterpret_cast<float*>(b + oSpV);
    c->sp_tb = reinterpret_cast<float*>(b + oSpT);
    c->sp_sel = reinterpret_cast<unsigned*>(b + oSpS);
  }
  for (int m = 0; m < order; ++m) {  // the non-negative orthant (eq. ADMoM_NTF)
    c->cons_kind[m] = NTF_CONSTRAINT_NONNEG;
    c->cons_lo[m] = 0.0f;
    c->cons_hi[m] = HUGE_VALF;
  }
  // tensor-core plans: the split tables must exist before the tensor maps are encoded
  if (e == cudaSuccess && tc) {
    // zero padding (a rows kernel that writes a table writes only its entries)
    e = cudaMemsetAsync(c->Wu, 0, wu_bytes, c->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->Wu_b, 0, wub_bytes, c->st);
    if (e == cudaSuccess) {
      // Copies of the tensor (params.tensor_copy), context-owned: a row-padded copy of
      // X[P_R, Q_R] when its rows are not 16-byte multiples, and the transposed copy
      // [Q_L, P_L] (rows padded likewise) for the second contraction.  Each is made only if
      // it takes at most half the free device memory (any size for tensor_copy = 1).
      const int64_t es = dtype == NTF_BF16 ? 2 : 4, al = 16 / es;
      const bool copies = p->tensor_copy != -1 && R <= 64;
      const auto fits = [&](size_t bytes) {
        size_t free_b = 0, total_b = 0;
        return p->tensor_copy == 1 ||
               (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess && bytes <= free_b / 2);
      };
      const void* xn = d_tensor;
      int64_t ldn = c->Q_R;
      if ((c->Q_R * es) % 16 != 0 && copies) {
        const int64_t qp = (c->Q_R + al - 1) / al * al;
        const size_t bytes = static_cast<size_t>(c->P_R * qp * es);
        if (fits(bytes) && cudaMalloc(&c->Xp, bytes) == cudaSuccess) {
          e = ntf::launch_pad_rows(d_tensor, static_cast<int>(es), c->P_R, c->Q_R, c->Xp, qp,
                                   c->st);
          xn = c->Xp;
          ldn = qp;
          c->copy_bytes += static_cast<int64_t>(bytes);
        } else {
          cudaGetLastError();  // no room: the first contraction runs on the FMA kernels
          c->Xp = nullptr;
        }
      }
      const bool okn = e == cudaSuccess && ntf::umma_plan(&c->un, false, dtype, xn, c->P_R,
                                                          c->Q_R, R, c->Wu, c->num_sms, ldn);
      // the second contraction X[P_L, Q_L]^T W: on the transposed copy [Q_L, P_L] (a K-major
      // product) when there is one, else on X with M-contiguous tiles, which needs rows of X
      // that are 16-byte multiples
      const bool direct_ok = (c->Q_L * es) % 16 == 0;
      bool copy = copies && (!direct_ok || p->tensor_copy == 1 || dtype != NTF_BF16);
      if (copies && direct_ok && p->tensor_copy == 0 && dtype == NTF_BF16) {
        // BF16: the row-major product on the copy is the faster one for a single-chunk
        // contraction with N = 32 and the table streamed through the stages; the
        // M-contiguous one is faster at N = 64 and when the range is cut into chunks
        ntf::UmmaPlan probe{};
        copy = ntf::umma_plan(&probe, true, dtype, d_tensor, c->P_L, c->Q_L, R, c->Wu_b,
                              c->num_sms) &&
               probe.N == 32 && probe.args.chunks == 1 && !probe.wres;
      }
      int64_t ldt = c->P_L;
      if (copy && e == cudaSuccess) {
        ldt = (c->P_L + al - 1) / al * al;
        const size_t bytes = static_cast<size_t>(c->Q_L * ldt * es);
        if (fits(bytes) && cudaMalloc(&c->Xt, bytes) == cudaSuccess) {
          e = ntf::launch_transpose(d_tensor, static_cast<int>(es), c->P_L, c->Q_L, c->Xt, c->st,
                                    ldt);
          c->copy_bytes += static_cast<int64_t>(bytes);
        } else {
          cudaGetLastError();  // no room: the contraction runs on X
          c->Xt = nullptr;
        }
      }
      const bool okt = e == cudaSuccess &&
                       (c->Xt ? ntf::umma_plan(&c->ut, false, dtype, c->Xt, c->Q_L, c->P_L, R,
                                               c->Wu_b, c->num_sms, ldt)
                              : ntf::umma_plan(&c->ut, true, dtype, d_tensor, c->P_L, c->Q_L, R,
                                               c->Wu_b, c->num_sms));
      // a copy whose plan failed is not kept
      if (e == cudaSuccess && ((!okt && c->Xt) || (!okn && c->Xp))) {
        e = cudaStreamSynchronize(c->st);
        if (!okt && c->Xt) {
          cudaFree(c->Xt);
          c->Xt = nullptr;
        }
        if (!okn && c->Xp) {
          cudaFree(c->Xp);
          c->Xp = nullptr;
        }
        c->copy_bytes = (c->Xt ? c->Q_L * ldt * es : 0) + (c->Xp ? c->P_R * ldn * es : 0);
      }
      if (p->contraction == NTF_CONTRACT_TENSOR && !(okn && okt)) {
        free_ctx(c);
        return fail(NTF_ERR_UNSUPPORTED,
                    "tensor-core contraction needs rank <= 64 and 16-byte aligned tensor rows");
      }
      if (c->un.on && c->un.args.chunks > 1)
        part = std::max<int64_t>(part, c->un.args.chunks * c->P_R * R);
      if (c->ut.on && c->ut.args.chunks > 1)
        part_b = std::max<int64_t>(part_b, c->ut.args.chunks * c->Q_L * R);
    }
  }
  // arena 1: the partial sums, sized by the plans
  Carver a1;
  const size_t oP = a1.take(part * sizeof(float)), oPb = a1.take(part_b * sizeof(float));
  // Factor 0's second tree level in the first contraction's epilogue: worth it when T_R is
  // not served from L2 by the separate level (at least half the L2: reading it back then costs
  // a DRAM pass, and its write-back competes) and N <= 32 (at N = 64 the epilogue's extra
  // registers slow the contraction more than the level costs).
  const bool fuse_fits = c->un.on && c->un.args.chunks == 1 && c->un.N <= 32 && c->s_R >= 2 &&
                         dims[1] >= 32;
  const bool fuse = fuse_fits && (p->fuse_level == 1 ||
                                  (p->fuse_level == 0 && static_cast<double>(c->P_R) * R *
                                                                 sizeof(float) >= 0.5 * l2_bytes));
  const size_t oFz = a1.take(fuse ? ((c->P_R + 31) / 32) * 2 * R * sizeof(float) : 0);
  if (e == cudaSuccess) e = cudaMalloc(&c->arena[1], a1.off);
  if (e == cudaSuccess) {
    c->partial = reinterpret_cast<float*>(static_cast<char*>(c->arena[1]) + oP);
    c->partial_b = reinterpret_cast<float*>(static_cast<char*>(c->arena[1]) + oPb);
    if (fuse) c->fpart = reinterpret_cast<float*>(static_cast<char*>(c->arena[1]) + oFz);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(c->umma_sched, 0, 4 * sizeof(unsigned), c->st);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(c->post_count, 0, (post_counts + 1) * sizeof(unsigned), c->st);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->sB, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->sC, cudaStreamNonBlocking);
  for (cudaEvent_t* ev : {&c->ev_start, &c->ev_tl, &c->ev_b, &c->ev_c})
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
  for (int m = 0; m < order && e == cudaSuccess; ++m) {
    e = cudaEventCreateWithFlags(&c->ev_sys[m], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_rows[m], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_red[m], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_post[m], cudaEventDisableTiming);
  }
  void* pin = nullptr;
  if (e == cudaSuccess) e = pinned_acquire(&pin);
  if (e == cudaSuccess) {
    c->h_ctrl = static_cast<Ctrl*>(pin);
    c->h_snap = reinterpret_cast<ntf::SweepSnap*>(static_cast<char*>(pin) +
                                                  kPinnedBytes - 2 * sizeof(ntf::SweepSnap));
    e = cudaHostGetDevicePointer((void**)&c->d_snap, c->h_snap, 0);
  }
  for (cudaEvent_t& ev : c->ev_sweep)
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    free_ctx(c);
    return fail(e == cudaErrorMemoryAllocation ? NTF_ERR_OOM : NTF_ERR_CUDA,
                "workspace allocation: %s", cudaGetErrorString(e));
  }
  std::memset(c->h_ctrl, 0, sizeof(Ctrl));
  for (int m = 0; m < order; ++m) c->h_ctrl->rho[m] = p->rho0;
  e = cudaMemcpyAsync(c->d_ctrl, c->h_ctrl, sizeof(Ctrl), cudaMemcpyHostToDevice, c->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->grams, 0, order * RR * sizeof(double), c->st);
  if (e == cudaSuccess)
    e = ntf::launch_norm2(d_tensor, dtype, c->numel, c->dpart, 1024, &c->d_ctrl->x_norm2, c->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&c->x_norm2, &c->d_ctrl->x_norm2, sizeof(double), cudaMemcpyDeviceToHost,
                        c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) {
    free_ctx(c);
    return fail(NTF_ERR_CUDA, "context setup: %s", cudaGetErrorString(e));
  }
  *out = c;
  return NTF_OK;
}

ntf_status ntf_destroy(ntf_ctx* ctx) {
  if (ctx) {
    cudaStreamSynchronize(ctx->st);
    free_ctx(ctx);
  }
  return NTF_OK;
}

ntf_status ntf_tensor_norm2(ntf_ctx* ctx, double* out) {
  if (!ctx || !out) return fail(NTF_ERR_INVALID_ARG, "null argument");
  *out = ctx->x_norm2;
  return NTF_OK;
}

ntf_status ntf_mttkrp(ntf_ctx* c, int mode, const float* const* F, float* d_M) {
  (void)cudaGetLastError();  // a stale non-sticky error is not this call's
  NTF_TRY(check_mode(c, mode));
  if (!F || !d_M) return fail(NTF_ERR_INVALID_ARG, "null factors or output");
  for (int m = 0; m < c->N; ++m)
    if (m != mode && (!F[m] || misaligned(F[m], sizeof(float))))
      return fail(NTF_ERR_INVALID_ARG, "null or misaligned factor %d", m);
  if (misaligned(d_M, sizeof(float))) return fail(NTF_ERR_INVALID_ARG, "misaligned output");
  if (mode < c->s_R) {
    float* T = c->s_R == 1 ? d_M : c->TR;
    NTF_TRY(contract_right(c, F, T, c->st, false, mode == 0));
    NTF_TRY(finish_mode(c, mode, T, F, d_M, c->st));
  } else {
    NTF_TRY(contract_left(c, F, c->TL, c->st));
    NTF_TRY(finish_mode(c, mode, c->TL, F, d_M, c->st));
  }
  return NTF_OK;
}

ntf_status ntf_gram(ntf_ctx* c, int mode, const float* d_F, double* d_G) {
  (void)cudaGetLastError();  // a stale non-sticky error is not this call's
  NTF_TRY(check_mode(c, mode));
  if (!d_F) return fail(NTF_ERR_INVALID_ARG, "null factor");
  if (misaligned(d_F, sizeof(float)) || misaligned(d_G, sizeof(double)))
    return fail(NTF_ERR_INVALID_ARG, "misaligned factor or Gram");
  const int64_t RR = static_cast<int64_t>(c->R) * c->R;
  double* G = c->grams + mode * RR;
  NTF_CUDA(ntf::launch_gram(d_F, c->dims[mode], c->R, G, c->st));
  if (d_G) NTF_CUDA(cudaMemcpyAsync(d_G, G, RR * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
  return NTF_OK;
}

ntf_status ntf_system(ntf_ctx* c, int mode, double* d_H, double* d_L, double* rho_out) {
  (void)cudaGetLastError();  // a stale non-sticky error is not this call's
  NTF_TRY(check_mode(c, mode));
  if (misaligned(d_H, sizeof(double)) || misaligned(d_L, sizeof(double)))
    return fail(NTF_ERR_INVALID_ARG, "misaligned output");
  const int64_t RR = static_cast<int64_t>(c->R) * c->R;
  double* L = c->chol + mode * RR;
  NTF_CUDA(ntf::launch_system(c->grams, c->N, mode, c->R, c->prm.rho_policy, c->d_ctrl, d_H, L,
                              c->st));
  if (d_L) NTF_CUDA(cudaMemcpyAsync(d_L, L, RR * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
  NTF_TRY(read_ctrl(c));
  if (rho_out) *rho_out = c->h_ctrl->stats[mode][5];
  return take_status(c);
}

ntf_status ntf_admm_update(ntf_ctx* c, int mode, const float* d_M, float* d_A, float* d_At,
                           float* d_Y, ntf_update_stats* stats) {
  (void)cudaGetLastError();  // a stale non-sticky error is not this call's
  NTF_TRY(check_mode(c, mode));
  if (!d_M || !d_A || !d_At || !d_Y) return fail(NTF_ERR_INVALID_ARG, "null matrix argument");
  for (const void* q : {static_cast<const void*>(d_M), static_cast<const void*>(d_A),
                        static_cast<const void*>(d_At), static_cast<const void*>(d_Y)})
    if (misaligned(q, sizeof(float))) return fail(NTF_ERR_INVALID_ARG, "misaligned matrix");
  c->ws_now = true;  // a single update consults an attached network
  NTF_TRY(enqueue_update(c, mode, d_M, d_A, d_At, d_Y, false));
  if (!stats) return NTF_OK;
  NTF_TRY(read_ctrl(c));
  const double* s = c->h_ctrl->stats[mode];
  stats->primal_res = s[0];
  stats->dual_res = s[1];
  stats->norm_A = s[2];
  stats->norm_At = s[3];
  stats->norm_Y = s[4];
  stats->rho = s[5];
  stats->kkt_neg_x = c->h_ctrl->kkt[mode][0];
  stats->kkt_dual = c->h_ctrl->kkt[mode][1];
  stats->kkt_comp = c->h_ctrl->kkt[mode][2];
  return take_status(c);
}

ntf_status ntf_set_rho(ntf_ctx* c, int mode, double rho) {
  NTF_TRY(check_mode(c, mode));
  if (!(rho > 0.0) || !std::isfinite(rho)) return fail(NTF_ERR_INVALID_ARG, "rho must be > 0");
  c->h_ctrl->rho[mode] = rho;  // staged through the pinned block
  NTF_CUDA(cudaMemcpyAsync(&c->d_ctrl->rho[mode], &c->h_ctrl->rho[mode], sizeof(double),
                           cudaMemcpyHostToDevice, c->st));
  NTF_CUDA(cudaStreamSynchronize(c->st));
  return NTF_OK;
}

ntf_status ntf_get_rho(ntf_ctx* c, int mode, double* rho) {
  NTF_TRY(check_mode(c, mode));
  if (!rho) return fail(NTF_ERR_INVALID_ARG, "null output");
  NTF_TRY(read_ctrl(c));
  *rho = c->h_ctrl->rho[mode];
  return NTF_OK;
}

ntf_status ntf_fit(ntf_ctx* c, const float* const* F, double* rel_err) {
  (void)cudaGetLastError();  // a stale non-sticky error is not this call's
  if (!c || !F || !rel_err) return fail(NTF_ERR_INVALID_ARG, "null argument");
  for (int m = 0; m < c->N; ++m)
    if (!F[m] || misaligned(F[m], sizeof(float)))
      return fail(NTF_ERR_INVALID_ARG, "null or misaligned factor %d", m);
  const int last = c->N - 1;
  NTF_TRY(ntf_mttkrp(c, last, F, c->Mbuf));
  const int64_t RR = static_cast<int64_t>(c->R) * c->R;
  for (int m = 0; m < c->N; ++m)
    NTF_CUDA(ntf::launch_gram(F[m], c->dims[m], c->R, c->grams_tmp + m * RR, c->st));
  NTF_CUDA(ntf::launch_fit(c->Mbuf, F[last], c->dims[last], c->R, c->grams_tmp, c->N,
                           c->fit_part, c->d_ctrl, c->st));
  NTF_TRY(read_ctrl(c));
  *rel_err = c->h_ctrl->rel_err;
  return take_status(c);
}

ntf_status ntf_fit_explicit(ntf_ctx* c, const float* const* F, double* rel_err) {
  (void)cudaGetLastError();  // a stale non-sticky error is not this call's
  if (!c || !F || !rel_err) return fail(NTF_ERR_INVALID_ARG, "null argument");
  for (int m = 0; m < c->N; ++m)
    if (!F[m] || misaligned(F[m], sizeof(float)))
      return fail(NTF_ERR_INVALID_ARG, "null or misaligned factor %d", m);
  NTF_CUDA(ntf::launch_fit_explicit(c->X, c->dtype, c->N, c->dims, F, c->R, c->dpart, 1024,
                                    c->d_ctrl, c->st));
  NTF_TRY(read_ctrl(c));
  *rel_err = c->h_ctrl->rel_err;
  return take_status(c);
}

ntf_status ntf_fit_from_mttkrp(ntf_ctx* c, const float* d_M_last, const float* d_F_last,
                               double* rel_err) {
  if (!c || !d_M_last || !d_F_last || !rel_err) return fail(NTF_ERR_INVALID_ARG, "null argument");
  if (misaligned(d_M_last, sizeof(float)) || misaligned(d_F_last, sizeof(float)))
    return fail(NTF_ERR_INVALID_ARG, "misaligned matrix");
  NTF_CUDA(ntf::launch_fit(d_M_last, d_F_last, c->dims[c->N - 1], c->R, c->grams, c->N,
                           c->fit_part, c->d_ctrl, c->st));
  NTF_TRY(read_ctrl(c));
  *rel_err = c->h_ctrl->rel_err;
  return take_status(c);
}

ntf_status ntf_profile_enable(ntf_ctx* c, int enable) {
  if (!c) return fail(NTF_ERR_INVALID_ARG, "null context");
  if (enable)
    for (auto& set : c->ev)
      for (auto& pair : set)
        for (auto& e : pair)
          if (!e) NTF_CUDA(cudaEventCreate(&e));
  c->prof = enable != 0;
  c->pr = ntf_profile{};
  for (auto& q : c->ev_pending) q[0] = q[1] = false;
  c->launches = 0;
  NTF_CUDA(cudaMemsetAsync(c->d_ctrl->ws_rows, 0, sizeof(c->d_ctrl->ws_rows), c->st));
  const double esize = c->dtype == NTF_BF16 ? 2.0 : 4.0;
  c->pr.contraction_bytes[0] = c->pr.contraction_bytes[1] = static_cast<double>(c->numel) * esize;
  return NTF_OK;
}

ntf_status ntf_trace_enable(ntf_ctx* c, int enable) {
  if (!c) return fail(NTF_ERR_INVALID_ARG, "null context");
  if (enable) {
    if (!c->tr_origin) NTF_CUDA(cudaEventCreate(&c->tr_origin));
    for (cudaEvent_t& e : c->tr_ev)
      if (!e) NTF_CUDA(cudaEventCreate(&e));
  }
  c->trace = enable != 0;
  c->tr_n = 0;
  return NTF_OK;
}

ntf_status ntf_trace_get(ntf_ctx* c, ntf_trace_entry* out, int max_entries, int* n_entries) {
  if (!c || !n_entries || (max_entries > 0 && !out))
    return fail(NTF_ERR_INVALID_ARG, "null argument");
  *n_entries = c->tr_n;
  if (c->tr_n == 0) return NTF_OK;
  NTF_CUDA(cudaStreamSynchronize(c->st));
  for (int i = 0; i < c->tr_n && i < max_entries; ++i) {
    float b = 0.0f, e = 0.0f;
    NTF_CUDA(cudaEventElapsedTime(&b, c->tr_origin, c->tr_ev[2 * i]));
    NTF_CUDA(cudaEventElapsedTime(&e, c->tr_origin, c->tr_ev[2 * i + 1]));
    ntf_trace_entry& o = out[i];
    std::memset(o.name, 0, sizeof o.name);
    std::strncpy(o.name, c->tr_info[i].name, sizeof o.name - 1);
    o.stream = c->tr_info[i].stream;
    o.mode = c->tr_info[i].mode;
    o.start_us = 1000.0 * b;
    o.end_us = 1000.0 * e;
  }
  return NTF_OK;
}

ntf_status ntf_profile_get(ntf_ctx* c, ntf_profile* out) {
  if (!c || !out) return fail(NTF_ERR_INVALID_ARG, "null argument");
  NTF_TRY(read_ctrl(c));
  *out = c->pr;
  out->kernel_launches = c->launches;
  out->ws_rows_considered = static_cast<int64_t>(c->h_ctrl->ws_rows[0]);
  out->ws_rows_accepted = static_cast<int64_t>(c->h_ctrl->ws_rows[1]);
  out->tensor_copy_bytes = c->copy_bytes;
  return NTF_OK;
}

ntf_status ntf_attach_warmstart(ntf_ctx* c, ntf_mlp* net, int sweeps) {
  if (!c) return fail(NTF_ERR_INVALID_ARG, "null context");
  if (sweeps < 0) return fail(NTF_ERR_INVALID_ARG, "sweeps must be >= 0");
  if (net && ntf::mlp_rank(net) != c->R)
    return fail(NTF_ERR_INVALID_ARG, "network rank %d differs from the context rank %d",
                ntf::mlp_rank(net), c->R);
  if (net && ntf::mlp_max_rows(net) < c->max_dim)
    return fail(NTF_ERR_INVALID_ARG, "network workspace (%d rows) smaller than a factor (%lld)",
                ntf::mlp_max_rows(net), static_cast<long long>(c->max_dim));
  c->ws = net;
  c->ws_sweeps = sweeps;
  return NTF_OK;
}

ntf_status ntf_warmstart_rows(ntf_ctx* c, int mode, const float* d_M, const float* d_At,
                              const float* d_Y, float* d_Gn, float* d_mrows, float* d_targets,
                              double* s_out) {
  (void)cudaGetLastError();  // a stale non-sticky error is not this call's
  NTF_TRY(check_mode(c, mode));
  if (!d_M || !d_Gn || !d_mrows || !s_out)
    return fail(NTF_ERR_INVALID_ARG, "null MTTKRP, feature output or s");
  if (d_targets && (!d_At || !d_Y))
    return fail(NTF_ERR_INVALID_ARG, "targets need the auxiliary and the dual");
  for (const void* q : {static_cast<const void*>(d_M), static_cast<const void*>(d_At),
                        static_cast<const void*>(d_Y), static_cast<const void*>(d_Gn),
                        static_cast<const void*>(d_mrows), static_cast<const void*>(d_targets)})
    if (misaligned(q, sizeof(float))) return fail(NTF_ERR_INVALID_ARG, "misaligned matrix");
  const int R = c->R;
  const int64_t I = c->dims[mode];
  // the factor's coefficient system, as its update builds it (stored Grams, penalty policy)
  NTF_CUDA(ntf::launch_update_system(make_call(c, mode, d_M, nullptr, nullptr, nullptr, false),
                                     c->st));
  float* s_dev = reinterpret_cast<float*>(c->dpart);  // scratch of the context
  NTF_CUDA(ntf::ws_prepare(ntf::update_sys_h32(c->sys, mode, R),
                           ntf::update_sys_hinv32(c->sys, mode, R), d_M, R, I, d_Gn, d_mrows,
                           s_dev, c->st));
  if (d_targets) NTF_CUDA(ntf::ws_targets(d_At, d_Y, s_dev, R, I, d_targets, c->st));
  float s_h = 0.0f;
  NTF_CUDA(cudaMemcpyAsync(&s_h, s_dev, sizeof(float), cudaMemcpyDeviceToHost, c->st));
  NTF_CUDA(cudaStreamSynchronize(c->st));
  *s_out = s_h;
  NTF_TRY(read_ctrl(c));
  return take_status(c);
}

ntf_status ntf_set_constraint(ntf_ctx* c, int mode, int kind, double lo, double hi,
                              int64_t max_nonzeros) {
  NTF_TRY(check_mode(c, mode));
  const int64_t n = c->dims[mode] * c->R;
  switch (kind) {
    case NTF_CONSTRAINT_NONNEG:
      lo = 0.0;
      hi = HUGE_VAL;
      break;
    case NTF_CONSTRAINT_BOX:
      if (!(lo <= hi) || std::isnan(lo) || std::isnan(hi) || lo == HUGE_VAL || hi == -HUGE_VAL)
        return fail(NTF_ERR_INVALID_ARG, "box constraint needs lo <= hi, not NaN");
      break;
    case NTF_CONSTRAINT_SPARSE:
      if (max_nonzeros < 0) return fail(NTF_ERR_INVALID_ARG, "max_nonzeros must be >= 0");
      if (n >= (int64_t{1} << 32))
        return fail(NTF_ERR_UNSUPPORTED, "sparsity constraint needs I_n R < 2^32");
      lo = 0.0;
      hi = HUGE_VAL;
      break;
    default:
      return fail(NTF_ERR_INVALID_ARG, "unknown constraint kind %d", kind);
  }
  c->cons_kind[mode] = kind;
  c->cons_lo[mode] = static_cast<float>(lo);
  c->cons_hi[mode] = static_cast<float>(hi);
  c->cons_c[mode] = max_nonzeros;
  // recorded sweeps hold the previous constraints: record them again at the next run
  for (ntf_ctx::SweepGraph& g : c->graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
    g.exec = nullptr;
    g.graph = nullptr;
  }
  return NTF_OK;
}

ntf_status ntf_sync(ntf_ctx* c) {
  if (!c) return fail(NTF_ERR_INVALID_ARG, "null context");
  NTF_TRY(read_ctrl(c));
  return take_status(c);
}

ntf_status ntf_watchdog_check(ntf_ctx* c, double limit_ms) {
  if (!c) return fail(NTF_ERR_INVALID_ARG, "null context");
  if (!(limit_ms > 0.0 && limit_ms <= 2000.0))
    return fail(NTF_ERR_INVALID_ARG, "limit_ms must be in (0, 2000]");
  NTF_TRY(ntf_sync(c));  // a status that was already pending is reported first
  NTF_CUDA(ntf::launch_wait_check(&c->d_ctrl->status, static_cast<uint64_t>(limit_ms * 1e6),
                                  c->st));
  return ntf_sync(c);
}

ntf_status ntf_run(ntf_ctx* c, float* const* A, float* const* At, float* const* Y, int max_outer,
                   double target_rfe, int check_every, double* rfe_hist, ntf_run_stats* out) {
  (void)cudaGetLastError();  // a stale non-sticky error is not this call's
  if (!c || !A || !At || !Y) return fail(NTF_ERR_INVALID_ARG, "null argument");
  if (max_outer < 1) return fail(NTF_ERR_INVALID_ARG, "max_outer must be >= 1");
  if (check_every < 1) check_every = 1;
  for (int m = 0; m < c->N; ++m)
    if (!A[m] || !At[m] || !Y[m]) return fail(NTF_ERR_INVALID_ARG, "null state of factor %d", m);
  for (int m = 0; m < c->N; ++m)
    if (misaligned(A[m], sizeof(float)) || misaligned(At[m], sizeof(float)) ||
        misaligned(Y[m], sizeof(float)))
      return fail(NTF_ERR_INVALID_ARG, "misaligned state of factor %d", m);
  const bool use_res = c->prm.eps_abs > 0.0 || c->prm.eps_rel > 0.0;
  const bool use_tgt = target_rfe > 0.0;
  const bool use_kkt = c->prm.kkt_dual_tol > 0.0 || c->prm.kkt_comp_tol > 0.0;
  if (rfe_hist)
    for (int i = 0; i < max_outer; ++i) rfe_hist[i] = NAN;
  const float* const* src = c->prm.kr_source == NTF_KR_AUX ? At : A;
  const int64_t RR = static_cast<int64_t>(c->R) * c->R;
  for (int m = 0; m < c->N; ++m)
    NTF_CUDA(ntf::launch_gram(src[m], c->dims[m], c->R, c->grams + m * RR, c->st));
  NTF_TRY(enqueue_prologue(c, A, At, Y));

  // Run control in the control block: the stopping rules are evaluated on the device by the
  // last factor's reduction of every checked sweep, which also writes the sweep's outcome to a
  // host-mapped slot.  The host enqueues sweep `it` before it reads the outcome of sweep it-1,
  // so the GPU does not wait for the host between sweeps; when sweep it-1 met a rule, sweep
  // it finds `stop` set and every kernel that would change the state returns at once.  (Sweeps
  // that consult the warm-start network, and traced sweeps, are read back before the next one
  // is enqueued: the network's kernels do not test `stop`, and a trace shows the last sweep.)
  {
    Ctrl& h = *c->h_ctrl;  // staging of the run-control fields
    h.stop = h.stop_next = h.sweep = 0;
    h.use_tgt = use_tgt;
    h.use_res = use_res;
    h.check_every = check_every;
    h.max_outer = max_outer;
    h.target_rfe = target_rfe;
    h.eps_rel = c->prm.eps_rel;
    for (int m = 0; m < c->N; ++m)
      h.res_base[m] = std::sqrt(static_cast<double>(c->dims[m]) * c->R) * c->prm.eps_abs;
    h.use_kkt = use_kkt;
    h.kkt_dual_tol = c->prm.kkt_dual_tol;
    h.kkt_comp_tol = c->prm.kkt_comp_tol;
    const size_t off = offsetof(Ctrl, stop), len = sizeof(Ctrl) - off;
    NTF_CUDA(cudaMemcpyAsync(reinterpret_cast<char*>(c->d_ctrl) + off,
                             reinterpret_cast<char*>(c->h_ctrl) + off, len,
                             cudaMemcpyHostToDevice, c->st));
    c->h_snap[0].sweep = c->h_snap[1].sweep = -1;
  }
  // however the run ends (an error included), the flags go back to zero on the stream after
  // its last sweep: kernels launched outside a run must not find it stopped
  struct StopReset {
    ntf_ctx* c;
    ~StopReset() { (void)cudaMemsetAsync(&c->d_ctrl->stop, 0, 3 * sizeof(int), c->st); }
  } stop_reset{c};

  // The sweep is recorded once as a CUDA graph (after one eager sweep has set every kernel
  // attribute) and replayed; it is re-recorded only if the state pointers change.  Sweeps
  // that consult the warm-start network have their own recording.
  ntf_run_stats rs{};
  rs.rel_err = NAN;
  rs.kkt_dual = rs.kkt_comp = NAN;
  ntf_status result = NTF_OK;
  bool done = false;
  // Capture needs a non-legacy stream; otherwise (or if capture fails) launch eagerly.
  bool can_graph = c->st != nullptr;
  int unread = -1;  // a checked sweep whose outcome has not been read yet
  // read the outcome of sweep k (completed or not): stopping rules, history, status
  auto read_sweep = [&](int k) -> ntf_status {
    NTF_CUDA(cudaEventSynchronize(c->ev_sweep[k & 1]));
    prof_collect(c, k & 1);
    const ntf::SweepSnap sn = c->h_snap[k & 1];
    if (sn.sweep != k + 1 || sn.status != 0) {
      // no outcome (a system failed) or a device-side error: the status says which
      NTF_CUDA(cudaStreamSynchronize(c->st));
      NTF_TRY(read_ctrl(c));
      NTF_TRY(take_status(c));
      if (sn.sweep != k + 1) return fail(NTF_ERR_CUDA, "sweep %d left no outcome", k);
    }
    rs.iters = k + 1;
    rs.rel_err = sn.rel_err;
    rs.kkt_dual = sn.kkt_dual;
    rs.kkt_comp = sn.kkt_comp;
    if (rfe_hist) rfe_hist[k] = sn.rel_err;
    if (sn.stop & 1) rs.reached_target = 1;
    if (sn.stop & 2) rs.converged = 1;
    if (sn.stop & 4) rs.kkt_met = 1;
    if (sn.stop) done = true;
    return NTF_OK;
  };
  ntf_status st_run = NTF_OK;
  for (int it = 0; it < max_outer && !done; ++it) {
    c->ws_now = c->ws != nullptr && (c->ws_sweeps == 0 || it < c->ws_sweeps);
    if (unread >= 0 && (c->ws_now || c->trace)) {  // read before such a sweep is enqueued
      st_run = read_sweep(unread);
      unread = -1;
      if (st_run != NTF_OK || done) break;
    }
    ntf_mlp* const sweep_ws = c->ws_now ? c->ws : nullptr;
    ntf_ctx::SweepGraph& g = c->graphs[sweep_ws ? 1 : 0];
    c->prof_par = it & 1;
    bool same = g.exec != nullptr && g.prof == c->prof && g.trace == c->trace &&
                g.ws == sweep_ws;
    for (int m = 0; m < c->N && same; ++m)
      same = g.key[3 * m] == A[m] && g.key[3 * m + 1] == At[m] && g.key[3 * m + 2] == Y[m];
    if (same) {
      NTF_TRY(launch_graph(c, g));
    } else if (!c->swept_eagerly || !can_graph) {
      NTF_TRY(enqueue_sweep(c, A, At, Y));
      c->swept_eagerly = true;
    } else {
      if (g.exec) cudaGraphExecDestroy(g.exec);
      if (g.graph) cudaGraphDestroy(g.graph);
      g.exec = nullptr;
      g.graph = nullptr;
      cudaGraph_t gr = nullptr;
      const int64_t before = c->launches;
      bool ok = cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      ntf_status sw = ok ? enqueue_sweep(c, A, At, Y) : NTF_OK;
      g.launches = static_cast<int>(c->launches - before);
      c->launches = before;
      if (ok) ok = cudaStreamEndCapture(c->st, &gr) == cudaSuccess && sw == NTF_OK;
      if (ok) ok = find_prof_nodes(c, gr, g) == NTF_OK;
      if (ok) ok = cudaGraphInstantiate(&g.exec, gr, 0) == cudaSuccess;
      if (!ok) {
        (void)cudaGetLastError();
        if (gr) cudaGraphDestroy(gr);
        if (g.exec) cudaGraphExecDestroy(g.exec);
        g.exec = nullptr;
        can_graph = false;
        NTF_TRY(enqueue_sweep(c, A, At, Y));
      } else {
        g.graph = gr;
        g.prof = c->prof;
        g.trace = c->trace;
        g.ws = sweep_ws;
        for (int m = 0; m < c->N; ++m) {
          g.key[3 * m] = A[m];
          g.key[3 * m + 1] = At[m];
          g.key[3 * m + 2] = Y[m];
        }
        NTF_TRY(launch_graph(c, g));
      }
    }
    NTF_CUDA(cudaEventRecord(c->ev_sweep[it & 1], c->st));
    if (c->prof) c->pr.sweeps += 1;
    rs.iters = it + 1;
    if (unread >= 0) {  // the previous checked sweep, while this one runs
      st_run = read_sweep(unread);
      unread = -1;
      if (st_run != NTF_OK) break;
      if (done) {
        rs.iters = it;  // sweep `it` finds stop set and leaves the state as it is
        break;
      }
    }
    const bool check = ((it + 1) % check_every == 0) || it + 1 == max_outer;
    if (check) unread = it;
    if (check && (c->ws_now || c->trace || it + 1 == max_outer)) {
      st_run = read_sweep(unread);
      unread = -1;
      if (st_run != NTF_OK) break;
    }
  }
  if (st_run == NTF_OK && unread >= 0) st_run = read_sweep(unread);
  if (st_run != NTF_OK) return st_run;
  if (!done && (use_res || use_tgt || use_kkt)) result = NTF_ERR_NOT_CONVERGED;
  if (out) *out = rs;
  if (result != NTF_OK) fail(result, "no stopping criterion met in %d iterations", max_outer);
  return result;
}

ntf_status ntf_to_bf16(const float* d_in, uint16_t* d_out, int64_t n, void* stream) {
  if (!d_in || !d_out || n < 0) return fail(NTF_ERR_INVALID_ARG, "bad argument");
  if (misaligned(d_in, sizeof(float)) || misaligned(d_out, sizeof(uint16_t)))
    return fail(NTF_ERR_INVALID_ARG, "input or output not aligned to its element size");
  if (n == 0) return NTF_OK;
  // the input is read through its device address: device memory as it is, page-locked host
  // memory through the address the device maps it at; anything else is refused
  cudaPointerAttributes at{};
  NTF_CUDA(cudaPointerGetAttributes(&at, d_in));
  const float* src = d_in;
  if (at.type == cudaMemoryTypeHost) {
    if (!at.devicePointer)
      return fail(NTF_ERR_INVALID_ARG, "host input is not mapped into the device address space");
    src = static_cast<const float*>(at.devicePointer);
  } else if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) {
    return fail(NTF_ERR_INVALID_ARG, "input is neither device memory nor page-locked host memory");
  }
  NTF_CUDA(ntf::launch_to_bf16(src, d_out, n, static_cast<cudaStream_t>(stream)));
  return NTF_OK;
}

}  // extern "C"
