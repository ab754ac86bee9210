// C ABI of the NTF library (include/ntf.h): context management, argument checking, the
// per-step entry points and the native outer-iteration driver.
//
// Tensor passes per outer iteration.  The tensor is handled as X[P, Q] with P = I_1..I_s,
// Q = I_{s+1}..I_N (s = 1 for N = 3, s = 2 for N = 4).  Factors 1..s are updated from one
// contraction T_R = X * KR(factors s+1..N), factors s+1..N from one contraction
// T_L = X^T * KR(factors 1..s).  Gauss-Seidel order (eq. ADMM_NTF_ALS_C) is respected: T_R
// only involves factors that are not updated before the factors it serves, and T_L is
// formed after factors 1..s have been updated.  So a sweep reads the tensor twice, whatever
// N is, and every M_n equals the MTTKRP of its definition up to summation order.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ntf_internal.cuh"

using ntf::Ctrl;
using ntf::GemmPlan;
using ntf::Group;

struct ntf_ctx {
  int N = 0, R = 0, dtype = 0, s = 0, num_sms = 0;
  int64_t dims[ntf::kMaxOrder] = {0, 0, 0, 0};
  int64_t P = 0, Q = 0, max_dim = 0;
  const void* X = nullptr;
  cudaStream_t st = nullptr;
  ntf_params prm{};
  GemmPlan pn{}, pt{};
  int post_split_left = 1, post_split_right = 1;
  // workspace
  float* partial = nullptr;      // split-K partials
  float* TR = nullptr;           // [P, R]
  float* TL = nullptr;           // [Q, R]
  float* Mbuf = nullptr;         // [max_dim, R]
  double* grams = nullptr;       // [N, R, R] stored Grams
  double* grams_tmp = nullptr;   // [N, R, R] for ntf_fit
  double* chol = nullptr;        // [N, R, R]
  double* norm_part = nullptr;   // [row blocks, 5]
  double* fit_part = nullptr;    // [64]
  double* dpart = nullptr;       // [1024] misc FP64 partials
  Ctrl* d_ctrl = nullptr;
  Ctrl* h_ctrl = nullptr;        // pinned
  double x_norm2 = 0.0;
  cudaGraphExec_t graph = nullptr;
  const void* graph_key[3 * ntf::kMaxOrder] = {};
  int graph_launches = 0;        // kernels in the recorded sweep
  bool graph_prof = false;       // whether the recorded sweep holds profiling events
  // profiling
  bool prof = false;
  cudaEvent_t ev[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  bool ev_pending[2] = {false, false};
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
ntf_status prof_mark(ntf_ctx* c, int k, int which) {
  if (!c->prof) return NTF_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  NTF_CUDA(cudaStreamIsCapturing(c->st, &cs));
  if (cs == cudaStreamCaptureStatusActive)
    NTF_CUDA(cudaEventRecordWithFlags(c->ev[k][which], c->st, cudaEventRecordExternal));
  else
    NTF_CUDA(cudaEventRecord(c->ev[k][which], c->st));
  if (which == 1) c->ev_pending[k] = true;
  return NTF_OK;
}

// T_R[P, R] = X * KR(factors s..N-1)
ntf_status contract_right(ntf_ctx* c, const float* const* F, float* dst) {
  const Group g = make_group(c, c->s, c->N - c->s, F);
  float* out = c->pn.splits > 1 ? c->partial : dst;
  NTF_TRY(prof_mark(c, 0, 0));
  NTF_CUDA(ntf::launch_gemm_n(c->X, c->dtype, c->P, c->Q, c->R, g, c->pn, out, c->st));
  NTF_TRY(prof_mark(c, 0, 1));
  c->launches += 1;
  if (c->pn.splits > 1) {
    NTF_CUDA(ntf::launch_sum_splits(c->partial, c->pn.splits, c->P * c->R, dst, c->st));
    c->launches += 1;
  }
  return NTF_OK;
}

// T_L[Q, R] = X^T * KR(factors 0..s-1)
ntf_status contract_left(ntf_ctx* c, const float* const* F, float* dst) {
  const Group g = make_group(c, 0, c->s, F);
  float* out = c->pt.splits > 1 ? c->partial : dst;
  NTF_TRY(prof_mark(c, 1, 0));
  NTF_CUDA(ntf::launch_gemm_t(c->X, c->dtype, c->P, c->Q, c->R, g, c->pt, out, c->st));
  NTF_TRY(prof_mark(c, 1, 1));
  c->launches += 1;
  if (c->pt.splits > 1) {
    NTF_CUDA(ntf::launch_sum_splits(c->partial, c->pt.splits, c->Q * c->R, dst, c->st));
    c->launches += 1;
  }
  return NTF_OK;
}

// After a host synchronisation: add the device time of the last recorded contractions.
void prof_collect(ntf_ctx* c) {
  if (!c->prof) return;
  for (int k = 0; k < 2; ++k) {
    if (!c->ev_pending[k]) continue;
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, c->ev[k][0], c->ev[k][1]) == cudaSuccess) {
      c->pr.contractions[k] += 1;
      c->pr.contraction_ms[k] += ms;
    } else {
      (void)cudaGetLastError();  // not recorded: leave no stale error behind
    }
  }
}

// Second tree level: M of `mode` from the group's contraction T (group of 1 or 2 modes).
ntf_status finish_mode(ntf_ctx* c, int mode, const float* T, const float* const* F, float* M) {
  const bool left = mode < c->s;
  const int first = left ? 0 : c->s;
  const int count = left ? c->s : c->N - c->s;
  if (count == 1) {
    if (T != M)
      NTF_CUDA(cudaMemcpyAsync(M, T, c->dims[mode] * c->R * sizeof(float),
                               cudaMemcpyDeviceToDevice, c->st));
    return NTF_OK;
  }
  const int64_t Ia = c->dims[first], Ib = c->dims[first + 1];
  if (mode == first) {
    NTF_CUDA(ntf::launch_post_fast(T, Ia, Ib, c->R, F[first + 1], M, c->st));
    c->launches += 1;
  } else {
    const int sp = left ? c->post_split_left : c->post_split_right;
    NTF_CUDA(ntf::launch_post_slow(T, Ia, Ib, c->R, F[first], sp, c->partial, M, c->st));
    c->launches += sp > 1 ? 2 : 1;
  }
  return NTF_OK;
}

ntf_status enqueue_update(ntf_ctx* c, int mode, const float* M, float* A, float* At, float* Y) {
  const int64_t I = c->dims[mode];
  const int R = c->R;
  double* L = c->chol + static_cast<int64_t>(mode) * R * R;
  NTF_CUDA(ntf::launch_system(c->grams, c->N, mode, R, c->prm.rho_policy, c->d_ctrl, nullptr, L,
                              c->st));
  NTF_CUDA(ntf::launch_admm_rows(M, A, At, Y, L, I, R, c->prm.inner_iters, mode, c->d_ctrl,
                                 c->norm_part, c->st));
  NTF_CUDA(ntf::launch_update_finalize(c->norm_part, ntf::admm_row_blocks(I), mode,
                                       c->prm.rho_policy, c->prm.mu, c->prm.tau_incr,
                                       c->prm.tau_decr, c->d_ctrl, c->st));
  const float* src = c->prm.kr_source == NTF_KR_AUX ? At : A;
  NTF_CUDA(ntf::launch_gram(src, I, R, c->grams + static_cast<int64_t>(mode) * R * R, c->st));
  c->launches += 4;
  return NTF_OK;
}

// One outer iteration in Gauss-Seidel order with two tensor passes, then the fit terms.
ntf_status enqueue_sweep(ntf_ctx* c, float* const* A, float* const* At, float* const* Y) {
  const float* const* src = c->prm.kr_source == NTF_KR_AUX ? At : A;
  const float* T = c->s == 1 ? c->Mbuf : c->TR;
  NTF_TRY(contract_right(c, src, const_cast<float*>(T)));
  for (int m = 0; m < c->s; ++m) {
    NTF_TRY(finish_mode(c, m, T, src, c->Mbuf));
    NTF_TRY(enqueue_update(c, m, c->Mbuf, A[m], At[m], Y[m]));
  }
  NTF_TRY(contract_left(c, src, c->TL));
  for (int m = c->s; m < c->N; ++m) {
    NTF_TRY(finish_mode(c, m, c->TL, src, c->Mbuf));
    NTF_TRY(enqueue_update(c, m, c->Mbuf, A[m], At[m], Y[m]));
  }
  NTF_CUDA(ntf::launch_fit(c->Mbuf, src[c->N - 1], c->dims[c->N - 1], c->R, c->grams, c->N,
                           c->fit_part, c->d_ctrl, c->st));
  c->launches += 2;
  return NTF_OK;
}

void free_ctx(ntf_ctx* c) {
  if (!c) return;
  if (c->graph) cudaGraphExecDestroy(c->graph);
  for (auto& pair : c->ev)
    for (auto& e : pair)
      if (e) cudaEventDestroy(e);
  cudaFree(c->partial);
  cudaFree(c->TR);
  cudaFree(c->TL);
  cudaFree(c->Mbuf);
  cudaFree(c->grams);
  cudaFree(c->grams_tmp);
  cudaFree(c->chol);
  cudaFree(c->norm_part);
  cudaFree(c->fit_part);
  cudaFree(c->dpart);
  cudaFree(c->d_ctrl);
  if (c->h_ctrl) cudaFreeHost(c->h_ctrl);
  delete c;
}

}  // namespace

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
  c->s = order / 2;
  c->P = 1;
  c->Q = 1;
  for (int m = 0; m < order; ++m) {
    c->dims[m] = dims[m];
    c->max_dim = std::max(c->max_dim, dims[m]);
    if (m < c->s) c->P *= dims[m];
    else c->Q *= dims[m];
  }
  if (c->P >= (int64_t{1} << 31) || c->Q >= (int64_t{1} << 31)) {
    delete c;
    return fail(NTF_ERR_UNSUPPORTED, "tensor halves must each have < 2^31 entries");
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    delete c;
    return fail(NTF_ERR_CUDA, "no CUDA device: %s", cudaGetErrorString(e));
  }
  const int R = rank;
  c->pn = ntf::plan_gemm_n(c->P, c->Q, R, dtype, d_tensor, c->num_sms);
  c->pt = ntf::plan_gemm_t(c->P, c->Q, R, dtype, d_tensor, c->num_sms);
  int64_t part = 0;
  if (c->pn.splits > 1) part = std::max<int64_t>(part, c->pn.splits * c->P * R);
  if (c->pt.splits > 1) part = std::max<int64_t>(part, c->pt.splits * c->Q * R);
  if (c->s == 2) {
    c->post_split_left = ntf::post_slow_splits(dims[0], dims[1], R, c->num_sms);
    part = std::max<int64_t>(part, c->post_split_left * dims[1] * R);
  }
  if (order - c->s == 2) {
    c->post_split_right = ntf::post_slow_splits(dims[c->s], dims[c->s + 1], R, c->num_sms);
    part = std::max<int64_t>(part, c->post_split_right * dims[c->s + 1] * R);
  }
  const int64_t RR = static_cast<int64_t>(R) * R;
  const int row_blocks = ntf::admm_row_blocks(c->max_dim);
  auto alloc = [&](void** ptr, size_t bytes) -> cudaError_t {
    return cudaMalloc(ptr, std::max<size_t>(bytes, 16));
  };
  e = cudaSuccess;
  if (e == cudaSuccess) e = alloc((void**)&c->partial, part * sizeof(float));
  if (e == cudaSuccess) e = alloc((void**)&c->TR, c->P * R * sizeof(float));
  if (e == cudaSuccess) e = alloc((void**)&c->TL, c->Q * R * sizeof(float));
  if (e == cudaSuccess) e = alloc((void**)&c->Mbuf, c->max_dim * R * sizeof(float));
  if (e == cudaSuccess) e = alloc((void**)&c->grams, order * RR * sizeof(double));
  if (e == cudaSuccess) e = alloc((void**)&c->grams_tmp, order * RR * sizeof(double));
  if (e == cudaSuccess) e = alloc((void**)&c->chol, order * RR * sizeof(double));
  if (e == cudaSuccess) e = alloc((void**)&c->norm_part, row_blocks * 5 * sizeof(double));
  if (e == cudaSuccess) e = alloc((void**)&c->fit_part, 64 * sizeof(double));
  if (e == cudaSuccess) e = alloc((void**)&c->dpart, 1024 * sizeof(double));
  if (e == cudaSuccess) e = alloc((void**)&c->d_ctrl, sizeof(Ctrl));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&c->h_ctrl, sizeof(Ctrl));
  if (e != cudaSuccess) {
    free_ctx(c);
    return fail(e == cudaErrorMemoryAllocation ? NTF_ERR_OOM : NTF_ERR_CUDA,
                "workspace allocation: %s", cudaGetErrorString(e));
  }
  std::memset(c->h_ctrl, 0, sizeof(Ctrl));
  for (int m = 0; m < order; ++m) c->h_ctrl->rho[m] = p->rho0;
  e = cudaMemcpyAsync(c->d_ctrl, c->h_ctrl, sizeof(Ctrl), cudaMemcpyHostToDevice, c->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->grams, 0, order * RR * sizeof(double), c->st);
  int64_t numel = c->P * c->Q;
  if (e == cudaSuccess)
    e = ntf::launch_norm2(d_tensor, dtype, numel, c->dpart, 1024, &c->d_ctrl->x_norm2, c->st);
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
    if (m != mode && !F[m]) return fail(NTF_ERR_INVALID_ARG, "null factor %d", m);
  if (mode < c->s) {
    float* T = c->s == 1 ? d_M : c->TR;
    NTF_TRY(contract_right(c, F, T));
    NTF_TRY(finish_mode(c, mode, T, F, d_M));
  } else {
    NTF_TRY(contract_left(c, F, c->TL));
    NTF_TRY(finish_mode(c, mode, c->TL, F, d_M));
  }
  return NTF_OK;
}

ntf_status ntf_gram(ntf_ctx* c, int mode, const float* d_F, double* d_G) {
  (void)cudaGetLastError();  // a stale non-sticky error is not this call's
  NTF_TRY(check_mode(c, mode));
  if (!d_F) return fail(NTF_ERR_INVALID_ARG, "null factor");
  const int64_t RR = static_cast<int64_t>(c->R) * c->R;
  double* G = c->grams + mode * RR;
  NTF_CUDA(ntf::launch_gram(d_F, c->dims[mode], c->R, G, c->st));
  if (d_G) NTF_CUDA(cudaMemcpyAsync(d_G, G, RR * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
  return NTF_OK;
}

ntf_status ntf_system(ntf_ctx* c, int mode, double* d_H, double* d_L, double* rho_out) {
  (void)cudaGetLastError();  // a stale non-sticky error is not this call's
  NTF_TRY(check_mode(c, mode));
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
  NTF_TRY(enqueue_update(c, mode, d_M, d_A, d_At, d_Y));
  if (!stats) return NTF_OK;
  NTF_TRY(read_ctrl(c));
  const double* s = c->h_ctrl->stats[mode];
  stats->primal_res = s[0];
  stats->dual_res = s[1];
  stats->norm_A = s[2];
  stats->norm_At = s[3];
  stats->norm_Y = s[4];
  stats->rho = s[5];
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
    if (!F[m]) return fail(NTF_ERR_INVALID_ARG, "null factor %d", m);
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

ntf_status ntf_fit_from_mttkrp(ntf_ctx* c, const float* d_M_last, const float* d_F_last,
                               double* rel_err) {
  if (!c || !d_M_last || !d_F_last || !rel_err) return fail(NTF_ERR_INVALID_ARG, "null argument");
  NTF_CUDA(ntf::launch_fit(d_M_last, d_F_last, c->dims[c->N - 1], c->R, c->grams, c->N,
                           c->fit_part, c->d_ctrl, c->st));
  NTF_TRY(read_ctrl(c));
  *rel_err = c->h_ctrl->rel_err;
  return take_status(c);
}

ntf_status ntf_profile_enable(ntf_ctx* c, int enable) {
  if (!c) return fail(NTF_ERR_INVALID_ARG, "null context");
  if (enable)
    for (auto& pair : c->ev)
      for (auto& e : pair)
        if (!e) NTF_CUDA(cudaEventCreate(&e));
  c->prof = enable != 0;
  c->pr = ntf_profile{};
  c->ev_pending[0] = c->ev_pending[1] = false;
  c->launches = 0;
  const double esize = c->dtype == NTF_BF16 ? 2.0 : 4.0;
  c->pr.contraction_bytes[0] = c->pr.contraction_bytes[1] =
      static_cast<double>(c->P) * static_cast<double>(c->Q) * esize;
  return NTF_OK;
}

ntf_status ntf_profile_get(ntf_ctx* c, ntf_profile* out) {
  if (!c || !out) return fail(NTF_ERR_INVALID_ARG, "null argument");
  *out = c->pr;
  out->kernel_launches = c->launches;
  return NTF_OK;
}

ntf_status ntf_sync(ntf_ctx* c) {
  if (!c) return fail(NTF_ERR_INVALID_ARG, "null context");
  NTF_TRY(read_ctrl(c));
  return take_status(c);
}

ntf_status ntf_run(ntf_ctx* c, float* const* A, float* const* At, float* const* Y, int max_outer,
                   double target_rfe, int check_every, double* rfe_hist, ntf_run_stats* out) {
  (void)cudaGetLastError();  // a stale non-sticky error is not this call's
  if (!c || !A || !At || !Y) return fail(NTF_ERR_INVALID_ARG, "null argument");
  if (max_outer < 1) return fail(NTF_ERR_INVALID_ARG, "max_outer must be >= 1");
  if (check_every < 1) check_every = 1;
  for (int m = 0; m < c->N; ++m)
    if (!A[m] || !At[m] || !Y[m]) return fail(NTF_ERR_INVALID_ARG, "null state of factor %d", m);
  const bool use_res = c->prm.eps_abs > 0.0 || c->prm.eps_rel > 0.0;
  const bool use_tgt = target_rfe > 0.0;
  if (rfe_hist)
    for (int i = 0; i < max_outer; ++i) rfe_hist[i] = NAN;
  const float* const* src = c->prm.kr_source == NTF_KR_AUX ? At : A;
  const int64_t RR = static_cast<int64_t>(c->R) * c->R;
  for (int m = 0; m < c->N; ++m)
    NTF_CUDA(ntf::launch_gram(src[m], c->dims[m], c->R, c->grams + m * RR, c->st));

  // The sweep is recorded once as a CUDA graph (after one eager sweep has set every kernel
  // attribute) and replayed; it is re-recorded only if the state pointers change.
  bool same = c->graph != nullptr && c->graph_prof == c->prof;
  for (int m = 0; m < c->N && same; ++m)
    same = c->graph_key[3 * m] == A[m] && c->graph_key[3 * m + 1] == At[m] &&
           c->graph_key[3 * m + 2] == Y[m];
  ntf_run_stats rs{};
  rs.rel_err = NAN;
  ntf_status result = NTF_OK;
  bool done = false;
  // Capture needs a non-legacy stream; otherwise (or if capture fails) launch eagerly.
  bool can_graph = c->st != nullptr;
  for (int it = 0; it < max_outer && !done; ++it) {
    if (same) {
      NTF_CUDA(cudaGraphLaunch(c->graph, c->st));
      c->launches += c->graph_launches;
    } else if (it == 0 || !can_graph) {
      NTF_TRY(enqueue_sweep(c, A, At, Y));
    } else {
      if (c->graph) {
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
      }
      cudaGraph_t g = nullptr;
      const int64_t before = c->launches;
      bool ok = cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      ntf_status sw = ok ? enqueue_sweep(c, A, At, Y) : NTF_OK;
      c->graph_launches = static_cast<int>(c->launches - before);
      c->launches = before;
      if (ok) ok = cudaStreamEndCapture(c->st, &g) == cudaSuccess && sw == NTF_OK;
      if (ok) ok = cudaGraphInstantiate(&c->graph, g, 0) == cudaSuccess;
      if (g) cudaGraphDestroy(g);
      if (!ok) {
        (void)cudaGetLastError();
        if (c->graph) cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
        can_graph = false;
        NTF_TRY(enqueue_sweep(c, A, At, Y));
      } else {
        c->graph_prof = c->prof;
        for (int m = 0; m < c->N; ++m) {
          c->graph_key[3 * m] = A[m];
          c->graph_key[3 * m + 1] = At[m];
          c->graph_key[3 * m + 2] = Y[m];
        }
        same = true;
        NTF_CUDA(cudaGraphLaunch(c->graph, c->st));
        c->launches += c->graph_launches;
      }
    }
    if (c->prof) c->pr.sweeps += 1;
    rs.iters = it + 1;
    const bool check = ((it + 1) % check_every == 0) || it + 1 == max_outer;
    if (!check) continue;
    NTF_TRY(read_ctrl(c));
    prof_collect(c);
    NTF_TRY(take_status(c));
    rs.rel_err = c->h_ctrl->rel_err;
    if (rfe_hist) rfe_hist[it] = rs.rel_err;
    if (use_tgt && rs.rel_err <= target_rfe) {
      rs.reached_target = 1;
      done = true;
    }
    if (use_res) {
      bool all = true;
      for (int m = 0; m < c->N && all; ++m) {
        const double* s = c->h_ctrl->stats[m];
        const double base = std::sqrt(static_cast<double>(c->dims[m]) * c->R) * c->prm.eps_abs;
        all = s[0] <= base + c->prm.eps_rel * std::max(s[2], s[3]) &&
              s[1] <= base + c->prm.eps_rel * s[4];
      }
      if (all) {
        rs.converged = 1;
        done = true;
      }
    }
  }
  if (!done && (use_res || use_tgt)) result = NTF_ERR_NOT_CONVERGED;
  if (out) *out = rs;
  if (result != NTF_OK) fail(result, "no stopping criterion met in %d iterations", max_outer);
  return result;
}

ntf_status ntf_to_bf16(const float* d_in, uint16_t* d_out, int64_t n, void* stream) {
  if (!d_in || !d_out || n < 0) return fail(NTF_ERR_INVALID_ARG, "bad argument");
  if (n == 0) return NTF_OK;
  NTF_CUDA(ntf::launch_to_bf16(d_in, d_out, n, static_cast<cudaStream_t>(stream)));
  return NTF_OK;
}

}  // extern "C"
