// C ABI of the warm-start network (include/ntf.h, ntf_mlp_*): parameters, forward, one
// training step, and attaching a network to a factorization context.
#include <cstring>
#include <string>

#include "ntf_internal.cuh"

struct ntf_mlp {
  ntf::MlpShape s{};
  cudaStream_t st = nullptr;
  int max_rows = 0, max_groups = 0, step = 0;
  float* p = nullptr;            // FP32 master parameters
  __nv_bfloat16* pb = nullptr;   // BF16 copies used in the products
  float* m = nullptr;            // Adam moments
  float* v = nullptr;
  float* grad = nullptr;
  float *z1 = nullptr, *h1 = nullptr, *z2 = nullptr, *h2 = nullptr;
  float *out = nullptr, *d_out = nullptr, *d_h2 = nullptr, *d_h1 = nullptr;
  float* hG = nullptr;           // [max_groups, H]
  float* gsum = nullptr;         // [max_groups, H]
  int* row_group = nullptr;      // [max_rows]
  int* all_offs = nullptr;       // {0, rows}
  float* Gn = nullptr;           // warm start: normalised G [R^2]
  float* mrows = nullptr;        // warm start: per-row inputs [max_rows, 2R]
  float* s_dev = nullptr;        // warm start: scale
  double* loss_part = nullptr;   // [64]
  double* loss_dev = nullptr;
  double* loss_host = nullptr;   // pinned
};

namespace {

thread_local std::string g_mlp_err;

ntf_status mfail(ntf_status s, const char* msg, cudaError_t e = cudaSuccess) {
  g_mlp_err = msg;
  if (e != cudaSuccess) {
    g_mlp_err += ": ";
    g_mlp_err += cudaGetErrorString(e);
  }
  return s;
}

#define MLP_CUDA(call)                                                              \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess)                                                          \
      return mfail(e_ == cudaErrorMemoryAllocation ? NTF_ERR_OOM : NTF_ERR_CUDA, #call, e_); \
  } while (0)

void mlp_free(ntf_mlp* n) {
  if (!n) return;
  for (void* q : {(void*)n->p, (void*)n->pb, (void*)n->m, (void*)n->v, (void*)n->grad,
                  (void*)n->z1, (void*)n->h1, (void*)n->z2, (void*)n->h2, (void*)n->out,
                  (void*)n->d_out, (void*)n->d_h2, (void*)n->d_h1, (void*)n->hG, (void*)n->gsum,
                  (void*)n->row_group, (void*)n->all_offs, (void*)n->Gn, (void*)n->mrows,
                  (void*)n->s_dev, (void*)n->loss_part, (void*)n->loss_dev})
    cudaFree(q);
  if (n->loss_host) cudaFreeHost(n->loss_host);
  delete n;
}

// Device arrays are read with loads of their element type (4 bytes here) at least.
bool misaligned4(const void* p) { return reinterpret_cast<uintptr_t>(p) % 4 != 0; }

ntf_status check_batch(const ntf_mlp* n, int groups, int rows) {
  if (!n) return mfail(NTF_ERR_INVALID_ARG, "null network");
  if (groups < 1 || groups > n->max_groups || rows < 1 || rows > n->max_rows)
    return mfail(NTF_ERR_INVALID_ARG, "groups or rows outside the sizes given at creation");
  return NTF_OK;
}

// Forward for a batch given as normalised coefficient matrices Gn [groups, R^2], CSR offsets
// (rows of a group contiguous) and per-row inputs [rows, 2R] = [m/s ; z].
ntf_status forward_batch(ntf_mlp* n, const float* Gn, const int* offs, int groups,
                         const float* mrows, int rows, cudaStream_t st) {
  MLP_CUDA(ntf::mlp_row_groups(offs, groups, n->row_group, st));
  MLP_CUDA(ntf::mlp_group_terms(n->s, n->pb, Gn, groups, n->hG, st));
  MLP_CUDA(ntf::mlp_forward_rows(n->s, n->p, n->pb, n->hG, n->row_group, mrows, rows, n->z1,
                                 n->h1, n->z2, n->h2, n->out, st));
  return NTF_OK;
}

}  // namespace

namespace ntf {
// Warm start of factor `mode` before its inner iterations (called by the context).
cudaError_t mlp_warm_start(ntf_mlp* n, const double* sys, int mode, const float* M, float* At,
                           float* Y, int64_t I, unsigned long long* counters, cudaStream_t st) {
  const int R = n->s.R;
  const float* G = update_sys_h32(sys, mode, R);
  if (ws_fused_ok(n->s))
    return ws_fused(n->s, n->p, n->pb, n->hG, G, update_sys_hinv32(sys, mode, R), M, At, Y, I,
                    counters, st);
  cudaError_t e = ws_prepare(G, update_sys_hinv32(sys, mode, R), M, R, I, n->Gn, n->mrows,
                             n->s_dev, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->row_group, 0, I * sizeof(int), st);
  if (e == cudaSuccess) e = mlp_group_terms(n->s, n->pb, n->Gn, 1, n->hG, st);
  if (e == cudaSuccess)
    e = mlp_forward_rows(n->s, n->p, n->pb, n->hG, n->row_group, n->mrows, static_cast<int>(I),
                         n->z1, n->h1, n->z2, n->h2, n->out, st);
  if (e == cudaSuccess) e = ws_judge(n->out, G, M, n->s_dev, At, Y, I, R, counters, st);
  return e;
}
int mlp_rank(const ntf_mlp* n) { return n->s.R; }
int mlp_ws_launches(const ntf_mlp* n) { return ws_fused_ok(n->s) ? 2 : 9; }
int mlp_max_rows(const ntf_mlp* n) { return n->max_rows; }
}  // namespace ntf

extern "C" {

int64_t ntf_mlp_param_count(int rank, int hidden) {
  if (rank < 1 || rank > ntf::kMaxRank || hidden < 1) return -1;
  return ntf::mlp_shape(rank, hidden).count;
}

ntf_status ntf_mlp_create(ntf_mlp** out, int rank, int hidden, const float* h_params,
                          int max_rows, int max_groups, void* stream) {
  if (!out) return mfail(NTF_ERR_INVALID_ARG, "null output pointer");
  *out = nullptr;
  if (rank < 1 || rank > ntf::kMaxRank || hidden < 1 || hidden > 4096 || !h_params ||
      max_rows < 1 || max_groups < 1)
    return mfail(NTF_ERR_INVALID_ARG, "bad rank, hidden width, sizes or parameters");
  ntf_mlp* n = new ntf_mlp();
  n->s = ntf::mlp_shape(rank, hidden);
  n->st = static_cast<cudaStream_t>(stream);
  n->max_rows = max_rows;
  n->max_groups = max_groups;
  const int64_t cnt = n->s.count, H = hidden, D = n->s.Dout, R = rank;
  cudaError_t e = cudaSuccess;
  auto A = [&](void** q, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(q, bytes < 16 ? 16 : bytes);
  };
  A((void**)&n->p, cnt * 4);
  A((void**)&n->pb, cnt * 2);
  A((void**)&n->m, cnt * 4);
  A((void**)&n->v, cnt * 4);
  A((void**)&n->grad, cnt * 4);
  for (float** q : {&n->z1, &n->h1, &n->z2, &n->h2, &n->d_h2, &n->d_h1})
    A((void**)q, static_cast<size_t>(max_rows) * H * 4);
  A((void**)&n->out, static_cast<size_t>(max_rows) * D * 4);
  A((void**)&n->d_out, static_cast<size_t>(max_rows) * D * 4);
  A((void**)&n->hG, static_cast<size_t>(max_groups) * H * 4);
  A((void**)&n->gsum, static_cast<size_t>(max_groups) * H * 4);
  A((void**)&n->row_group, static_cast<size_t>(max_rows) * 4);
  A((void**)&n->all_offs, 2 * 4);
  A((void**)&n->Gn, R * R * 4);
  A((void**)&n->mrows, static_cast<size_t>(max_rows) * 2 * R * 4);
  A((void**)&n->s_dev, 4);
  A((void**)&n->loss_part, 64 * 8);
  A((void**)&n->loss_dev, 8);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&n->loss_host, 8);
  if (e == cudaSuccess) e = cudaMemcpyAsync(n->p, h_params, cnt * 4, cudaMemcpyHostToDevice, n->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->m, 0, cnt * 4, n->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->v, 0, cnt * 4, n->st);
  if (e == cudaSuccess) e = ntf::mlp_refresh_bf16(n->s, n->p, n->pb, n->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(n->st);
  if (e != cudaSuccess) {
    mlp_free(n);
    return mfail(e == cudaErrorMemoryAllocation ? NTF_ERR_OOM : NTF_ERR_CUDA, "network setup", e);
  }
  *out = n;
  return NTF_OK;
}

ntf_status ntf_mlp_destroy(ntf_mlp* n) {
  if (n) {
    cudaStreamSynchronize(n->st);
    mlp_free(n);
  }
  return NTF_OK;
}

ntf_status ntf_mlp_get_params(ntf_mlp* n, float* h_params) {
  if (!n || !h_params) return mfail(NTF_ERR_INVALID_ARG, "null argument");
  MLP_CUDA(cudaMemcpyAsync(h_params, n->p, n->s.count * 4, cudaMemcpyDeviceToHost, n->st));
  MLP_CUDA(cudaStreamSynchronize(n->st));
  return NTF_OK;
}

ntf_status ntf_mlp_forward(ntf_mlp* n, const float* d_Gn, const int* d_offsets, int groups,
                           const float* d_mrows, int rows, float* d_out) {
  ntf_status s = check_batch(n, groups, rows);
  if (s != NTF_OK) return s;
  if (!d_Gn || !d_offsets || !d_mrows || !d_out) return mfail(NTF_ERR_INVALID_ARG, "null pointer");
  if (misaligned4(d_Gn) || misaligned4(d_offsets) || misaligned4(d_mrows) || misaligned4(d_out))
    return mfail(NTF_ERR_INVALID_ARG, "pointer not aligned to its element size");
  s = forward_batch(n, d_Gn, d_offsets, groups, d_mrows, rows, n->st);
  if (s != NTF_OK) return s;
  MLP_CUDA(cudaMemcpyAsync(d_out, n->out, static_cast<size_t>(rows) * n->s.Dout * 4,
                           cudaMemcpyDeviceToDevice, n->st));
  return NTF_OK;
}

ntf_status ntf_mlp_train_step(ntf_mlp* n, const float* d_Gn, const int* d_offsets, int groups,
                              const float* d_mrows, const float* d_targets, int rows, float lr,
                              int apply, double* loss, float* d_grad_out) {
  ntf_status s = check_batch(n, groups, rows);
  if (s != NTF_OK) return s;
  if (!d_Gn || !d_offsets || !d_mrows || !d_targets) return mfail(NTF_ERR_INVALID_ARG, "null pointer");
  if (misaligned4(d_Gn) || misaligned4(d_offsets) || misaligned4(d_mrows) ||
      misaligned4(d_targets) || misaligned4(d_grad_out))
    return mfail(NTF_ERR_INVALID_ARG, "pointer not aligned to its element size");
  s = forward_batch(n, d_Gn, d_offsets, groups, d_mrows, rows, n->st);
  if (s != NTF_OK) return s;
  const int offs_h[2] = {0, rows};
  MLP_CUDA(cudaMemcpyAsync(n->all_offs, offs_h, sizeof offs_h, cudaMemcpyHostToDevice, n->st));
  MLP_CUDA(ntf::mlp_backward(n->s, n->pb, d_Gn, d_offsets, groups, n->all_offs, d_mrows, rows,
                             d_targets, n->z1, n->h1, n->z2, n->h2, n->out, n->d_out, n->d_h2,
                             n->d_h1, n->gsum, n->grad, n->loss_part, n->loss_dev, n->st));
  if (d_grad_out)
    MLP_CUDA(cudaMemcpyAsync(d_grad_out, n->grad, n->s.count * 4, cudaMemcpyDeviceToDevice, n->st));
  if (apply) {
    n->step += 1;
    MLP_CUDA(ntf::mlp_adam(n->s, n->p, n->grad, n->m, n->v, n->pb, lr, n->step, n->st));
  }
  if (loss) {
    MLP_CUDA(cudaMemcpyAsync(n->loss_host, n->loss_dev, 8, cudaMemcpyDeviceToHost, n->st));
    MLP_CUDA(cudaStreamSynchronize(n->st));
    *loss = *n->loss_host;
  }
  return NTF_OK;
}

const char* ntf_mlp_last_error(void) { return g_mlp_err.c_str(); }

}  // extern "C"
