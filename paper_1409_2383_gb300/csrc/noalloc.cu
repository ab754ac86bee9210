// ntf_mttkrp_noalloc: the MTTKRP of ntf_mttkrp for callers that cannot allocate device
// memory.  Its scratch (split-K partial sums and the contraction intermediate) lives in one
// file-scope device array instead of a context workspace, and no context is created.
#include <algorithm>
#include <mutex>

#include "ntf_internal.cuh"

// 32 MiB of FP32 scratch.  Every GPU that loads the library holds this array until the
// process exits; all calls on a device share it.
static constexpr int64_t kScratchFloats = int64_t{8} << 20;
static __device__ __align__(256) float g_scratch[kScratchFloats];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
float* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_scratch on the current device.  In host code the symbol is a host-side
// stand-in, so the address is looked up once per device (with that device current) and
// cached.
ntf_status scratch_on_current_device(float** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return NTF_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return NTF_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) return NTF_ERR_CUDA;
    g_scratch_ptr[dev] = static_cast<float*>(p);
  }
  *out = g_scratch_ptr[dev];
  return NTF_OK;
}

}  // namespace

extern "C" ntf_status ntf_mttkrp_noalloc(int order, const int64_t* dims, int rank, int dtype,
                                         const void* d_tensor, int mode,
                                         const float* const* d_factors, float* d_M,
                                         void* stream) {
  if (order < 3 || order > ntf::kMaxOrder || !dims || rank < 1 || rank > ntf::kMaxRank ||
      (dtype != NTF_F32 && dtype != NTF_BF16) || !d_tensor || !d_factors || !d_M || mode < 0 ||
      mode >= order)
    return NTF_ERR_INVALID_ARG;
  for (int m = 0; m < order; ++m) {
    if (dims[m] < 1 || dims[m] > (int64_t{1} << 30)) return NTF_ERR_INVALID_ARG;
    if (m != mode && !d_factors[m]) return NTF_ERR_INVALID_ARG;
  }
  const int s = order / 2;
  int64_t P = 1, Q = 1;
  for (int m = 0; m < order; ++m) (m < s ? P : Q) *= dims[m];
  if (P >= (int64_t{1} << 31) || Q >= (int64_t{1} << 31)) return NTF_ERR_UNSUPPORTED;
  const int R = rank;
  const bool left = mode < s;
  const int first = left ? 0 : s;
  const int count = left ? s : order - s;
  const int64_t rows = left ? P : Q;  // rows of the contraction output T
  // The contraction output goes straight to d_M when the mode's group has one mode;
  // otherwise it is an intermediate in scratch.
  const int64_t t_floats = count == 1 ? 0 : rows * R;

  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return NTF_ERR_CUDA;
  ntf::GemmPlan plan = left ? ntf::plan_gemm_n(P, Q, R, dtype, d_tensor, sms)
                            : ntf::plan_gemm_t(P, Q, R, dtype, d_tensor, sms);
  // The intermediate must fit in the scratch array; split-K partial sums use what is left
  // (fewer splits when the full plan would not fit).
  const int64_t room = kScratchFloats - t_floats;
  if (room < 0) return NTF_ERR_INVALID_ARG;
  if (plan.splits > 1 && plan.splits * rows * R > room)
    plan.splits = static_cast<int>(std::max<int64_t>(1, room / (rows * R)));
  int post_splits = 1;
  if (count == 2 && mode != first) {
    post_splits = ntf::post_slow_splits(dims[first], dims[first + 1], R, sms);
    const int64_t need = post_splits * dims[first + 1] * R;
    if (need > room)
      post_splits = static_cast<int>(std::max<int64_t>(1, room / (dims[first + 1] * R)));
  }

  float* scratch = nullptr;
  ntf_status st = scratch_on_current_device(&scratch);
  if (st != NTF_OK) return st;
  float* T = count == 1 ? d_M : scratch;
  float* part = scratch + t_floats;

  ntf::Group g{};
  const int gfirst = left ? s : 0;
  const int gcount = left ? order - s : s;
  g.n = gcount;
  for (int j = 0; j < gcount; ++j) {
    g.F[j] = d_factors[gfirst + j];
    g.dim[j] = static_cast<int>(dims[gfirst + j]);
  }
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  (void)cudaGetLastError();
  float* out = plan.splits > 1 ? part : T;
  e = left ? ntf::launch_gemm_n(d_tensor, dtype, P, Q, R, g, plan, out, cs)
           : ntf::launch_gemm_t(d_tensor, dtype, P, Q, R, g, plan, out, cs);
  if (e == cudaSuccess && plan.splits > 1)
    e = ntf::launch_sum_splits(part, plan.splits, rows * R, T, cs);
  if (e == cudaSuccess && count == 2) {
    const int64_t Ia = dims[first], Ib = dims[first + 1];
    if (mode == first)
      e = ntf::launch_post_fast(T, Ia, Ib, R, d_factors[first + 1], d_M, cs);
    else
      e = ntf::launch_post_slow(T, Ia, Ib, R, d_factors[first], post_splits, part, d_M, cs);
  }
  if (e != cudaSuccess) return NTF_ERR_CUDA;
  return NTF_OK;
}
