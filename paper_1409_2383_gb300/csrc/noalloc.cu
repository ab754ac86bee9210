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

// The device that `p` lives on, if it is device (or managed) memory of that device; -1 for
// host memory, memory of no CUDA allocation, or a failed query.  cudaPointerGetAttributes
// allocates nothing.
int device_of(const void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return -1;
  }
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) return -1;
  return at.device;
}

}  // namespace

extern "C" ntf_status ntf_mttkrp_noalloc(int order, const int64_t* dims, int rank, int dtype,
                                         const void* d_tensor, int mode,
                                         const float* const* d_factors, float* d_M,
                                         void* stream) {
  using ntf::record_error;
  if (order < 3 || order > ntf::kMaxOrder || !dims || rank < 1 || rank > ntf::kMaxRank ||
      (dtype != NTF_F32 && dtype != NTF_BF16) || !d_tensor || !d_factors || !d_M || mode < 0 ||
      mode >= order)
    return record_error(NTF_ERR_INVALID_ARG,
                        "ntf_mttkrp_noalloc: invalid order, rank, dtype, mode or null pointer");
  // device arrays are read with loads of their element type: pointers must be multiples of it
  const auto misaligned = [](const void* p, uintptr_t elem) {
    return reinterpret_cast<uintptr_t>(p) % elem != 0;
  };
  if (misaligned(d_tensor, dtype == NTF_BF16 ? 2 : 4) || misaligned(d_M, 4))
    return record_error(NTF_ERR_INVALID_ARG, "ntf_mttkrp_noalloc: misaligned tensor or output");
  for (int m = 0; m < order; ++m) {
    if (dims[m] < 1 || dims[m] > (int64_t{1} << 30))
      return record_error(NTF_ERR_INVALID_ARG, "ntf_mttkrp_noalloc: dims[%d] out of range", m);
    if (m != mode && (!d_factors[m] || misaligned(d_factors[m], 4)))
      return record_error(NTF_ERR_INVALID_ARG,
                          "ntf_mttkrp_noalloc: factor %d is null or misaligned", m);
  }
  // The same two contractions as the context path: the leading factors' modes come from
  // X[P_R, Q_R] * KR(trailing factors), the others from X[P_L, Q_L]^T * KR(leading factors).
  const int s_R = 2, s_L = order == 3 ? 1 : 2;
  // each half is a product of at most two dims (<= 2^60): no overflow before the check
  int64_t P_R = 1, Q_R = 1, P_L = 1, Q_L = 1;
  for (int m = 0; m < order; ++m) {
    (m < s_R ? P_R : Q_R) *= dims[m];
    (m < s_L ? P_L : Q_L) *= dims[m];
  }
  if (P_R >= (int64_t{1} << 31) || Q_R >= (int64_t{1} << 31) || P_L >= (int64_t{1} << 31) ||
      Q_L >= (int64_t{1} << 31))
    return record_error(NTF_ERR_UNSUPPORTED,
                        "ntf_mttkrp_noalloc: a matrix view of the tensor has 2^31 or more "
                        "entries");
  const int R = rank;
  const bool left = mode < s_R;
  const int first = left ? 0 : s_L;
  const int count = left ? s_R : order - s_L;
  const int64_t rows = left ? P_R : Q_L;   // rows of the contraction output T
  const int64_t K = left ? Q_R : P_L;      // contraction length
  const int64_t w_floats = ntf::kr_rows_padded(K) * ntf::round_rp(R);
  // The contraction output goes straight to d_M when the mode's group has one mode;
  // otherwise it is an intermediate in scratch, after the Khatri-Rao table.
  const int64_t t_floats = count == 1 ? 0 : rows * R;
  const int64_t room = kScratchFloats - w_floats - t_floats;
  if (room < 0)
    return record_error(NTF_ERR_INVALID_ARG,
                        "ntf_mttkrp_noalloc: mode %d needs %lld scratch floats (Khatri-Rao "
                        "table %lld + intermediate %lld), more than the %lld of the static "
                        "scratch array",
                        mode, static_cast<long long>(w_floats + t_floats),
                        static_cast<long long>(w_floats), static_cast<long long>(t_floats),
                        static_cast<long long>(kScratchFloats));

  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess)
    return record_error(NTF_ERR_CUDA, "ntf_mttkrp_noalloc: %s", cudaGetErrorString(e));
  // every array the kernels touch must be memory of the current device: the kernels run there
  if (device_of(d_tensor) != dev || device_of(d_M) != dev)
    return record_error(NTF_ERR_INVALID_ARG,
                        "ntf_mttkrp_noalloc: the tensor and the output must be device memory "
                        "of the current device (%d)", dev);
  for (int m = 0; m < order; ++m)
    if (m != mode && device_of(d_factors[m]) != dev)
      return record_error(NTF_ERR_INVALID_ARG,
                          "ntf_mttkrp_noalloc: factor %d is not device memory of the current "
                          "device (%d)", m, dev);
  ntf::GemmPlan plan = left ? ntf::plan_gemm_n(P_R, Q_R, dtype, d_tensor, sms)
                            : ntf::plan_gemm_t(P_L, Q_L, dtype, d_tensor, sms);
  // Partial sums of a split contraction range use what is left of the scratch; when they do
  // not fit, the range is not split.
  if (plan.chunks > 1 && plan.chunks * rows * R > room) {
    plan.chunks = 1;
    plan.chunk_len = K;
  }
  int post_splits = 1;
  if (count == 2 && mode != first) {
    post_splits = ntf::post_slow_splits(dims[first], dims[first + 1], R, sms);
    const int64_t need = post_splits * dims[first + 1] * R;
    if (need > room)
      post_splits = static_cast<int>(std::max<int64_t>(1, room / (dims[first + 1] * R)));
  }

  float* scratch = nullptr;
  ntf_status st = scratch_on_current_device(&scratch);
  if (st != NTF_OK)
    return record_error(st, "ntf_mttkrp_noalloc: the scratch array's device address was not "
                            "found on device %d", dev);
  float* W = scratch;
  float* T = count == 1 ? d_M : scratch + w_floats;
  float* part = scratch + w_floats + t_floats;

  ntf::Group g{};
  const int gfirst = left ? s_R : 0;
  const int gcount = left ? order - s_R : s_L;
  g.n = gcount;
  for (int j = 0; j < gcount; ++j) {
    g.F[j] = d_factors[gfirst + j];
    g.dim[j] = static_cast<int>(dims[gfirst + j]);
  }
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  (void)cudaGetLastError();
  e = ntf::launch_kr_table(g, K, R, W, cs);
  float* out = plan.chunks > 1 ? part : T;
  if (e == cudaSuccess)
    e = left ? ntf::launch_gemm_n(d_tensor, dtype, P_R, Q_R, R, W, plan, out, cs)
             : ntf::launch_gemm_t(d_tensor, dtype, P_L, Q_L, R, W, plan, out, cs);
  if (e == cudaSuccess && plan.chunks > 1)
    e = ntf::launch_sum_splits(part, plan.chunks, rows * R, T, cs);
  if (e == cudaSuccess && count == 2) {
    const int64_t Ia = dims[first], Ib = dims[first + 1];
    if (mode == first)
      e = ntf::launch_post_fast(T, Ia, Ib, R, d_factors[first + 1], d_M, cs);
    else
      e = ntf::launch_post_slow(T, Ia, Ib, R, d_factors[first], post_splits, part, d_M, cs);
  }
  if (e != cudaSuccess)
    return record_error(NTF_ERR_CUDA, "ntf_mttkrp_noalloc: launch failed: %s",
                        cudaGetErrorString(e));
  return NTF_OK;
}
