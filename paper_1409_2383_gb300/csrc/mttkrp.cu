// MTTKRP building blocks (Sec. III-A item 1 of Liavas & Sidiropoulos).
//
// The tensor is viewed as a row-major matrix X[P, Q] with P = I_1...I_s and Q =
// I_{s+1}...I_N.  Every MTTKRP is one of two skinny contractions of that matrix followed by
// a small reduction that applies the remaining factor of the mode's group:
//
//   GEMM-N:  T_R[p, r] = sum_q X[p, q] * KR_right[q, r]   (modes 1..s)
//   GEMM-T:  T_L[q, r] = sum_p X[p, q] * KR_left[p, r]    (modes s+1..N)
//
// KR_* rows are Khatri-Rao rows of the group's factors, built on the fly in shared memory
// for each stage and never materialised.  Both contractions stream X from HBM exactly once;
// X tiles are staged with 16-byte cp.async in a multi-stage ring; FP32 accumulation for FP32
// and BF16 storage alike.  Split-K partial sums are reduced by a separate kernel in a fixed
// order, so results are deterministic.
#include <algorithm>
#include <cstdio>

#include "mttkrp_kernels.cuh"

namespace ntf {
namespace detail {
// One instantiation unit per storage type and contraction (gemm_{n,t}_{f32,bf16}.cu).
extern template cudaError_t gemm_n_typed<float>(const float*, int64_t, int64_t, int,
                                                const Group&, const GemmPlan&, float*, cudaStream_t);
extern template cudaError_t gemm_n_typed<__nv_bfloat16>(const __nv_bfloat16*, int64_t, int64_t,
                                                        int, const Group&, const GemmPlan&,
                                                        float*, cudaStream_t);
extern template cudaError_t gemm_t_typed<float>(const float*, int64_t, int64_t, int,
                                                const Group&, const GemmPlan&, float*, cudaStream_t);
extern template cudaError_t gemm_t_typed<__nv_bfloat16>(const __nv_bfloat16*, int64_t, int64_t,
                                                        int, const Group&, const GemmPlan&,
                                                        float*, cudaStream_t);
}  // namespace detail

namespace {
using namespace detail;
// --------------------------------------------------------------------- reductions
__global__ void k_sum_splits(const float* __restrict__ part, int splits, int64_t n,
                             float* __restrict__ out) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    float s = 0.0f;
    for (int k = 0; k < splits; ++k) s += part[k * n + i];
    out[i] = s;
  }
}

// out[a, r] = sum_b T[a, b, r] * F[b, r]: one CTA per a; thread t handles column r = t % R
// for the b's of its lane group; groups are summed in a fixed order.
__global__ void k_post_fast(const float* __restrict__ T, int64_t Ia, int64_t Ib, int R,
                            const float* __restrict__ F, float* __restrict__ out) {
  __shared__ float red[256];
  const int tid = threadIdx.x;
  const int groups = blockDim.x / R;
  const int grp = tid / R, r = tid % R;
  for (int64_t a = blockIdx.x; a < Ia; a += gridDim.x) {
    float s = 0.0f;
    if (grp < groups) {
      const float* Ta = T + a * Ib * R;
      for (int64_t b = grp; b < Ib; b += groups) s = fmaf(Ta[b * R + r], __ldg(F + b * R + r), s);
    }
    red[tid] = s;
    __syncthreads();
    if (tid < R) {
      float acc = 0.0f;
      for (int k = 0; k < groups; ++k) acc += red[k * R + tid];
      out[a * R + tid] = acc;
    }
    __syncthreads();
  }
}

// out[b, r] = sum_a T[a, b, r] * F[a, r]: CTA (split, b-block of 256/R rows); thread t
// handles (b, r) = (b0 + t / R, t % R) over its split's a-range.
__global__ void k_post_slow(const float* __restrict__ T, int64_t Ia, int64_t Ib, int R,
                            const float* __restrict__ F, int splits, float* __restrict__ out) {
  const int bpb = blockDim.x / R;
  const int tid = threadIdx.x;
  if (tid >= bpb * R) return;
  const int split = blockIdx.x;
  const int64_t b = static_cast<int64_t>(blockIdx.y) * bpb + tid / R;
  const int r = tid % R;
  if (b >= Ib) return;
  const int64_t a_beg = Ia * split / splits, a_end = Ia * (split + 1) / splits;
  float s = 0.0f;
  for (int64_t a = a_beg; a < a_end; ++a) s = fmaf(T[(a * Ib + b) * R + r], __ldg(F + a * R + r), s);
  out[(static_cast<int64_t>(split) * Ib + b) * R + r] = s;
}

// ||X||^2 with FP64 accumulation; per-block partials then one block sums them in order.
template <typename T>
__global__ void k_norm2(const T* __restrict__ X, int64_t n, double* __restrict__ partial) {
  __shared__ double red[256];
  double s = 0.0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const double v = static_cast<double>(Elem<T>::load1(X + i));
    s = fma(v, v, s);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void k_sum_doubles(const double* __restrict__ v, int n, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += v[i];
    *out = s;
  }
}

__global__ void k_to_bf16(const float* __restrict__ in, __nv_bfloat16* __restrict__ out,
                          int64_t n) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    out[i] = __float2bfloat16_rn(in[i]);
}

}  // namespace

// ------------------------------------------------------------------------- plans
GemmPlan plan_gemm_n(int64_t P, int64_t Q, int R, int dtype, const void* X, int num_sms) {
  GemmPlan pl{};
  const int esize = dtype == NTF_BF16 ? 2 : 4;
  pl.vec16 = (Q * esize) % 16 == 0 && (reinterpret_cast<uintptr_t>(X) % 16) == 0;
  const int64_t max_rows = 512;
  const int64_t nblk = (P + max_rows - 1) / max_rows;
  pl.rows_per_blk = static_cast<int>((P + nblk - 1) / nblk);
  pl.blocks = static_cast<int>(nblk);
  const int per16 = 16 / esize;
  const int64_t ntiles = (Q + 2 * per16 - 1) / (2 * per16);
  const int64_t target = static_cast<int64_t>(num_sms) * 2;
  int64_t splits = (target + nblk - 1) / nblk;
  splits = std::max<int64_t>(1, std::min<int64_t>(splits, ntiles));
  if (!pl.vec16) splits = std::max<int64_t>(1, std::min<int64_t>(Q / 64, 64));
  pl.splits = static_cast<int>(splits);
  return pl;
}

GemmPlan plan_gemm_t(int64_t P, int64_t Q, int R, int dtype, const void* X, int num_sms) {
  GemmPlan pl{};
  const int esize = dtype == NTF_BF16 ? 2 : 4;
  pl.vec16 = (Q * esize) % 16 == 0 && (reinterpret_cast<uintptr_t>(X) % 16) == 0;
  const int cols = round_rp(R) <= 32 ? 512 : 256;
  const int64_t nblk = (Q + cols - 1) / cols;
  pl.blocks = static_cast<int>(nblk);
  pl.rows_per_blk = 0;
  const int64_t target = static_cast<int64_t>(num_sms) * 2;
  int64_t splits = nblk >= target ? 1 : (target + nblk - 1) / nblk;
  const int64_t tp = 8192 / (cols * esize);
  splits = std::max<int64_t>(1, std::min<int64_t>(splits, (P + tp - 1) / tp));
  if (!pl.vec16) {
    pl.blocks = 0;
    splits = std::max<int64_t>(1, std::min<int64_t>(P / 64, 64));
  }
  pl.splits = static_cast<int>(splits);
  return pl;
}

cudaError_t launch_gemm_n(const void* X, int dtype, int64_t P, int64_t Q, int R, const Group& g,
                          const GemmPlan& plan, float* out, cudaStream_t st) {
  if (dtype == NTF_BF16)
    return gemm_n_typed(static_cast<const __nv_bfloat16*>(X), P, Q, R, g, plan, out, st);
  return gemm_n_typed(static_cast<const float*>(X), P, Q, R, g, plan, out, st);
}

cudaError_t launch_gemm_t(const void* X, int dtype, int64_t P, int64_t Q, int R, const Group& g,
                          const GemmPlan& plan, float* out, cudaStream_t st) {
  if (dtype == NTF_BF16)
    return gemm_t_typed(static_cast<const __nv_bfloat16*>(X), P, Q, R, g, plan, out, st);
  return gemm_t_typed(static_cast<const float*>(X), P, Q, R, g, plan, out, st);
}

cudaError_t launch_sum_splits(const float* partial, int splits, int64_t n, float* out,
                              cudaStream_t st) {
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 2048);
  k_sum_splits<<<static_cast<unsigned>(std::max<int64_t>(blocks, 1)), 256, 0, st>>>(partial, splits, n, out);
  return cudaGetLastError();
}

cudaError_t launch_post_fast(const float* T, int64_t Ia, int64_t Ib, int R, const float* F,
                             float* out, cudaStream_t st) {
  const unsigned blocks = static_cast<unsigned>(std::min<int64_t>(Ia, 65535));
  k_post_fast<<<blocks, 256, 0, st>>>(T, Ia, Ib, R, F, out);
  return cudaGetLastError();
}

int post_slow_splits(int64_t Ia, int64_t Ib, int R, int num_sms) {
  const int bpb = 256 / R;
  const int64_t bblocks = (Ib + bpb - 1) / bpb;
  int64_t splits = (static_cast<int64_t>(num_sms) * 4 + bblocks - 1) / bblocks;
  splits = std::max<int64_t>(1, std::min<int64_t>(splits, std::max<int64_t>(1, Ia / 8)));
  return static_cast<int>(splits);
}

cudaError_t launch_post_slow(const float* T, int64_t Ia, int64_t Ib, int R, const float* F,
                             int splits, float* partial, float* out, cudaStream_t st) {
  const int bpb = 256 / R;
  dim3 grid(splits, static_cast<unsigned>((Ib + bpb - 1) / bpb));
  float* dst = splits > 1 ? partial : out;
  k_post_slow<<<grid, 256, 0, st>>>(T, Ia, Ib, R, F, splits, dst);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || splits == 1) return e;
  return launch_sum_splits(partial, splits, Ib * R, out, st);
}

cudaError_t launch_norm2(const void* X, int dtype, int64_t n, double* partial, int blocks,
                         double* out, cudaStream_t st) {
  if (dtype == NTF_BF16)
    k_norm2<__nv_bfloat16><<<blocks, 256, 0, st>>>(static_cast<const __nv_bfloat16*>(X), n, partial);
  else
    k_norm2<float><<<blocks, 256, 0, st>>>(static_cast<const float*>(X), n, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_sum_doubles<<<1, 32, 0, st>>>(partial, blocks, out);
  return cudaGetLastError();
}

cudaError_t launch_to_bf16(const float* in, uint16_t* out, int64_t n, cudaStream_t st) {
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 8192));
  k_to_bf16<<<static_cast<unsigned>(blocks), 256, 0, st>>>(in, reinterpret_cast<__nv_bfloat16*>(out), n);
  return cudaGetLastError();
}

}  // namespace ntf
