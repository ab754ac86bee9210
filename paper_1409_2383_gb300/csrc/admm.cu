// Gram, coefficient-matrix and fit kernels of the stand-alone entry points (Sec. IV-A item
// 2, Sec. VI-A of Liavas & Sidiropoulos); the fused factor update is in update.cu.
//
// Precision: Grams, the Hadamard product, rho and the Cholesky factorisation run in FP64
// (small rho makes G + rho I ill-conditioned); factors and MTTKRP rows are stored in FP32.
// All reductions use a fixed order.
#include <algorithm>
#include <cmath>

#include "ntf_internal.cuh"

namespace ntf {
namespace {

constexpr int kGramPairsPerBlock = 16;

// G = F^T F: CTA handles 16 (r, s) pairs of the lower triangle; 16 threads per pair stride
// over the rows and are combined by a fixed shuffle tree.
__global__ void k_gram(const float* __restrict__ F, int64_t I, int R, double* __restrict__ G) {
  const int pair = blockIdx.x * kGramPairsPerBlock + threadIdx.x / 16;
  const int l16 = threadIdx.x % 16;
  const int npairs = R * (R + 1) / 2;
  int r = 0, s = 0;
  if (pair < npairs) {
    // pair k -> (r, s), s <= r, in row order of the lower triangle
    int k = pair;
    while (k > r) { k -= r + 1; ++r; }
    s = k;
  }
  double acc = 0.0;
  if (pair < npairs)
    for (int64_t i = l16; i < I; i += 16)
      acc = fma(static_cast<double>(F[i * R + r]), static_cast<double>(F[i * R + s]), acc);
#pragma unroll
  for (int off = 8; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off, 16);
  if (pair < npairs && l16 == 0) {
    G[r * R + s] = acc;
    G[s * R + r] = acc;
  }
}

// H = Hadamard_{m != mode} Gram_m + rho I, then H = L L^T (right-looking, one CTA).
__global__ void k_system(const double* __restrict__ grams, int N, int mode, int R,
                         int rho_policy, Ctrl* ctrl, double* __restrict__ H_out,
                         double* __restrict__ L_out) {
  __shared__ double A[kMaxRank * kMaxRank];
  __shared__ int fail;
  const int tid = threadIdx.x;
  const int RR = R * R;
  for (int idx = tid; idx < RR; idx += blockDim.x) {
    double v = 1.0;
    for (int m = 0; m < N; ++m)
      if (m != mode) v *= grams[m * RR + idx];
    A[idx] = v;
  }
  __syncthreads();
  if (tid == 0) {
    double rho;
    if (rho_policy == NTF_RHO_TRACE) {
      double tr = 0.0;
      for (int i = 0; i < R; ++i) tr += A[i * R + i];
      rho = tr / R;
    } else {
      rho = ctrl->rho[mode];
    }
    fail = !(rho > 0.0) || !isfinite(rho);
    for (int i = 0; i < R; ++i) A[i * R + i] += rho;
    ctrl->stats[mode][5] = rho;
  }
  __syncthreads();
  if (H_out)
    for (int idx = tid; idx < RR; idx += blockDim.x) H_out[idx] = A[idx];
  __syncthreads();
  for (int k = 0; k < R && !fail; ++k) {
    if (tid == 0) {
      const double d = A[k * R + k];
      if (!(d > 0.0) || !isfinite(d)) fail = 1;
      else A[k * R + k] = sqrt(d);
    }
    __syncthreads();
    if (fail) break;
    const double dk = A[k * R + k];
    for (int i = k + 1 + tid; i < R; i += blockDim.x) A[i * R + k] /= dk;
    __syncthreads();
    const int n = R - k - 1;
    for (int idx = tid; idx < n * n; idx += blockDim.x) {
      const int i = k + 1 + idx / n, j = k + 1 + idx % n;
      if (j <= i) A[i * R + j] -= A[i * R + k] * A[j * R + k];
    }
    __syncthreads();
  }
  for (int idx = tid; idx < RR; idx += blockDim.x) {
    const int i = idx / R, j = idx % R;
    L_out[idx] = (j <= i && !fail) ? A[idx] : (i == j ? 1.0 : 0.0);
  }
  if (tid == 0) {
    ctrl->bad[mode] = fail;
    if (fail) atomicOr(&ctrl->status, kStNotSpd);
  }
}

constexpr int kFitThreads = 256;

__global__ void k_fit_partial(const float* __restrict__ M, const float* __restrict__ F,
                              int64_t n, double* __restrict__ part) {
  __shared__ double red[kFitThreads];
  double s = 0.0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    s = fma(static_cast<double>(M[i]), static_cast<double>(F[i]), s);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_fit_finalize(const double* __restrict__ part, int nblocks,
                               const double* __restrict__ grams, int N, int R, Ctrl* ctrl) {
  __shared__ double red[kFitThreads];
  double g = 0.0;
  for (int idx = threadIdx.x; idx < R * R; idx += blockDim.x) {
    double v = 1.0;
    for (int m = 0; m < N; ++m) v *= grams[m * R * R + idx];
    g += v;
  }
  red[threadIdx.x] = g;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double inner = 0.0;
    for (int b = 0; b < nblocks; ++b) inner += part[b];
    const double x2 = ctrl->x_norm2;
    const double e2 = x2 - 2.0 * inner + red[0];
    ctrl->fit_inner = inner;
    ctrl->fit_gram = red[0];
    ctrl->rel_err = sqrt(fmax(e2, 0.0) / x2);
    if (!isfinite(e2)) atomicOr(&ctrl->status, kStNonFinite);
  }
}

// Relative error by explicit reconstruction (Sec. VI-A): sum over the tensor of
// (x - sum_r prod_m F_m[i_m, r])^2, with no cancellation between large terms (the Gram identity
// of the fit subtracts quantities of size ||X||^2, so an error e ||X||^2 in <M, F> moves the
// squared error by 2 e ||X||^2 -- visible at low noise).  One warp per tensor row of the last
// mode: the product p_r of the other factors' rows is formed once (lanes over r, broadcast
// through shared memory), then lanes take the row's entries k = lane, lane + 32, ... with the
// model value sum_r p_r F_last[k, r] in FP32 and the squared residuals summed in FP32 per lane
// and in FP64 across lanes, warps and blocks (fixed order).
constexpr int kExWarps = 8;

template <typename T>
__global__ void __launch_bounds__(kExWarps * 32) k_fit_explicit(
    const T* __restrict__ X, int N, int64_t d0, int64_t d1, int64_t d2, int64_t K,
    const float* __restrict__ F0, const float* __restrict__ F1, const float* __restrict__ F2,
    const float* __restrict__ FL, int R, double* __restrict__ part) {
  __shared__ float p[kExWarps][64];
  __shared__ double red[kExWarps];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t rows = N == 3 ? d0 * d1 : d0 * d1 * d2;
  double acc = 0.0;
  for (int64_t row = static_cast<int64_t>(blockIdx.x) * kExWarps + warp; row < rows;
       row += static_cast<int64_t>(gridDim.x) * kExWarps) {
    // row index -> (i0, i1[, i2]) of the leading modes, last of them fastest
    int64_t i0, i1, i2 = 0;
    if (N == 3) {
      i0 = row / d1;
      i1 = row % d1;
    } else {
      i0 = row / (d1 * d2);
      i1 = (row / d2) % d1;
      i2 = row % d2;
    }
    for (int r = lane; r < R; r += 32) {
      float v = F0[i0 * R + r] * F1[i1 * R + r];
      if (N == 4) v *= F2[i2 * R + r];
      p[warp][r] = v;
    }
    __syncwarp();
    const T* x = X + row * K;
    float s = 0.0f;
    for (int64_t k = lane; k < K; k += 32) {
      const float* fl = FL + k * R;
      float m0 = 0.0f, m1 = 0.0f;
      int r = 0;
      for (; r + 1 < R; r += 2) {
        m0 = fmaf(p[warp][r], fl[r], m0);
        m1 = fmaf(p[warp][r + 1], fl[r + 1], m1);
      }
      if (r < R) m0 = fmaf(p[warp][r], fl[r], m0);
      float xv;
      if constexpr (sizeof(T) == 2) xv = __bfloat162float(x[k]);
      else xv = x[k];
      const float d = xv - (m0 + m1);
      s = fmaf(d, d, s);
    }
    __syncwarp();
    double sd = s;
    for (int off = 16; off > 0; off >>= 1) sd += __shfl_xor_sync(0xffffffffu, sd, off);
    acc += sd;
  }
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kExWarps; ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}

__global__ void k_fit_explicit_finalize(const double* __restrict__ part, int nblocks, Ctrl* ctrl) {
  if (threadIdx.x != 0) return;
  double e2 = 0.0;
  for (int b = 0; b < nblocks; ++b) e2 += part[b];
  ctrl->rel_err = sqrt(e2 / ctrl->x_norm2);
  if (!isfinite(e2)) atomicOr(&ctrl->status, kStNonFinite);
}

}  // namespace

cudaError_t launch_fit_explicit(const void* X, int dtype, int N, const int64_t* dims,
                                const float* const* F, int R, double* partial, int max_blocks,
                                Ctrl* ctrl, cudaStream_t st) {
  const int64_t rows = N == 3 ? dims[0] * dims[1] : dims[0] * dims[1] * dims[2];
  const int nb = static_cast<int>(std::max<int64_t>(
      1, std::min<int64_t>((rows + kExWarps - 1) / kExWarps, max_blocks)));
  const int64_t K = dims[N - 1];
  const float* F2 = N == 4 ? F[2] : nullptr;
  if (dtype == NTF_BF16)
    k_fit_explicit<__nv_bfloat16><<<nb, kExWarps * 32, 0, st>>>(
        static_cast<const __nv_bfloat16*>(X), N, dims[0], dims[1], N == 4 ? dims[2] : 1, K,
        F[0], F[1], F2, F[N - 1], R, partial);
  else
    k_fit_explicit<float><<<nb, kExWarps * 32, 0, st>>>(
        static_cast<const float*>(X), N, dims[0], dims[1], N == 4 ? dims[2] : 1, K, F[0], F[1],
        F2, F[N - 1], R, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_fit_explicit_finalize<<<1, 32, 0, st>>>(partial, nb, ctrl);
  return cudaGetLastError();
}

cudaError_t launch_gram(const float* F, int64_t I, int R, double* G, cudaStream_t st) {
  const int npairs = R * (R + 1) / 2;
  k_gram<<<(npairs + kGramPairsPerBlock - 1) / kGramPairsPerBlock, kGramPairsPerBlock * 16, 0,
           st>>>(F, I, R, G);
  return cudaGetLastError();
}

cudaError_t launch_system(const double* grams, int N, int mode, int R, int rho_policy,
                          Ctrl* ctrl, double* H, double* L, cudaStream_t st) {
  k_system<<<1, 256, 0, st>>>(grams, N, mode, R, rho_policy, ctrl, H, L);
  return cudaGetLastError();
}

int fit_blocks(int64_t I, int R) {
  return static_cast<int>(std::min<int64_t>(std::max<int64_t>((I * R + kFitThreads - 1) / kFitThreads, 1), 64));
}

cudaError_t launch_fit(const float* M, const float* F, int64_t I, int R, const double* grams,
                       int N, double* partial, Ctrl* ctrl, cudaStream_t st) {
  const int nb = fit_blocks(I, R);
  k_fit_partial<<<nb, kFitThreads, 0, st>>>(M, F, I * R, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_fit_finalize<<<1, kFitThreads, 0, st>>>(partial, nb, grams, N, R, ctrl);
  return cudaGetLastError();
}

}  // namespace ntf
