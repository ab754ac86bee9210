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

}  // namespace

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
