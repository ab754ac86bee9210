// Coefficient matrix, factor update and fit kernels (Sec. III-A items 2-3, eqs.
// ADMM_NTF_ALS_C / ADMoM_NTF, Sec. III-C/D, Sec. V-A of Liavas & Sidiropoulos).
//
// Precision: Grams, the Hadamard product, rho, the Cholesky factorisation and the per-row
// solves run in FP64 (small rho makes G + rho I ill-conditioned); factors, auxiliaries,
// duals and MTTKRP rows are stored in FP32.  All reductions use a fixed order.
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
  __shared__ double rho_s;
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
    rho_s = rho;
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
  (void)rho_s;
}

// One warp per row; lanes own elements j = lane and lane + 32.  L (row-major) and L^T are
// staged in shared memory so that both triangular sweeps read consecutive addresses.
constexpr int kRowWarps = 8;

__global__ void __launch_bounds__(kRowWarps * 32)
    k_admm_rows(const float* __restrict__ M, float* __restrict__ A, float* __restrict__ At,
                float* __restrict__ Y, const double* __restrict__ Lg, int64_t I, int R,
                int inner, int mode, Ctrl* ctrl, double* __restrict__ norm_part) {
  extern __shared__ double sh[];
  double* L = sh;                 // [R][R]  L[j][k]
  double* Lt = sh + R * R;        // [R][R]  Lt[k][j] = L[j][k]
  double* invd = sh + 2 * R * R;  // [R]
  __shared__ double red[kRowWarps][5];
  if (ctrl->bad[mode]) return;  // uniform across the grid
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int idx = tid; idx < R * R; idx += blockDim.x) {
    const double v = Lg[idx];
    L[idx] = v;
    Lt[(idx % R) * R + idx / R] = v;
  }
  for (int k = tid; k < R; k += blockDim.x) invd[k] = 1.0 / Lg[k * R + k];
  __syncthreads();
  const double rho = ctrl->stats[mode][5];
  const double rinv = 1.0 / rho;
  const int64_t row = static_cast<int64_t>(blockIdx.x) * kRowWarps + warp;
  double nrm[5] = {0, 0, 0, 0, 0};
  if (row < I) {
    const int j0 = lane, j1 = lane + 32;
    const bool h0 = j0 < R, h1 = j1 < R;
    const int64_t base = row * R;
    const double m0 = h0 ? M[base + j0] : 0.0, m1 = h1 ? M[base + j1] : 0.0;
    double t0 = h0 ? At[base + j0] : 0.0, t1 = h1 ? At[base + j1] : 0.0;
    double y0 = h0 ? Y[base + j0] : 0.0, y1 = h1 ? Y[base + j1] : 0.0;
    const double s0 = t0, s1 = t1;
    double x0 = 0.0, x1 = 0.0;
    for (int it = 0; it < inner; ++it) {
      double v0 = h0 ? m0 + rho * t0 - y0 : 0.0;
      double v1 = h1 ? m1 + rho * t1 - y1 : 0.0;
      // forward: L z = v  (z overwrites v)
      for (int k = 0; k < R; ++k) {
        const double own = (k < 32 ? v0 : v1) * invd[k];
        const double zk = __shfl_sync(0xffffffffu, own, k & 31);
        if (lane == (k & 31)) {
          if (k < 32) v0 = zk; else v1 = zk;
        }
        const double* col = Lt + k * R;
        if (h0 && j0 > k) v0 -= col[j0] * zk;
        if (h1 && j1 > k) v1 -= col[j1] * zk;
      }
      // backward: L^T x = z  (x overwrites v)
      for (int k = R - 1; k >= 0; --k) {
        const double own = (k < 32 ? v0 : v1) * invd[k];
        const double xk = __shfl_sync(0xffffffffu, own, k & 31);
        if (lane == (k & 31)) {
          if (k < 32) v0 = xk; else v1 = xk;
        }
        const double* rowk = L + k * R;
        if (h0 && j0 < k) v0 -= rowk[j0] * xk;
        if (h1 && j1 < k) v1 -= rowk[j1] * xk;
      }
      x0 = v0;
      x1 = v1;
      // projection onto the non-negative orthant, then dual ascent
      const double n0 = fmax(0.0, x0 + y0 * rinv), n1 = fmax(0.0, x1 + y1 * rinv);
      y0 += rho * (x0 - n0);
      y1 += rho * (x1 - n1);
      t0 = h0 ? n0 : 0.0;
      t1 = h1 ? n1 : 0.0;
      if (!h0) y0 = 0.0;
      if (!h1) y1 = 0.0;
    }
    if (h0) {
      A[base + j0] = static_cast<float>(x0);
      At[base + j0] = static_cast<float>(t0);
      Y[base + j0] = static_cast<float>(y0);
    }
    if (h1) {
      A[base + j1] = static_cast<float>(x1);
      At[base + j1] = static_cast<float>(t1);
      Y[base + j1] = static_cast<float>(y1);
    }
    if (!h0) x0 = 0.0;
    if (!h1) x1 = 0.0;
    nrm[0] = (x0 - t0) * (x0 - t0) + (x1 - t1) * (x1 - t1);
    nrm[1] = (t0 - s0) * (t0 - s0) + (t1 - s1) * (t1 - s1);
    nrm[2] = x0 * x0 + x1 * x1;
    nrm[3] = t0 * t0 + t1 * t1;
    nrm[4] = y0 * y0 + y1 * y1;
  }
#pragma unroll
  for (int q = 0; q < 5; ++q)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) nrm[q] += __shfl_xor_sync(0xffffffffu, nrm[q], off);
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < 5; ++q) red[warp][q] = nrm[q];
  __syncthreads();
  if (tid < 5) {
    double s = 0.0;
    for (int w = 0; w < kRowWarps; ++w) s += red[w][tid];
    norm_part[blockIdx.x * 5 + tid] = s;
  }
}

__global__ void k_update_finalize(const double* __restrict__ part, int nblocks, int mode,
                                  int rho_policy, double mu, double tau_incr, double tau_decr,
                                  Ctrl* ctrl) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (ctrl->bad[mode]) return;
  double s[5] = {0, 0, 0, 0, 0};
  for (int b = 0; b < nblocks; ++b)
    for (int q = 0; q < 5; ++q) s[q] += part[b * 5 + q];
  const double rho = ctrl->stats[mode][5];
  const double P = sqrt(s[0]), D = rho * sqrt(s[1]);
  ctrl->stats[mode][0] = P;
  ctrl->stats[mode][1] = D;
  ctrl->stats[mode][2] = sqrt(s[2]);
  ctrl->stats[mode][3] = sqrt(s[3]);
  ctrl->stats[mode][4] = sqrt(s[4]);
  bool finite = true;
  for (int q = 0; q < 5; ++q) finite = finite && isfinite(s[q]);
  if (!finite) atomicOr(&ctrl->status, kStNonFinite);
  if (rho_policy == NTF_RHO_ADAPTIVE) {
    // eq. (varying_penalty_rule); the cases exclude each other because mu > 1
    double r = rho;
    if (P > mu * D) r = tau_incr * rho;
    else if (D > mu * P) r = rho / tau_decr;
    ctrl->rho[mode] = r;
  } else if (rho_policy == NTF_RHO_TRACE) {
    ctrl->rho[mode] = rho;
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

int admm_row_blocks(int64_t I) { return static_cast<int>((I + kRowWarps - 1) / kRowWarps); }

cudaError_t launch_admm_rows(const float* M, float* A, float* At, float* Y, const double* L,
                             int64_t I, int R, int inner, int mode, Ctrl* ctrl,
                             double* norm_part, cudaStream_t st) {
  const size_t smem = (2 * static_cast<size_t>(R) * R + R) * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(k_admm_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  k_admm_rows<<<admm_row_blocks(I), kRowWarps * 32, smem, st>>>(M, A, At, Y, L, I, R, inner,
                                                                 mode, ctrl, norm_part);
  return cudaGetLastError();
}

cudaError_t launch_update_finalize(const double* norm_part, int nblocks, int mode,
                                   int rho_policy, double mu, double tau_incr,
                                   double tau_decr, Ctrl* ctrl, cudaStream_t st) {
  k_update_finalize<<<1, 32, 0, st>>>(norm_part, nblocks, mode, rho_policy, mu, tau_incr,
                                      tau_decr, ctrl);
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
