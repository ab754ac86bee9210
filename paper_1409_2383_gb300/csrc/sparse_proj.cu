// Factor update with the sparsity constraint of Sec. IV-E (eq. g_new_def): the auxiliary is
// projected onto the non-negative matrices with at most c nonzero entries.  Keeping entry v
// of V = A + Y / rho costs (max(v, 0) - v)^2 and zeroing it costs v^2, so the projection keeps
// the c largest positive entries of the whole factor and zeroes the rest -- a selection over
// all rows, which the row-parallel inner loop of update.cu cannot make.  Each of the L inner
// iterations therefore runs as three launches:
//
//   k_sp_primal  one warp per row: x = H^{-1} (m + rho At - Y)   (eq. ADMM_NTF_ALS_C), with
//                the coefficient inverse of the update's system slot (FP32 under the trace
//                policy, FP64 otherwise); stores x in A and V = x + Y / rho.
//   k_sp_select  one CTA: the c-th largest positive entry of V by a most-significant-digit
//                radix selection on the bit patterns (positive IEEE floats order as their
//                bits), 8 bits per pass; among entries equal to it, those of lower flat index
//                are kept first (the order of a stable sort).
//   k_sp_apply   At = kept entries of V (0 elsewhere), Y += rho (A - At)   (eq. ADMoM_NTF).
//
// The rows kernel of update.cu then forms the partial sums of the update (residuals, Gram,
// fit, KKT terms) from the stored A, At, Y and the auxiliary before the update.  Every kernel
// leaves the state untouched when the factor's system failed or the run has stopped.
#include <algorithm>

#include "ntf_internal.cuh"

namespace ntf {
namespace {

constexpr int kSpWarps = 8;
constexpr int kSelThreads = 1024;

struct SpArgs {
  const double* hinv64;  // [R, R] (FP64 policies)
  const float* hinv32;   // [R, R] (trace policy)
  const float* M;
  float* A;
  float* At;
  float* Y;
  float* V;              // [I, R]
  unsigned* sel;         // [2]: threshold bits, flat index of the last kept tie
  const Ctrl* ctrl;
  int64_t I;
  int mode, R, fp64;
  int64_t c;             // at most c nonzeros
};

__device__ __forceinline__ bool sp_skip(const SpArgs& a) {
  return a.ctrl->bad[a.mode] != 0 || a.ctrl->stop != 0;
}

// One warp per row; lane j holds elements j and j + 32.
__global__ void __launch_bounds__(kSpWarps * 32) k_sp_primal(SpArgs a) {
  if (sp_skip(a)) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t row = static_cast<int64_t>(blockIdx.x) * kSpWarps + warp;
  if (row >= a.I) return;  // warp-uniform
  const int R = a.R;
  const double rho = a.ctrl->stats[a.mode][5];
  const int j0 = lane, j1 = lane + 32;
  const bool h0 = j0 < R, h1 = j1 < R;
  const int64_t base = row * R;
  // v = m + rho At - Y, in the row's precision
  double v0 = 0.0, v1 = 0.0, y0 = 0.0, y1 = 0.0;
  if (h0) {
    y0 = a.Y[base + j0];
    v0 = static_cast<double>(a.M[base + j0]) + rho * a.At[base + j0] - y0;
  }
  if (h1) {
    y1 = a.Y[base + j1];
    v1 = static_cast<double>(a.M[base + j1]) + rho * a.At[base + j1] - y1;
  }
  double x0 = 0.0, x1 = 0.0;
  if (a.fp64) {
    for (int k = 0; k < R; ++k) {
      const double vk = __shfl_sync(0xffffffffu, k < 32 ? v0 : v1, k & 31);
      if (h0) x0 = fma(a.hinv64[k * R + j0], vk, x0);
      if (h1) x1 = fma(a.hinv64[k * R + j1], vk, x1);
    }
  } else {
    const float f0 = static_cast<float>(v0), f1 = static_cast<float>(v1);
    float p0 = 0.0f, p1 = 0.0f;
    for (int k = 0; k < R; ++k) {
      const float vk = __shfl_sync(0xffffffffu, k < 32 ? f0 : f1, k & 31);
      if (h0) p0 = fmaf(a.hinv32[k * R + j0], vk, p0);
      if (h1) p1 = fmaf(a.hinv32[k * R + j1], vk, p1);
    }
    x0 = p0;
    x1 = p1;
  }
  const double rinv = 1.0 / rho;
  if (h0) {
    a.A[base + j0] = static_cast<float>(x0);
    a.V[base + j0] = static_cast<float>(x0 + y0 * rinv);
  }
  if (h1) {
    a.A[base + j1] = static_cast<float>(x1);
    a.V[base + j1] = static_cast<float>(x1 + y1 * rinv);
  }
}

// Selection key of an entry: its bit pattern if it is positive, else 0 (never kept).
__device__ __forceinline__ unsigned sp_key(float v) {
  return v > 0.0f ? __float_as_uint(v) : 0u;
}

// One CTA.  sel[0] = key of the c-th largest positive entry (0: fewer than c positive entries,
// keep every positive one); sel[1] = the flat index of the last entry equal to it that is
// kept (entries equal to it are kept in increasing flat index).
__global__ void __launch_bounds__(kSelThreads) k_sp_select(SpArgs a) {
  __shared__ unsigned hist[256];
  __shared__ unsigned s_prefix, s_rank, s_gt;
  __shared__ unsigned s_scan[kSelThreads];
  if (sp_skip(a)) return;
  const int tid = threadIdx.x;
  const int64_t n = a.I * a.R;
  // rank (1-based, from the top) of the wanted key among the positive keys
  if (tid == 0) {
    s_prefix = 0;
    s_rank = static_cast<unsigned>(a.c < n ? a.c : n);
    s_gt = 0;
  }
  __syncthreads();
  // number of positive entries: if at most c, every positive entry is kept
  unsigned pos = 0;
  for (int64_t e = tid; e < n; e += kSelThreads) pos += sp_key(a.V[e]) != 0u;
  for (int off = 16; off > 0; off >>= 1) pos += __shfl_xor_sync(0xffffffffu, pos, off);
  if ((tid & 31) == 0) s_scan[tid >> 5] = pos;
  __syncthreads();
  if (tid == 0) {
    unsigned tot = 0;
    for (int w = 0; w < kSelThreads / 32; ++w) tot += s_scan[w];
    if (static_cast<int64_t>(tot) <= a.c || a.c == 0) s_rank = 0;  // no threshold needed
    if (a.c == 0) s_prefix = 0xFFFFFFFFu;                           // keep nothing
  }
  __syncthreads();
  if (s_rank == 0) {
    if (tid == 0) {
      a.sel[0] = s_prefix;  // 0: keep every positive entry; ~0: keep none
      a.sel[1] = 0;
    }
    return;
  }
  // most significant digit first: after pass d, s_prefix holds the top 8 (d + 1) bits of the
  // wanted key and s_rank its rank among the keys that share them
  for (int d = 0; d < 4; ++d) {
    const int shift = 24 - 8 * d;
    const unsigned mask_hi = d == 0 ? 0u : 0xFFFFFFFFu << (shift + 8);
    for (int b = tid; b < 256; b += kSelThreads) hist[b] = 0;
    __syncthreads();
    const unsigned pre = s_prefix;
    for (int64_t e = tid; e < n; e += kSelThreads) {
      const unsigned k = sp_key(a.V[e]);
      if (k != 0u && (k & mask_hi) == pre) atomicAdd(&hist[(k >> shift) & 0xFFu], 1u);
    }
    __syncthreads();
    if (tid == 0) {
      unsigned acc = 0, r = s_rank;
      int b = 255;
      for (; b > 0 && acc + hist[b] < r; --b) acc += hist[b];
      s_prefix = pre | (static_cast<unsigned>(b) << shift);
      s_rank = r - acc;      // rank within the bin
      s_gt += acc;           // keys above the bin
    }
    __syncthreads();
  }
  const unsigned thr = s_prefix;
  const unsigned need = s_rank;  // entries equal to thr that are kept (>= 1)
  // the need-th entry equal to thr in flat order: per-thread counts over contiguous chunks,
  // then a scan over the threads
  const int64_t chunk = (n + kSelThreads - 1) / kSelThreads;
  const int64_t e0 = tid * chunk, e1 = e0 + chunk < n ? e0 + chunk : n;
  unsigned cnt = 0;
  for (int64_t e = e0; e < e1; ++e) cnt += sp_key(a.V[e]) == thr;
  s_scan[tid] = cnt;
  __syncthreads();
  for (int off = 1; off < kSelThreads; off <<= 1) {  // inclusive scan (Hillis-Steele)
    const unsigned v = tid >= off ? s_scan[tid - off] : 0u;
    __syncthreads();
    s_scan[tid] += v;
    __syncthreads();
  }
  const unsigned before = s_scan[tid] - cnt;
  if (before < need && need <= s_scan[tid]) {
    unsigned k = before;
    for (int64_t e = e0; e < e1; ++e)
      if (sp_key(a.V[e]) == thr && ++k == need) {
        a.sel[0] = thr;
        a.sel[1] = static_cast<unsigned>(e);
        break;
      }
  }
}

__global__ void k_sp_apply(SpArgs a) {
  if (sp_skip(a)) return;
  const int64_t n = a.I * a.R;
  const unsigned thr = a.sel[0];
  const int64_t cut = a.sel[1];
  const double rho = a.ctrl->stats[a.mode][5];
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < n;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float v = a.V[e];
    const unsigned k = sp_key(v);
    const bool keep = k != 0u && (k > thr || (k == thr && e <= cut));
    const float t = keep ? v : 0.0f;
    a.At[e] = t;
    a.Y[e] = static_cast<float>(a.Y[e] + rho * (static_cast<double>(a.A[e]) - t));
  }
}

}  // namespace

cudaError_t launch_sparse_inner(const UpdateCall& u, int64_t c, float* V, float* t_before,
                                unsigned* sel, cudaStream_t st) {
  SpArgs a{};
  a.hinv64 = update_sys_hinv64(u.sys, u.mode, u.R);
  a.hinv32 = update_sys_hinv32(u.sys, u.mode, u.R);
  a.M = u.M;
  a.A = u.A;
  a.At = u.At;
  a.Y = u.Y;
  a.V = V;
  a.sel = sel;
  a.ctrl = u.ctrl;
  a.I = u.I;
  a.mode = u.mode;
  a.R = u.R;
  a.fp64 = u.rho_policy != NTF_RHO_TRACE;
  a.c = c;
  const int64_t n = u.I * u.R;
  cudaError_t e = cudaMemcpyAsync(t_before, u.At, n * sizeof(float), cudaMemcpyDeviceToDevice, st);
  const unsigned rows_blocks = static_cast<unsigned>((u.I + kSpWarps - 1) / kSpWarps);
  const unsigned ew_blocks = static_cast<unsigned>(std::min<int64_t>((n + 255) / 256, 4 * kNumSM));
  for (int it = 0; it < u.inner && e == cudaSuccess; ++it) {
    k_sp_primal<<<rows_blocks, kSpWarps * 32, 0, st>>>(a);
    k_sp_select<<<1, kSelThreads, 0, st>>>(a);
    k_sp_apply<<<ew_blocks, 256, 0, st>>>(a);
    e = cudaGetLastError();
  }
  return e;
}

int sparse_inner_launches(int inner) { return 1 + 3 * inner; }

}  // namespace ntf
