// Warm-start network for the per-row non-negative least squares of a factor update.
//
// With the other factors fixed, every row of the factor solves min_{x >= 0} 1/2 x^T G x - m^T x
// (G: coefficient matrix of eq. ADMM_NTF_ALS_C without rho, m: MTTKRP row); ADMoM converges to
// x* with dual y* = m - G x* (eq. KKT_NTF).  The network maps [vec(G/s) ; m/s ; z],
// s = trace(G)/R, z = (G + s I)^{-1} m (the first primal iterate of the row's ADMM from zero),
// to [x* ; y*/s] (the problem is invariant under (G, m) -> (cG, cm) with x* and z fixed and y*
// scaled by c).  Layers: R^2+2R -> H -> H -> 2R, exact GELU, BF16 weights in the products
// with FP32 master copies and FP32 accumulation everywhere; the training GEMMs run on the
// tensor cores (FP32 activations and gradients as two BF16 parts).  The first layer is split
// W1 = [W1_G | W1_u]: W1_G vec(G/s) is formed once per coefficient matrix and shared by all
// of its rows; W1_u acts on the per-row input u = [m/s ; z] (2R values).  Training: mean
// squared error, Adam (Kingma & Ba).  All reductions run in a fixed order.
#include <cmath>
#include <cstdint>

#include "ntf_internal.cuh"

namespace ntf {
namespace {

// ------------------------------------------------------------------------ GEMM
// C[M, N] = op(A)[M, K] * op(B)[K, N] (+ bias[N]) (+ C if accumulate), FP32 accumulation on the
// tensor cores (mma.sync m16n8k16, BF16 operands).  TA: A is stored [K, M] (else [M, K]); TB:
// B is stored [N, K] (else [K, N]).  FP32 operands are split into BF16 parts v = hi + lo
// (hi = bf16(v), lo = bf16(v - hi): 16 significant bits; the remainder is below 2^-16 |v|) and
// the products formed as hi hi + hi lo + lo hi (lo lo, below 2^-16 relative, is dropped); BF16
// weights are exact and need one part.  64 x 64 output tile per CTA of 8 warps (2 x 4, each
// 32 x 16 = 2 x 2 MMA tiles), K staged 32 at a time through shared memory (K-contiguous rows,
// padded so that the fragment loads are free of bank conflicts).
template <typename T>
__device__ __forceinline__ float to_f(T v);
template <>
__device__ __forceinline__ float to_f<float>(float v) { return v; }
template <>
__device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

constexpr int kGT = 64;       // output tile
constexpr int kGK = 32;       // K per stage
constexpr int kGLd = kGK + 8; // padded row (bf16 elements)

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, "
      "{%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16* p) {
  return *reinterpret_cast<const uint32_t*>(p);
}

template <bool TA, bool TB, typename TBt>
__global__ void __launch_bounds__(256)
    k_gemm(int M, int N, int K, const float* __restrict__ A, int lda, const TBt* __restrict__ B,
           int ldb, float* __restrict__ C, int ldc, const float* __restrict__ bias, int accumulate) {
  constexpr bool kBSplit = sizeof(TBt) == 4;  // FP32 B: two parts
  __shared__ __align__(16) __nv_bfloat16 Ah[kGT][kGLd], Al[kGT][kGLd];
  __shared__ __align__(16) __nv_bfloat16 Bh[kGT][kGLd], Bl[kBSplit ? kGT : 1][kGLd];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp >> 2, wn = warp & 3;    // warp tile: rows 32 wm .., columns 16 wn ..
  const int g = lane >> 2, t = lane & 3;
  const int m0 = blockIdx.y * kGT, n0 = blockIdx.x * kGT;
  float acc[2][2][4] = {};
  for (int k0 = 0; k0 < K; k0 += kGK) {
    // stage op(A)[m0.., k0..] and op(B)^T[n0.., k0..] as K-contiguous BF16 parts
    for (int idx = tid; idx < kGT * kGK; idx += 256) {
      int r, kk;
      if (TA) {  // A stored [K, M]: consecutive threads along M
        kk = idx / kGT;
        r = idx % kGT;
      } else {   // A stored [M, K]: consecutive threads along K
        r = idx / kGK;
        kk = idx % kGK;
      }
      const int gm = m0 + r, gk = k0 + kk;
      float a = 0.0f;
      if (gm < M && gk < K)
        a = TA ? A[static_cast<int64_t>(gk) * lda + gm] : A[static_cast<int64_t>(gm) * lda + gk];
      const __nv_bfloat16 h = __float2bfloat16_rn(a);
      Ah[r][kk] = h;
      Al[r][kk] = __float2bfloat16_rn(a - __bfloat162float(h));
    }
    for (int idx = tid; idx < kGT * kGK; idx += 256) {
      int c, kk;
      if (TB) {  // B stored [N, K]: along K
        c = idx / kGK;
        kk = idx % kGK;
      } else {   // B stored [K, N]: along N
        kk = idx / kGT;
        c = idx % kGT;
      }
      const int gn = n0 + c, gk = k0 + kk;
      float b = 0.0f;
      if (gn < N && gk < K)
        b = TB ? to_f<TBt>(B[static_cast<int64_t>(gn) * ldb + gk])
               : to_f<TBt>(B[static_cast<int64_t>(gk) * ldb + gn]);
      const __nv_bfloat16 h = __float2bfloat16_rn(b);
      Bh[c][kk] = h;
      if constexpr (kBSplit) Bl[c][kk] = __float2bfloat16_rn(b - __bfloat162float(h));
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < kGK; ks += 16) {
      uint32_t ah[2][4], al[2][4];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int r = 32 * wm + 16 * i + g;
        ah[i][0] = ld32(&Ah[r][ks + 2 * t]);
        ah[i][1] = ld32(&Ah[r + 8][ks + 2 * t]);
        ah[i][2] = ld32(&Ah[r][ks + 2 * t + 8]);
        ah[i][3] = ld32(&Ah[r + 8][ks + 2 * t + 8]);
        al[i][0] = ld32(&Al[r][ks + 2 * t]);
        al[i][1] = ld32(&Al[r + 8][ks + 2 * t]);
        al[i][2] = ld32(&Al[r][ks + 2 * t + 8]);
        al[i][3] = ld32(&Al[r + 8][ks + 2 * t + 8]);
      }
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int c = 16 * wn + 8 * j + g;
        const uint32_t bh0 = ld32(&Bh[c][ks + 2 * t]), bh1 = ld32(&Bh[c][ks + 2 * t + 8]);
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          mma_bf16(acc[i][j], ah[i], bh0, bh1);
          mma_bf16(acc[i][j], al[i], bh0, bh1);
        }
        if constexpr (kBSplit) {
          const uint32_t bl0 = ld32(&Bl[c][ks + 2 * t]), bl1 = ld32(&Bl[c][ks + 2 * t + 8]);
#pragma unroll
          for (int i = 0; i < 2; ++i) mma_bf16(acc[i][j], ah[i], bl0, bl1);
        }
      }
    }
    __syncthreads();
  }
  // accumulator layout: acc[i][j] = rows (g, g + 8) x columns (2t, 2t + 1) of the 16 x 8 tile
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int gm = m0 + 32 * wm + 16 * i + g + (q >= 2 ? 8 : 0);
        const int gn = n0 + 16 * wn + 8 * j + 2 * t + (q & 1);
        if (gm >= M || gn >= N) continue;
        float v = acc[i][j][q];
        if (bias) v += bias[gn];
        float* cp = C + static_cast<int64_t>(gm) * ldc + gn;
        *cp = accumulate ? *cp + v : v;
      }
}

template <bool TA, bool TB, typename TBt>
cudaError_t gemm(int M, int N, int K, const float* A, int lda, const TBt* B, int ldb, float* C,
                 int ldc, const float* bias, bool accumulate, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  dim3 grid((N + kGT - 1) / kGT, (M + kGT - 1) / kGT);
  k_gemm<TA, TB, TBt><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, bias,
                                            accumulate ? 1 : 0);
  return cudaGetLastError();
}

// ------------------------------------------------------------------- elementwise
__device__ __forceinline__ float gelu(float z) {
  return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_grad(float z) {
  const float cdf = 0.5f * (1.0f + erff(z * 0.70710678118654752f));
  const float pdf = 0.39894228040143268f * expf(-0.5f * z * z);
  return cdf + z * pdf;
}

__global__ void k_gelu(const float* __restrict__ z, float* __restrict__ h, int64_t n) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    h[i] = gelu(z[i]);
}

__global__ void k_gelu_back(const float* __restrict__ z, float* __restrict__ d, int64_t n) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    d[i] *= gelu_grad(z[i]);
}

// z1[i, :] += hG[group(i), :] + b1, group given by CSR offsets (rows of a group contiguous)
__global__ void k_first_layer_add(float* __restrict__ z1, const float* __restrict__ hG,
                                  const float* __restrict__ b1, const int* __restrict__ row_group,
                                  int rows, int H) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
       i < static_cast<int64_t>(rows) * H; i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int r = static_cast<int>(i / H), h = static_cast<int>(i % H);
    z1[i] += hG[static_cast<int64_t>(row_group[r]) * H + h] + b1[h];
  }
}

// d_out = 2 (out - T) / (rows * D); per-block partial sums of the squared error
__global__ void k_mse(const float* __restrict__ out, const float* __restrict__ T,
                      float* __restrict__ d, int64_t n, double* __restrict__ part) {
  __shared__ double red[256];
  double s = 0.0;
  const float scale = 2.0f / static_cast<float>(n);
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float e = out[i] - T[i];
    d[i] = scale * e;
    s += static_cast<double>(e) * e;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_sum_parts(const double* __restrict__ part, int n, double scale,
                            double* __restrict__ out) {
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += part[i];
    *out = s * scale;
  }
}

// out[seg, c] = sum over rows of segment seg (CSR offsets) of X[row, c]  (fixed order)
__global__ void k_segment_sum(const float* __restrict__ X, const int* __restrict__ offs,
                              int nseg, int cols, float* __restrict__ out) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
       i < static_cast<int64_t>(nseg) * cols; i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int sgi = static_cast<int>(i / cols), c = static_cast<int>(i % cols);
    float s = 0.0f;
    for (int r = offs[sgi]; r < offs[sgi + 1]; ++r) s += X[static_cast<int64_t>(r) * cols + c];
    out[i] = s;
  }
}

// Adam (bias-corrected moments), FP32 master weights, refreshed BF16 copies (weights only).
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, __nv_bfloat16* __restrict__ pb, int64_t n, float lr,
                       float b1, float b2, float eps, float c1, float c2) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float w = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = w;
    if (pb) pb[i] = __float2bfloat16_rn(w);
  }
}

// row_group[r] = g for offs[g] <= r < offs[g + 1]
__global__ void k_row_groups(const int* __restrict__ offs, int groups, int* __restrict__ rg) {
  for (int g = blockIdx.x; g < groups; g += gridDim.x)
    for (int r = offs[g] + threadIdx.x; r < offs[g + 1]; r += blockDim.x) rg[r] = g;
}

__global__ void k_to_bf16_copy(const float* __restrict__ in, __nv_bfloat16* __restrict__ out,
                               int64_t n) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    out[i] = __float2bfloat16_rn(in[i]);
}

unsigned blocks_for(int64_t n) {
  const int64_t b = (n + 255) / 256;
  return static_cast<unsigned>(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

}  // namespace

// ----------------------------------------------------------------------------- host side
MlpShape mlp_shape(int R, int H) {
  MlpShape s{};
  s.R = R;
  s.H = H;
  s.P = 2 * R;
  s.Din = R * R + s.P;
  s.Dout = 2 * R;
  s.oW1 = 0;
  s.ob1 = s.oW1 + static_cast<int64_t>(H) * s.Din;
  s.oW2 = s.ob1 + H;
  s.ob2 = s.oW2 + static_cast<int64_t>(H) * H;
  s.oW3 = s.ob2 + H;
  s.ob3 = s.oW3 + static_cast<int64_t>(s.Dout) * H;
  s.count = s.ob3 + s.Dout;
  return s;
}

// Forward for `rows` rows given per-group first-layer terms hG [groups, H] (already W1_G
// vec(G/s)), row_group[rows] and the per-row inputs mrows [rows, 2R] = [m/s ; z].  Work
// buffers: z1, h1, z2, h2 [rows, H], out [rows, Dout].
cudaError_t mlp_forward_rows(const MlpShape& s, const float* p, const __nv_bfloat16* pb,
                             const float* hG, const int* row_group, const float* mrows, int rows,
                             float* z1, float* h1, float* z2, float* h2, float* out,
                             cudaStream_t st) {
  const int H = s.H, R = s.R;
  // z1 = mrows W1_u^T (columns R^2 .. R^2+2R-1 of W1), then + hG[group] + b1
  cudaError_t e = gemm<false, true, __nv_bfloat16>(rows, H, s.P, mrows, s.P, pb + s.oW1 + R * R,
                                                   s.Din, z1, H, nullptr, false, st);
  if (e != cudaSuccess) return e;
  k_first_layer_add<<<blocks_for(static_cast<int64_t>(rows) * H), 256, 0, st>>>(
      z1, hG, p + s.ob1, row_group, rows, H);
  k_gelu<<<blocks_for(static_cast<int64_t>(rows) * H), 256, 0, st>>>(z1, h1, static_cast<int64_t>(rows) * H);
  e = gemm<false, true, __nv_bfloat16>(rows, H, H, h1, H, pb + s.oW2, H, z2, H, p + s.ob2, false, st);
  if (e != cudaSuccess) return e;
  k_gelu<<<blocks_for(static_cast<int64_t>(rows) * H), 256, 0, st>>>(z2, h2, static_cast<int64_t>(rows) * H);
  e = gemm<false, true, __nv_bfloat16>(rows, s.Dout, H, h2, H, pb + s.oW3, H, out, s.Dout,
                                       p + s.ob3, false, st);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// hG[g, :] = W1_G vec(Gn[g])  for `groups` normalised coefficient matrices Gn [groups, R^2]
cudaError_t mlp_group_terms(const MlpShape& s, const __nv_bfloat16* pb, const float* Gn,
                            int groups, float* hG, cudaStream_t st) {
  return gemm<false, true, __nv_bfloat16>(groups, s.H, s.R * s.R, Gn, s.R * s.R, pb + s.oW1,
                                          s.Din, hG, s.H, nullptr, false, st);
}

// Gradients of the mean squared error for one batch (rows sorted by group, CSR offsets
// offs[groups + 1]); writes grad [count] and the loss.  Expects the forward buffers filled.
cudaError_t mlp_backward(const MlpShape& s, const __nv_bfloat16* pb, const float* Gn,
                         const int* offs, int groups, const int* all_offs, const float* mrows,
                         int rows,
                         const float* T, const float* z1, const float* h1, const float* z2,
                         const float* h2, const float* out, float* d_out, float* d_h2,
                         float* d_h1, float* gsum, float* grad, double* loss_part,
                         double* loss, cudaStream_t st) {
  const int H = s.H, R = s.R, D = s.Dout;
  const int64_t n_out = static_cast<int64_t>(rows) * D;
  const unsigned lb = blocks_for(n_out) > 64 ? 64 : blocks_for(n_out);
  k_mse<<<lb, 256, 0, st>>>(out, T, d_out, n_out, loss_part);
  k_sum_parts<<<1, 32, 0, st>>>(loss_part, static_cast<int>(lb), 1.0 / static_cast<double>(n_out), loss);
  // layer 3: dW3 = d_out^T h2, db3 = colsum(d_out), d_h2 = d_out W3
  cudaError_t e = gemm<true, false, float>(D, H, rows, d_out, D, h2, H, grad + s.oW3, H, nullptr, false, st);
  if (e != cudaSuccess) return e;
  e = gemm<false, false, __nv_bfloat16>(rows, H, D, d_out, D, pb + s.oW3, H, d_h2, H, nullptr, false, st);
  if (e != cudaSuccess) return e;
  k_gelu_back<<<blocks_for(static_cast<int64_t>(rows) * H), 256, 0, st>>>(z2, d_h2, static_cast<int64_t>(rows) * H);
  // layer 2 (d_h2 now holds dz2)
  e = gemm<true, false, float>(H, H, rows, d_h2, H, h1, H, grad + s.oW2, H, nullptr, false, st);
  if (e != cudaSuccess) return e;
  e = gemm<false, false, __nv_bfloat16>(rows, H, H, d_h2, H, pb + s.oW2, H, d_h1, H, nullptr, false, st);
  if (e != cudaSuccess) return e;
  k_gelu_back<<<blocks_for(static_cast<int64_t>(rows) * H), 256, 0, st>>>(z1, d_h1, static_cast<int64_t>(rows) * H);
  // layer 1 (d_h1 holds dz1): dW1_u = dz1^T mrows into columns R^2.., dW1_G = gsum^T Gn
  e = gemm<true, false, float>(H, s.P, rows, d_h1, H, mrows, s.P, grad + s.oW1 + R * R, s.Din, nullptr, false, st);
  if (e != cudaSuccess) return e;
  k_segment_sum<<<blocks_for(static_cast<int64_t>(groups) * H), 256, 0, st>>>(d_h1, offs, groups, H, gsum);
  e = gemm<true, false, float>(H, R * R, groups, gsum, H, Gn, R * R, grad + s.oW1, s.Din, nullptr, false, st);
  if (e != cudaSuccess) return e;
  // biases: column sums over all rows (all_offs = {0, rows}: one segment)
  k_segment_sum<<<blocks_for(D), 256, 0, st>>>(d_out, all_offs, 1, D, grad + s.ob3);
  k_segment_sum<<<blocks_for(H), 256, 0, st>>>(d_h2, all_offs, 1, H, grad + s.ob2);
  k_segment_sum<<<blocks_for(H), 256, 0, st>>>(d_h1, all_offs, 1, H, grad + s.ob1);
  return cudaGetLastError();
}

cudaError_t mlp_adam(const MlpShape& s, float* p, const float* grad, float* m, float* v,
                     __nv_bfloat16* pb, float lr, int step, cudaStream_t st) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = 1.0f - powf(b1, static_cast<float>(step));
  const float c2 = 1.0f - powf(b2, static_cast<float>(step));
  k_adam<<<blocks_for(s.count), 256, 0, st>>>(p, grad, m, v, pb, s.count, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

cudaError_t mlp_row_groups(const int* offs, int groups, int* row_group, cudaStream_t st) {
  k_row_groups<<<groups < 1024 ? (groups > 0 ? groups : 1) : 1024, 128, 0, st>>>(offs, groups, row_group);
  return cudaGetLastError();
}

cudaError_t mlp_refresh_bf16(const MlpShape& s, const float* p, __nv_bfloat16* pb, cudaStream_t st) {
  k_to_bf16_copy<<<blocks_for(s.count), 256, 0, st>>>(p, pb, s.count);
  return cudaGetLastError();
}

}  // namespace ntf

// --------------------------------------------------------------------- warm start
namespace ntf {
namespace {

// Gn = G / s and the per-row inputs mrows[i] = [m_i / s ; z_i], z_i = Hinv m_i, with
// s = trace(G) / R (G: FP32 coefficient matrix without rho; Hinv: the update's FP32
// (G + rho I)^{-1}, rho = s under the trace policy).  One thread per output value.
__global__ void k_ws_prepare(const float* __restrict__ G, const float* __restrict__ Hinv,
                             const float* __restrict__ M, int R, int64_t I, float* __restrict__ Gn,
                             float* __restrict__ mrows, float* __restrict__ s_out) {
  float tr = 0.0f;
  for (int i = 0; i < R; ++i) tr += G[i * R + i];
  const float s = tr / R, inv = 1.0f / s;
  const int64_t nG = static_cast<int64_t>(R) * R, nM = I * 2 * R;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < nG + nM;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    if (i < nG) {
      Gn[i] = G[i] * inv;
      continue;
    }
    const int64_t k = i - nG, row = k / (2 * R);
    const int c = static_cast<int>(k % (2 * R));
    const float* m = M + row * R;
    float v;
    if (c < R) {
      v = m[c] * inv;
    } else {
      v = 0.0f;
      for (int j = 0; j < R; ++j) v = fmaf(Hinv[j * R + (c - R)], m[j], v);  // Hinv symmetric
    }
    mrows[k] = v;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *s_out = s;
}

// Per row (one warp): candidate from the network, x = max(0, out[:R]), y = min(0, s out[R:]);
// it replaces the carried-over (At, Y) row only if it is better on both counts: a smaller
// row objective q(x) = 1/2 x^T G x - m^T x = 1/2 sum_j x_j ((G x - m)_j - m_j) (the row's
// share of the fit) and a smaller KKT natural residual ||min(x, G x - m)||.  Counts
// considered / accepted rows.
__global__ void k_ws_judge(const float* __restrict__ out, const float* __restrict__ G,
                           const float* __restrict__ M, const float* __restrict__ s_ptr,
                           float* __restrict__ At, float* __restrict__ Y, int64_t I, int R,
                           unsigned long long* counters) {
  __shared__ float xs[8][2][64];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t row = static_cast<int64_t>(blockIdx.x) * 8 + warp;
  if (row >= I) return;
  const float s = *s_ptr;
  const int D = 2 * R;
  float xc[2], yc[2], xo[2], m[2];
  for (int h = 0; h < 2; ++h) {
    const int j = lane + 32 * h;
    xc[h] = yc[h] = xo[h] = m[h] = 0.0f;
    if (j < R) {
      xc[h] = fmaxf(0.0f, out[row * D + j]);
      yc[h] = fminf(0.0f, s * out[row * D + R + j]);
      xo[h] = At[row * R + j];
      m[h] = M[row * R + j];
      xs[warp][0][j] = xc[h];
      xs[warp][1][j] = xo[h];
    }
  }
  __syncwarp();
  float rc = 0.0f, ro = 0.0f, qc = 0.0f, qo = 0.0f;  // q: twice the row objective
  for (int h = 0; h < 2; ++h) {
    const int j = lane + 32 * h;
    if (j >= R) continue;
    float gc = -m[h], go = -m[h];
    for (int k = 0; k < R; ++k) {
      const float gk = G[k * R + j];  // G symmetric
      gc = fmaf(gk, xs[warp][0][k], gc);
      go = fmaf(gk, xs[warp][1][k], go);
    }
    const float a = fminf(xc[h], gc), b = fminf(xo[h], go);
    rc += a * a;
    ro += b * b;
    qc += xc[h] * (gc - m[h]);
    qo += xo[h] * (go - m[h]);
  }
  for (int off = 16; off > 0; off >>= 1) {
    rc += __shfl_xor_sync(0xffffffffu, rc, off);
    ro += __shfl_xor_sync(0xffffffffu, ro, off);
    qc += __shfl_xor_sync(0xffffffffu, qc, off);
    qo += __shfl_xor_sync(0xffffffffu, qo, off);
  }
  const bool take = rc < ro && qc < qo;
  if (take) {
    for (int h = 0; h < 2; ++h) {
      const int j = lane + 32 * h;
      if (j < R) {
        At[row * R + j] = xc[h];
        Y[row * R + j] = yc[h];
      }
    }
  }
  if (lane == 0) {
    atomicAdd(&counters[0], 1ull);
    if (take) atomicAdd(&counters[1], 1ull);
  }
}

// The warm start of one factor in two kernels (one coefficient matrix G shared by all rows):
// k_ws_group forms the group term W1_G vec(G/s) once; k_ws_fused, per CTA of kWsRows rows,
// the inputs [m/s ; Hinv m], the three layers (weights and activations in shared memory) and
// the judge (one warp per row).  Layers: warp w forms outputs w, w + 8, ...; lane l takes the
// inputs l, l + 32, ... of every row (weights read along their rows, so a warp's loads are
// contiguous), and the eight rows' partial sums are combined across the lanes by a fixed
// exchange-and-add tree.
constexpr int kWsRows = 8;
constexpr int kWsMaxK = 256;  // widest layer input held in registers (8 per lane)

__device__ __forceinline__ void ws_judge_row(const float* out, const float* G, const float* M,
                                             float s, float* At, float* Y, int64_t row, int R,
                                             float* xs, int lane,
                                             unsigned long long* counters) {
  float xc[2], yc[2], xo[2], m[2];
  for (int h = 0; h < 2; ++h) {
    const int j = lane + 32 * h;
    xc[h] = yc[h] = xo[h] = m[h] = 0.0f;
    if (j < R) {
      xc[h] = fmaxf(0.0f, out[j]);
      yc[h] = fminf(0.0f, s * out[R + j]);
      xo[h] = At[row * R + j];
      m[h] = M[row * R + j];
      xs[j] = xc[h];
      xs[64 + j] = xo[h];
    }
  }
  __syncwarp();
  float rc = 0.0f, ro = 0.0f, qc = 0.0f, qo = 0.0f;  // q: twice the row objective
  for (int h = 0; h < 2; ++h) {
    const int j = lane + 32 * h;
    if (j >= R) continue;
    float gc = -m[h], go = -m[h];
    for (int k = 0; k < R; ++k) {
      const float gk = G[k * R + j];  // G symmetric
      gc = fmaf(gk, xs[k], gc);
      go = fmaf(gk, xs[64 + k], go);
    }
    const float a = fminf(xc[h], gc), b = fminf(xo[h], go);
    rc += a * a;
    ro += b * b;
    qc += xc[h] * (gc - m[h]);
    qo += xo[h] * (go - m[h]);
  }
  for (int off = 16; off > 0; off >>= 1) {
    rc += __shfl_xor_sync(0xffffffffu, rc, off);
    ro += __shfl_xor_sync(0xffffffffu, ro, off);
    qc += __shfl_xor_sync(0xffffffffu, qc, off);
    qo += __shfl_xor_sync(0xffffffffu, qo, off);
  }
  const bool take = rc < ro && qc < qo;
  if (take) {
    for (int h = 0; h < 2; ++h) {
      const int j = lane + 32 * h;
      if (j < R) {
        At[row * R + j] = xc[h];
        Y[row * R + j] = yc[h];
      }
    }
  }
  if (lane == 0) {
    atomicAdd(&counters[0], 1ull);
    if (take) atomicAdd(&counters[1], 1ull);
  }
}

// Sums of v[0..7] over the 32 lanes: lane l returns the sum for row (l >> 2) & 7.  Halves of
// the set are exchanged at distances 16, 8, 4 (each lane keeps the half its lane bit selects
// and adds its partner's copy), then distances 2 and 1 complete the sum.
__device__ __forceinline__ float rows8_sum(const float (&v)[kWsRows], int lane) {
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
  float w[4], u[2];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float send = b4 ? v[i] : v[i + 4];
    const float keep = b4 ? v[i + 4] : v[i];
    w[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const float send = b3 ? w[i] : w[i + 2];
    const float keep = b3 ? w[i + 2] : w[i];
    u[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  float t = (b2 ? u[1] : u[0]) + __shfl_xor_sync(0xffffffffu, b2 ? u[0] : u[1], 4);
  t += __shfl_xor_sync(0xffffffffu, t, 2);
  t += __shfl_xor_sync(0xffffffffu, t, 1);
  return t;
}

// One layer for the CTA's rows: y[r][o] = act(b[o] + W[o, 0:K] x[r]) for o < Nout, W
// [Nout][K] (BF16), b, x [kWsRows][K] and y [kWsRows][ldy] in shared memory, K <= kWsMaxK;
// warp w of nw forms outputs w, w + nw, ...
template <bool kGelu>
__device__ __forceinline__ void ws_layer(const __nv_bfloat16* W, int K, int Nout,
                                         const float* bias, const float* x, float* y, int ldy,
                                         int warp, int nw, int lane) {
  float xr[kWsMaxK / 32][kWsRows];
#pragma unroll
  for (int j = 0; j < kWsMaxK / 32; ++j)
#pragma unroll
    for (int r = 0; r < kWsRows; ++r) {
      const int k = lane + 32 * j;
      xr[j][r] = k < K ? x[r * K + k] : 0.0f;
    }
  const int rl = (lane >> 2) & 7;
  // four outputs per pass, so that their exchange trees overlap
  for (int o0 = 4 * warp; o0 < Nout; o0 += 4 * nw) {
    float acc[4][kWsRows] = {};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int o = o0 + q < Nout ? o0 + q : Nout - 1;  // (a repeat past the end is dropped)
      const __nv_bfloat16* w = W + o * K;
#pragma unroll
      for (int j = 0; j < kWsMaxK / 32; ++j) {
        const int k = lane + 32 * j;
        if (32 * j < K) {
          const float wk = k < K ? __bfloat162float(w[k]) : 0.0f;
#pragma unroll
          for (int r = 0; r < kWsRows; ++r) acc[q][r] = fmaf(xr[j][r], wk, acc[q][r]);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int o = o0 + q;
      const float t = rows8_sum(acc[q], lane);
      if ((lane & 3) == 0 && o < Nout) {  // rows past nr: from zeros
        const float z = t + bias[o];
        y[rl * ldy + o] = kGelu ? gelu(z) : z;
      }
    }
  }
}

// n BF16 values from global to shared memory: asynchronous 16-byte copies (cp.async, all in
// flight until ws_stage_wait) when both ends allow, else plain loads eight at a time.
// (rot: where the copy order starts, so that CTAs copying the same block begin at different
// places of it and spread over the L2 slices)
__device__ __forceinline__ void ws_stage(__nv_bfloat16* dst, const __nv_bfloat16* src, int n,
                                         int tid, int nt, int rot = 0) {
  if (((reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(src)) & 15) == 0 &&
      n % 8 == 0) {
    const int n8 = n / 8;
    for (int i0 = tid; i0 < n8; i0 += nt) {
      const int i = (i0 + rot) % n8;
      const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst + 8 * i));
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src + 8 * i)
                   : "memory");
    }
  } else {
    for (int i0 = tid; i0 < n; i0 += 8 * nt) {
      __nv_bfloat16 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (i0 + u * nt < n) v[u] = src[i0 + u * nt];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (i0 + u * nt < n) dst[i0 + u * nt] = v[u];
    }
  }
}
__device__ __forceinline__ void ws_stage_wait() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

constexpr int kWsThreads = 512;

// trace(G) by one warp in a fixed order (lane l adds the diagonal entries l, l + 32, then a
// butterfly), the same in both warm-start kernels
__device__ __forceinline__ float ws_trace(const float* G, int R, int lane) {
  float t = 0.0f;
  for (int i = lane; i < R; i += 32) t += G[i * R + i];
  for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
  return t;
}

// The group term of the first layer, hG = W1_G vec(G/s) (s = trace(G)/R), once per factor:
// warp per hidden unit, lanes along the R^2 inputs.
__global__ void __launch_bounds__(256)
    k_ws_group(MlpShape s, const __nv_bfloat16* __restrict__ pb, const float* __restrict__ G,
               float* __restrict__ hG) {
  const int R = s.R, RR = R * R, lane = threadIdx.x & 31;
  const int h = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (h >= s.H) return;  // whole warps
  const float inv = 1.0f / (ws_trace(G, R, lane) / R);
  const __nv_bfloat16* w = pb + s.oW1 + static_cast<int64_t>(h) * s.Din;
  float g = 0.0f;
  for (int k0 = 0; k0 < RR; k0 += 32 * 16) {
    float gv[16], wv[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int k = k0 + lane + 32 * j;
      gv[j] = k < RR ? G[k] : 0.0f;
      wv[j] = k < RR ? __bfloat162float(w[k]) : 0.0f;
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) g = fmaf(gv[j] * inv, wv[j], g);
  }
  for (int off = 16; off > 0; off >>= 1) g += __shfl_xor_sync(0xffffffffu, g, off);
  if (lane == 0) hG[h] = g;
}

size_t ws_fused_smem(const MlpShape& s) {
  const size_t RR = static_cast<size_t>(s.R) * s.R, H = s.H, P = s.P, D = s.Dout;
  const size_t wbytes = (H * H + D * H + H * P) * sizeof(__nv_bfloat16);
  const size_t fbytes =
      (2 * RR + kWsRows * (s.R + P + 2 * H + D) + 3 * H + D + kWsRows * 128) * sizeof(float);
  return ((wbytes + 15) / 16) * 16 + fbytes;
}

__global__ void __launch_bounds__(kWsThreads)
    k_ws_fused(MlpShape s, const float* __restrict__ p, const __nv_bfloat16* __restrict__ pb,
               const float* __restrict__ hG, const float* __restrict__ G,
               const float* __restrict__ Hinv, const float* __restrict__ M,
               float* __restrict__ At, float* __restrict__ Y, int64_t I,
               unsigned long long* counters) {
  extern __shared__ __align__(16) unsigned char ws_smem[];
  __shared__ float s_scale[2];
  const int R = s.R, P = s.P, H = s.H, D = s.Dout, RR = R * R;
  __nv_bfloat16* sW2 = reinterpret_cast<__nv_bfloat16*>(ws_smem);  // [H][H]
  __nv_bfloat16* sW3 = sW2 + H * H;                                  // [D][H]
  __nv_bfloat16* sW1u = sW3 + D * H;                                 // [H][P]
  const size_t wbytes = (static_cast<size_t>(H) * H + D * H + H * P) * sizeof(__nv_bfloat16);
  float* sG = reinterpret_cast<float*>(ws_smem + ((wbytes + 15) / 16) * 16);  // [RR] G
  float* sHi = sG + RR;           // [RR] (G + rho I)^{-1}
  float* sM = sHi + RR;           // [kWsRows][R] MTTKRP rows
  float* su = sM + kWsRows * R;   // [kWsRows][P] per-row inputs
  float* sh1 = su + kWsRows * P;  // [kWsRows][H]
  float* sh2 = sh1 + kWsRows * H; // [kWsRows][H]
  float* sout = sh2 + kWsRows * H;// [kWsRows][D]
  float* sg = sout + kWsRows * D; // [H] group term + b1
  float* sb2 = sg + H;            // [H]
  float* sb3 = sb2 + H;           // [D]
  float* sxs = sb3 + D;           // [kWsRows][128] judge scratch
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nt = blockDim.x;
  const int nw = nt >> 5;
  const int64_t row0 = static_cast<int64_t>(blockIdx.x) * kWsRows;
  const int nr = static_cast<int>(I - row0 < kWsRows ? I - row0 : kWsRows);
  // the small inputs first (one round of loads), then the weights of layers 2, 3 and the
  // per-row part of layer 1 by asynchronous copies, in flight while the inputs are formed
  for (int i = tid; i < RR; i += nt) {
    sG[i] = G[i];
    sHi[i] = Hinv[i];
  }
  for (int i = tid; i < kWsRows * R; i += nt) sM[i] = i < nr * R ? M[row0 * R + i] : 0.0f;
  for (int i = tid; i < H; i += nt) {
    sg[i] = hG[i] + p[s.ob1 + i];
    sb2[i] = p[s.ob2 + i];
  }
  for (int i = tid; i < D; i += nt) sb3[i] = p[s.ob3 + i];
  const int rot = blockIdx.x * 997;
  ws_stage(sW2, pb + s.oW2, H * H, tid, nt, rot);
  ws_stage(sW3, pb + s.oW3, D * H, tid, nt, rot);
  for (int h0 = 0; h0 < H; h0 += nw) {  // the per-row columns of W1, row by row
    const int h = (h0 + warp + blockIdx.x) % H;
    if (h0 + warp < H)
      ws_stage(sW1u + h * P, pb + s.oW1 + static_cast<int64_t>(h) * s.Din + RR, P, lane, 32);
  }
  __syncthreads();
  if (warp == 0) {
    const float tr = ws_trace(sG, R, lane);
    if (lane == 0) {
      const float sc = tr / R;
      s_scale[0] = sc;
      s_scale[1] = 1.0f / sc;
    }
  }
  __syncthreads();
  const float sc = s_scale[0], inv = s_scale[1];
  for (int i = tid; i < kWsRows * P; i += nt) {
    const int r = i / P, c = i - r * P;
    const float* m = sM + r * R;  // zeros past nr
    float v;
    if (c < R) {
      v = m[c] * inv;
    } else {
      v = 0.0f;
      for (int j = 0; j < R; ++j) v = fmaf(sHi[j * R + (c - R)], m[j], v);  // Hinv symmetric
    }
    su[i] = v;
  }
  ws_stage_wait();
  __syncthreads();
  ws_layer<true>(sW1u, P, H, sg, su, sh1, H, warp, nw, lane);
  __syncthreads();
  ws_layer<true>(sW2, H, H, sb2, sh1, sh2, H, warp, nw, lane);
  __syncthreads();
  ws_layer<false>(sW3, H, D, sb3, sh2, sout, D, warp, nw, lane);
  __syncthreads();
  if (warp < nr)
    ws_judge_row(sout + warp * D, sG, M, sc, At, Y, row0 + warp, R, sxs + warp * 128, lane,
                 counters);
}

}  // namespace

bool ws_fused_ok(const MlpShape& s) {
  return s.H <= kWsMaxK && s.P <= kWsMaxK && ws_fused_smem(s) <= 220 * 1024;
}

cudaError_t ws_fused(const MlpShape& s, const float* p, const __nv_bfloat16* pb, float* hG,
                     const float* G, const float* Hinv, const float* M, float* At, float* Y,
                     int64_t I, unsigned long long* counters, cudaStream_t st) {
  const size_t smem = ws_fused_smem(s);
  cudaError_t e = cudaFuncSetAttribute(k_ws_fused, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  k_ws_group<<<(s.H + 7) / 8, 256, 0, st>>>(s, pb, G, hG);
  k_ws_fused<<<static_cast<unsigned>((I + kWsRows - 1) / kWsRows), kWsThreads, smem, st>>>(
      s, p, pb, hG, G, Hinv, M, At, Y, I, counters);
  return cudaGetLastError();
}

cudaError_t ws_prepare(const float* G, const float* Hinv, const float* M, int R, int64_t I,
                       float* Gn, float* mrows, float* s_out, cudaStream_t st) {
  const int64_t n = static_cast<int64_t>(R) * R + I * 2 * R;
  k_ws_prepare<<<blocks_for(n), 256, 0, st>>>(G, Hinv, M, R, I, Gn, mrows, s_out);
  return cudaGetLastError();
}

// Training targets of factor rows: out[row] = [At_row ; Y_row / s] (s = trace(G)/R on the
// device), the network's output layout.
__global__ void k_ws_targets(const float* __restrict__ At, const float* __restrict__ Y,
                             const float* __restrict__ s_ptr, int R, int64_t I,
                             float* __restrict__ out) {
  const float inv = 1.0f / *s_ptr;
  const int64_t n = I * 2 * R;
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < n;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t row = k / (2 * R);
    const int c = static_cast<int>(k % (2 * R));
    out[k] = c < R ? At[row * R + c] : Y[row * R + c - R] * inv;
  }
}

cudaError_t ws_targets(const float* At, const float* Y, const float* s_ptr, int R, int64_t I,
                       float* out, cudaStream_t st) {
  const int64_t n = I * 2 * R;
  k_ws_targets<<<blocks_for(n), 256, 0, st>>>(At, Y, s_ptr, R, I, out);
  return cudaGetLastError();
}

cudaError_t ws_judge(const float* out, const float* G, const float* M, const float* s_ptr,
                     float* At, float* Y, int64_t I, int R, unsigned long long* counters,
                     cudaStream_t st) {
  k_ws_judge<<<static_cast<unsigned>((I + 7) / 8), 256, 0, st>>>(out, G, M, s_ptr, At, Y, I, R,
                                                                 counters);
  return cudaGetLastError();
}

}  // namespace ntf
