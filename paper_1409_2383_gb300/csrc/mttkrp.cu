// MTTKRP building blocks (Sec. IV-A item 1 of Liavas & Sidiropoulos).
//
// The tensor is viewed as a row-major matrix X[P, Q] (P = product of the leading modes,
// Q = product of the trailing ones).  Every MTTKRP is one of two skinny contractions of such a
// view followed by a small reduction that applies the remaining factor of the mode's group:
//
//   GEMM-N:  T_R[p, r] = sum_q X[p, q] * W[q, r]     W = Khatri-Rao rows of the trailing factors
//   GEMM-T:  T_L[q, r] = sum_p X[p, q] * W[p, r]     W = Khatri-Rao rows of the leading factors
//
// W is built once per contraction into a zero-padded [K_pad, RP] table (K = contraction
// length) and read through L1 by every CTA.  Both contractions stream X from HBM exactly once
// with 16-byte cp.async and FP32 accumulation (FP32 or BF16 storage).  When the contraction
// range is split across CTAs the partial sums are added by a separate kernel in a fixed order,
// so every result is deterministic.
#include <algorithm>
#include <cstdio>

#include "mttkrp_kernels.cuh"

namespace ntf {
namespace detail {
// One instantiation unit per storage type and contraction (gemm_{n,t}_{f32,bf16}.cu).
extern template cudaError_t gemm_n_typed<float>(const float*, int64_t, int64_t, int,
                                                const float*, const GemmPlan&, float*,
                                                cudaStream_t);
extern template cudaError_t gemm_n_typed<__nv_bfloat16>(const __nv_bfloat16*, int64_t, int64_t,
                                                        int, const float*, const GemmPlan&,
                                                        float*, cudaStream_t);
extern template cudaError_t gemm_t_typed<float>(const float*, int64_t, int64_t, int,
                                                const float*, const GemmPlan&, float*,
                                                cudaStream_t);
extern template cudaError_t gemm_t_typed<__nv_bfloat16>(const __nv_bfloat16*, int64_t, int64_t,
                                                        int, const float*, const GemmPlan&,
                                                        float*, cudaStream_t);
}  // namespace detail

namespace {
using namespace detail;
// Entry r of Khatri-Rao row q of a group (last mode fastest).
__device__ __forceinline__ float kr_entry(const Group& g, int64_t q, int r, int R) {
  float v = 1.0f;
#pragma unroll
  for (int j = 2; j >= 0; --j) {
    if (j < g.n) {
      const int64_t d = g.dim[j];
      const int64_t i = q % d;
      q /= d;
      v *= __ldg(g.F[j] + i * R + r);
    }
  }
  return v;
}

// W[q, r] = Khatri-Rao row q of the group for q < K and r < R; 0 in the padding.
__global__ void k_kr_table(Group g, int64_t K, int R, int RP, int64_t n, float* __restrict__ W) {
  for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < n;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t q = idx / RP;
    const int r = static_cast<int>(idx % RP);
    W[idx] = (q < K && r < R) ? kr_entry(g, q, r, R) : 0.0f;
  }
}

// Split Khatri-Rao table of the tensor-core contractions: [splits * N rows][K_pad], K
// contiguous; row s * N + r holds part s of column r (split_store).
template <bool kBF16>
__global__ void k_kr_split(Group g, int64_t K, int R, int N, int64_t K_pad, void* __restrict__ W) {
  const int64_t n = static_cast<int64_t>(N) * K_pad;
  for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < n;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int r = static_cast<int>(idx / K_pad);
    const int64_t q = idx % K_pad;
    const float w = (q < K && r < R) ? kr_entry(g, q, r, R) : 0.0f;
    split_store(W, n, idx, w, kBF16);
  }
}

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
    float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
    if (grp < groups) {
      const float* Ta = T + a * Ib * R;
      int64_t b = grp;
      for (; b + 3 * groups < Ib; b += 4 * groups) {
        s0 = fmaf(Ta[b * R + r], __ldg(F + b * R + r), s0);
        s1 = fmaf(Ta[(b + groups) * R + r], __ldg(F + (b + groups) * R + r), s1);
        s2 = fmaf(Ta[(b + 2 * groups) * R + r], __ldg(F + (b + 2 * groups) * R + r), s2);
        s3 = fmaf(Ta[(b + 3 * groups) * R + r], __ldg(F + (b + 3 * groups) * R + r), s3);
      }
      for (; b < Ib; b += groups) s0 = fmaf(Ta[b * R + r], __ldg(F + b * R + r), s0);
    }
    red[tid] = (s0 + s1) + (s2 + s3);
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
  float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
  int64_t a = a_beg;
  for (; a + 3 < a_end; a += 4) {
    s0 = fmaf(T[(a * Ib + b) * R + r], __ldg(F + a * R + r), s0);
    s1 = fmaf(T[((a + 1) * Ib + b) * R + r], __ldg(F + (a + 1) * R + r), s1);
    s2 = fmaf(T[((a + 2) * Ib + b) * R + r], __ldg(F + (a + 2) * R + r), s2);
    s3 = fmaf(T[((a + 3) * Ib + b) * R + r], __ldg(F + (a + 3) * R + r), s3);
  }
  for (; a < a_end; ++a) s0 = fmaf(T[(a * Ib + b) * R + r], __ldg(F + a * R + r), s0);
  out[(static_cast<int64_t>(split) * Ib + b) * R + r] = (s0 + s1) + (s2 + s3);
}

// Vectorised second tree level for R % 4 == 0 (T, F, out 16-byte aligned), Q = R / 4 float4
// chunks per row.
//
// fast: out[a, :] = sum_b T[a, b, :] * F[b, :].  One CTA (32 Q threads) per a; the slab
// T[a] (Ib Q float4, contiguous) is read in order: thread t takes chunk q = t % Q of rows
// b = t / Q, t / Q + 32, ... (eight rows in flight), so consecutive threads read
// consecutive float4; then the 32 partial sums of each chunk are added in a fixed order
// through shared memory.
__global__ void __launch_bounds__(512) k_post_fast4(const float4* __restrict__ T, int64_t Ia,
                                                   int64_t Ib, int Q,
                                                   const float4* __restrict__ F,
                                                   float4* __restrict__ out) {
  __shared__ float4 part[512];
  const int t = threadIdx.x, q = t % Q, b0 = t / Q;
  for (int64_t a = blockIdx.x; a < Ia; a += gridDim.x) {
    const float4* Ta = T + a * Ib * Q;
    float4 s[2] = {make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f)};
    for (int64_t bb = b0; bb < Ib; bb += 32 * 8) {
      float4 tv[8], fv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int64_t b = bb + 32 * u;
        tv[u] = fv[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (b < Ib) {
          tv[u] = Ta[b * Q + q];
          fv[u] = __ldg(F + b * Q + q);
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        s[u & 1].x = fmaf(tv[u].x, fv[u].x, s[u & 1].x);
        s[u & 1].y = fmaf(tv[u].y, fv[u].y, s[u & 1].y);
        s[u & 1].z = fmaf(tv[u].z, fv[u].z, s[u & 1].z);
        s[u & 1].w = fmaf(tv[u].w, fv[u].w, s[u & 1].w);
      }
    }
    part[t] = make_float4(s[0].x + s[1].x, s[0].y + s[1].y, s[0].z + s[1].z, s[0].w + s[1].w);
    __syncthreads();
    if (t < Q) {  // chunk t: partials t, t + Q, ..., t + 31 Q
      float4 v = part[t];
      for (int j = 1; j < 32; ++j) {
        const float4 p = part[t + j * Q];
        v.x += p.x;
        v.y += p.y;
        v.z += p.z;
        v.w += p.w;
      }
      out[a * Q + t] = v;
    }
    __syncthreads();
  }
}

// The same for even R that is not a multiple of 4, in float2 vectors (R <= 64: up to 32 Q =
// 1024 threads).  The kernels below are written over the vector type V and instantiated for
// float2 only (float4 instances of them ran 18 % slower than the kernels above).
template <typename V>
constexpr int kPostMaxThreads = 1024;
// b-block of the slow level in float2 vectors: 8 rows (8 Q <= 256 threads: a CTA fits on an
// SM beside a persistent contraction CTA, which the 32-row block of up to 1024 threads
// does not, and the level runs beside the contraction in a sweep)
constexpr int kPostBB2 = 8;
template <typename V> __device__ __forceinline__ V vzero();
template <> __device__ __forceinline__ float2 vzero<float2>() { return make_float2(0.f, 0.f); }
__device__ __forceinline__ void vfma(float2& s, const float2& a, const float2& b) {
  s.x = fmaf(a.x, b.x, s.x);
  s.y = fmaf(a.y, b.y, s.y);
}
__device__ __forceinline__ void vadd(float2& s, const float2& p) {
  s.x += p.x;
  s.y += p.y;
}

// The fast level in V vectors (Q = R / V's width per row; T, F, out aligned to V):
// out[a, :] = sum_b T[a, b, :] * F[b, :].  One CTA (32 Q threads) per a; the slab
// T[a] (Ib Q vectors, contiguous) is read in order: thread t takes vector q = t % Q of rows
// b = t / Q, t / Q + 32, ... (eight rows in flight), so consecutive threads read
// consecutive vectors; then the 32 partial sums of each vector are added in a fixed order
// through shared memory.
template <typename V>
__global__ void __launch_bounds__(kPostMaxThreads<V>) k_post_fastv(const V* __restrict__ T, int64_t Ia,
                                                    int64_t Ib, int Q, const V* __restrict__ F,
                                                    V* __restrict__ out) {
  __shared__ V part[1024];
  const int t = threadIdx.x, q = t % Q, b0 = t / Q;
  for (int64_t a = blockIdx.x; a < Ia; a += gridDim.x) {
    const V* Ta = T + a * Ib * Q;
    V s[2] = {vzero<V>(), vzero<V>()};
    for (int64_t bb = b0; bb < Ib; bb += 32 * 8) {
      V tv[8], fv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int64_t b = bb + 32 * u;
        tv[u] = fv[u] = vzero<V>();
        if (b < Ib) {
          tv[u] = Ta[b * Q + q];
          fv[u] = __ldg(F + b * Q + q);
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) vfma(s[u & 1], tv[u], fv[u]);
    }
    vadd(s[0], s[1]);
    part[t] = s[0];
    __syncthreads();
    if (t < Q) {  // vector t: partials t, t + Q, ..., t + 31 Q
      V v = part[t];
      for (int j = 1; j < 32; ++j) vadd(v, part[t + j * Q]);
      out[a * Q + t] = v;
    }
    __syncthreads();
  }
}

// The last step of the second tree level formed in the GEMM-N epilogue: the 32-row groups
// holding rows of a summed per row.  Each row a takes kPartWarps warps (lane = r), each the
// sums of a quarter of its groups in increasing order, eight loads in flight; the quarters
// are added in order 0, 1, ... through shared memory (a fixed order: deterministic).
constexpr int kPartWarps = 4;
__global__ void __launch_bounds__(256) k_post_part(const float* __restrict__ part, int64_t Ia,
                                                   int64_t Ib, int R, float* __restrict__ out) {
  __shared__ float s_sum[8][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = warp % kPartWarps;
  const int64_t a = static_cast<int64_t>(blockIdx.x) * (8 / kPartWarps) + warp / kPartWarps;
  float acc = 0.0f;
  if (a < Ia && lane < R) {
    const int64_t g0 = (a * Ib) / 32, g1 = ((a + 1) * Ib - 1) / 32, n = g1 - g0 + 1;
    // the first group may hold a's rows in its second slot; every later one in its first
    const int64_t slot0 = a - (g0 * 32) / Ib;
    const int64_t k0 = n * q / kPartWarps, k1 = n * (q + 1) / kPartWarps;
    for (int64_t k = k0; k < k1; k += 8) {
      float v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int64_t kk = k + u;
        v[u] = kk < k1 ? part[((g0 + kk) * 2 + (kk == 0 ? slot0 : 0)) * R + lane] : 0.0f;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) acc += v[u];
    }
  }
  s_sum[warp][lane] = acc;
  __syncthreads();
  if (q == 0 && a < Ia && lane < R) {
    float t = s_sum[warp][lane];
#pragma unroll
    for (int j = 1; j < kPartWarps; ++j) t += s_sum[warp + j][lane];
    out[a * R + lane] = t;
  }
}

// slow: out[b, :] = sum_a T[a, b, :] * F[a, :].  CTA (b-block of kPostBB rows, a-split):
// thread (bb, chunk) accumulates over its split's a-range; every CTA writes its partial,
// and the last CTA of a b-block to finish (counter) adds the splits in order 0, 1, ... and
// resets the counter.
constexpr int kPostBB = 32;
__global__ void k_post_slow4(const float4* __restrict__ T, int64_t Ia, int64_t Ib, int Q,
                             const float4* __restrict__ F, int splits,
                             float4* __restrict__ partial, unsigned* __restrict__ count,
                             float4* __restrict__ out) {
  const int split = blockIdx.y;
  const int64_t b0 = static_cast<int64_t>(blockIdx.x) * kPostBB;
  const int t = threadIdx.x;
  const int bb = t / Q, q = t - bb * Q;
  const int64_t b = b0 + bb;
  const int64_t a_beg = Ia * split / splits, a_end = Ia * (split + 1) / splits;
  float4 s[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) s[u] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (b < Ib) {
    int64_t a = a_beg;
    for (; a + 7 < a_end; a += 8) {  // eight rows' loads in flight
      float4 tv[8], fv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        tv[u] = T[((a + u) * Ib + b) * Q + q];
        fv[u] = __ldg(F + (a + u) * Q + q);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        s[u & 3].x = fmaf(tv[u].x, fv[u].x, s[u & 3].x);
        s[u & 3].y = fmaf(tv[u].y, fv[u].y, s[u & 3].y);
        s[u & 3].z = fmaf(tv[u].z, fv[u].z, s[u & 3].z);
        s[u & 3].w = fmaf(tv[u].w, fv[u].w, s[u & 3].w);
      }
    }
    for (; a + 3 < a_end; a += 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float4 tv = T[((a + u) * Ib + b) * Q + q], f = __ldg(F + (a + u) * Q + q);
        s[u].x = fmaf(tv.x, f.x, s[u].x);
        s[u].y = fmaf(tv.y, f.y, s[u].y);
        s[u].z = fmaf(tv.z, f.z, s[u].z);
        s[u].w = fmaf(tv.w, f.w, s[u].w);
      }
    }
    for (; a < a_end; ++a) {
      const float4 tv = T[(a * Ib + b) * Q + q], f = __ldg(F + a * Q + q);
      s[0].x = fmaf(tv.x, f.x, s[0].x);
      s[0].y = fmaf(tv.y, f.y, s[0].y);
      s[0].z = fmaf(tv.z, f.z, s[0].z);
      s[0].w = fmaf(tv.w, f.w, s[0].w);
    }
  }
  float4 v;
  v.x = (s[0].x + s[1].x) + (s[2].x + s[3].x);
  v.y = (s[0].y + s[1].y) + (s[2].y + s[3].y);
  v.z = (s[0].z + s[1].z) + (s[2].z + s[3].z);
  v.w = (s[0].w + s[1].w) + (s[2].w + s[3].w);
  if (splits == 1) {
    if (b < Ib) out[b * Q + q] = v;
    return;
  }
  if (b < Ib) partial[(static_cast<int64_t>(split) * Ib + b) * Q + q] = v;
  __shared__ int s_last;
  __threadfence();
  __syncthreads();
  if (t == 0) s_last = atomicAdd(count + blockIdx.x, 1u) == static_cast<unsigned>(splits - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (b < Ib) {
    // splits added in order 0, 1, ...; loads issued eight at a time (independent) so that
    // the L2 round trips overlap
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    int k = 0;
    for (; k + 8 <= splits; k += 8) {
      float4 p[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        p[u] = __ldcg(partial + (static_cast<int64_t>(k + u) * Ib + b) * Q + q);
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        acc.x += p[u].x;
        acc.y += p[u].y;
        acc.z += p[u].z;
        acc.w += p[u].w;
      }
    }
    for (; k < splits; ++k) {
      const float4 p = __ldcg(partial + (static_cast<int64_t>(k) * Ib + b) * Q + q);
      acc.x += p.x;
      acc.y += p.y;
      acc.z += p.z;
      acc.w += p.w;
    }
    out[b * Q + q] = acc;
  }
  if (t == 0) count[blockIdx.x] = 0;
}

template <typename V>
__global__ void __launch_bounds__(kPostMaxThreads<V>) k_post_slowv(const V* __restrict__ T, int64_t Ia,
                                                    int64_t Ib, int Q, const V* __restrict__ F,
                                                    int splits, V* __restrict__ partial,
                                                    unsigned* __restrict__ count,
                                                    V* __restrict__ out) {
  const int split = blockIdx.y;
  const int64_t b0 = static_cast<int64_t>(blockIdx.x) * kPostBB2;
  const int t = threadIdx.x;
  const int bb = t / Q, q = t - bb * Q;
  const int64_t b = b0 + bb;
  const int64_t a_beg = Ia * split / splits, a_end = Ia * (split + 1) / splits;
  V s[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) s[u] = vzero<V>();
  if (b < Ib) {
    int64_t a = a_beg;
    for (; a + 7 < a_end; a += 8) {  // eight rows' loads in flight
      V tv[8], fv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        tv[u] = T[((a + u) * Ib + b) * Q + q];
        fv[u] = __ldg(F + (a + u) * Q + q);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) vfma(s[u & 3], tv[u], fv[u]);
    }
    for (; a + 3 < a_end; a += 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u) vfma(s[u], T[((a + u) * Ib + b) * Q + q], __ldg(F + (a + u) * Q + q));
    }
    for (; a < a_end; ++a) vfma(s[0], T[(a * Ib + b) * Q + q], __ldg(F + a * Q + q));
  }
  vadd(s[0], s[1]);
  vadd(s[2], s[3]);
  vadd(s[0], s[2]);
  const V v = s[0];
  if (splits == 1) {
    if (b < Ib) out[b * Q + q] = v;
    return;
  }
  if (b < Ib) partial[(static_cast<int64_t>(split) * Ib + b) * Q + q] = v;
  __shared__ int s_last;
  __threadfence();
  __syncthreads();
  if (t == 0) s_last = atomicAdd(count + blockIdx.x, 1u) == static_cast<unsigned>(splits - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (b < Ib) {
    // splits added in order 0, 1, ...; loads issued eight at a time (independent) so that
    // the L2 round trips overlap
    V acc = vzero<V>();
    int k = 0;
    for (; k + 8 <= splits; k += 8) {
      V pv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        pv[u] = __ldcg(partial + (static_cast<int64_t>(k + u) * Ib + b) * Q + q);
#pragma unroll
      for (int u = 0; u < 8; ++u) vadd(acc, pv[u]);
    }
    for (; k < splits; ++k) vadd(acc, __ldcg(partial + (static_cast<int64_t>(k) * Ib + b) * Q + q));
    out[b * Q + q] = acc;
  }
  if (t == 0) count[blockIdx.x] = 0;
}

// ||X||^2: every thread sums the squares of its elements (16-byte loads where aligned) as a
// pair of FP32 numbers hi + lo: each square is split exactly into p + e (p = v v rounded,
// e = fma(v, v, -p)), p is added to hi by Knuth's two-sum, whose exact error goes to lo with
// e (relative error of the pair about 2^-44); the block adds the threads' hi + lo in FP64 by
// a fixed tree, and k_sum_doubles adds the blocks' in FP64 in a fixed order.  (FP64 per
// element would run at this GPU's FP64 rate, a small fraction of its FP32 rate.)
template <typename T>
__global__ void k_norm2(const T* __restrict__ X, int64_t n, double* __restrict__ partial) {
  __shared__ double red[256];
  float hi = 0.0f, lo = 0.0f;
  const auto add = [&](float v) {  // (rounded operations that the compiler may not fuse)
    const float p = __fmul_rn(v, v);
    const float e = fmaf(v, v, -p);
    const float s = __fadd_rn(hi, p);
    const float bb = __fsub_rn(s, hi);
    lo = __fadd_rn(lo, __fadd_rn(__fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb)), e));
    hi = s;
  };
  constexpr int kV = Elem<T>::kPer16;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int64_t tid = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  int64_t done = 0;
  if ((reinterpret_cast<uintptr_t>(X) & 15) == 0) {
    const int64_t nv = n / kV;
    const uint4* X4 = reinterpret_cast<const uint4*>(X);
    for (int64_t i = tid; i < nv; i += stride) {
      float f[kV];
      Elem<T>::unpack16(__ldg(X4 + i), f);
#pragma unroll
      for (int u = 0; u < kV; ++u) add(f[u]);
    }
    done = nv * kV;
  }
  for (int64_t i = done + tid; i < n; i += stride) add(Elem<T>::load1(X + i));
  red[threadIdx.x] = static_cast<double>(hi) + static_cast<double>(lo);
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// out = sum of v[0..n): one warp, lane l adds v[l], v[l + 32], ..., then a fixed butterfly.
__global__ void k_sum_doubles(const double* __restrict__ v, int n, double* __restrict__ out) {
  if (blockIdx.x != 0 || threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  double s = 0.0;
  for (int i = lane; i < n; i += 32) s += v[i];
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (lane == 0) *out = s;
}

// FP32 -> BF16, round to nearest even.  16-byte loads and 8-byte stores when both arrays
// allow (the input may be host memory that the device reads over the host link: wide reads
// matter there), then the tail one by one.
__global__ void k_to_bf16(const float* __restrict__ in, __nv_bfloat16* __restrict__ out,
                          int64_t n) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int64_t tid = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  int64_t done = 0;
  if (((reinterpret_cast<uintptr_t>(in) & 15) | (reinterpret_cast<uintptr_t>(out) & 7)) == 0) {
    const int64_t n4 = n / 4;
    const float4* in4 = reinterpret_cast<const float4*>(in);
    uint2* out4 = reinterpret_cast<uint2*>(out);
    for (int64_t i = tid; i < n4; i += stride) {
      const float4 v = in4[i];
      const __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y);
      const __nv_bfloat162 b = __floats2bfloat162_rn(v.z, v.w);
      out4[i] = make_uint2(*reinterpret_cast<const uint32_t*>(&a),
                           *reinterpret_cast<const uint32_t*>(&b));
    }
    done = n4 * 4;
  }
  for (int64_t i = done + tid; i < n; i += stride) out[i] = __float2bfloat16_rn(in[i]);
}

}  // namespace

// ------------------------------------------------------------------------- plans
namespace {

// Tiles of 64 rows (GEMM-N) or 64 columns (GEMM-T).  The contraction range is split across
// CTAs only when there are too few tiles to fill the GPU several times over; a split range is
// a multiple of 64 long.
GemmPlan make_plan(int64_t tiles_extent, int64_t K, int dtype, const void* X, int64_t row_len,
                   int num_sms) {
  GemmPlan pl{};
  const int esize = dtype == NTF_BF16 ? 2 : 4;
  pl.vec16 = (row_len * esize) % 16 == 0 && (reinterpret_cast<uintptr_t>(X) % 16) == 0;
  const int64_t tiles = (tiles_extent + 63) / 64;
  pl.tiles = static_cast<int>(tiles);
  const int64_t want = static_cast<int64_t>(num_sms) * 8;
  int64_t chunks = tiles >= want ? 1 : (want + tiles - 1) / tiles;
  chunks = std::max<int64_t>(1, std::min<int64_t>(chunks, (K + 1023) / 1024));
  int64_t len = (K + chunks - 1) / chunks;
  len = ((len + 63) / 64) * 64;
  chunks = (K + len - 1) / len;
  if (!pl.vec16) {
    chunks = 1;
    len = K;
  }
  pl.chunks = static_cast<int>(chunks);
  pl.chunk_len = len;
  return pl;
}

}  // namespace

int round_rp(int R) { return detail::round_rp(R); }
int64_t kr_rows_padded(int64_t K) { return ((K + 63) / 64) * 64; }

GemmPlan plan_gemm_n(int64_t P, int64_t Q, int dtype, const void* X, int num_sms) {
  return make_plan(P, Q, dtype, X, Q, num_sms);
}

GemmPlan plan_gemm_t(int64_t P, int64_t Q, int dtype, const void* X, int num_sms) {
  return make_plan(Q, P, dtype, X, Q, num_sms);
}

cudaError_t launch_kr_table(const Group& g, int64_t K, int R, float* W, cudaStream_t st) {
  const int RP = detail::round_rp(R);
  const int64_t n = kr_rows_padded(K) * RP;
  const unsigned blocks = static_cast<unsigned>(std::min<int64_t>((n + 255) / 256, 4096));
  k_kr_table<<<blocks, 256, 0, st>>>(g, K, R, RP, n, W);
  return cudaGetLastError();
}

cudaError_t launch_kr_split(const Group& g, const UmmaPlan& plan, int R, void* Wsplit,
                            cudaStream_t st) {
  const int64_t n = static_cast<int64_t>(plan.N) * plan.K_pad;
  const unsigned blocks = static_cast<unsigned>(std::min<int64_t>((n + 255) / 256, 4096));
  if (plan.f32)
    k_kr_split<false><<<blocks, 256, 0, st>>>(g, plan.args.K, R, plan.N, plan.K_pad, Wsplit);
  else
    k_kr_split<true><<<blocks, 256, 0, st>>>(g, plan.args.K, R, plan.N, plan.K_pad, Wsplit);
  return cudaGetLastError();
}

cudaError_t launch_gemm_n(const void* X, int dtype, int64_t P, int64_t Q, int R, const float* W,
                          const GemmPlan& plan, float* out, cudaStream_t st) {
  if (dtype == NTF_BF16)
    return detail::gemm_n_typed(static_cast<const __nv_bfloat16*>(X), P, Q, R, W, plan, out, st);
  return detail::gemm_n_typed(static_cast<const float*>(X), P, Q, R, W, plan, out, st);
}

cudaError_t launch_gemm_t(const void* X, int dtype, int64_t P, int64_t Q, int R, const float* W,
                          const GemmPlan& plan, float* out, cudaStream_t st) {
  if (dtype == NTF_BF16)
    return detail::gemm_t_typed(static_cast<const __nv_bfloat16*>(X), P, Q, R, W, plan, out, st);
  return detail::gemm_t_typed(static_cast<const float*>(X), P, Q, R, W, plan, out, st);
}

// Transposed copy of the tensor, y[Q, P] = x[P, Q]^T: 32 x 32 tiles through shared memory
// (rows of x read and rows of y written 32 elements at a time), tiles walked by a
// grid-stride loop.  Runs once per context.
template <typename T>
__global__ void __launch_bounds__(256) k_transpose(const T* __restrict__ x, int64_t P, int64_t Q,
                                                   T* __restrict__ y, int64_t ldy) {
  __shared__ T tile[32][33];
  const int64_t tp = (P + 31) / 32, tq = (Q + 31) / 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int64_t t = blockIdx.x; t < tp * tq; t += gridDim.x) {
    const int64_t p0 = (t / tq) * 32, q0 = (t % tq) * 32;
#pragma unroll
    for (int i = ty; i < 32; i += 8)
      if (p0 + i < P && q0 + tx < Q) tile[i][tx] = x[(p0 + i) * Q + q0 + tx];
    __syncthreads();
#pragma unroll
    for (int i = ty; i < 32; i += 8)
      if (q0 + i < Q && p0 + tx < P) y[(q0 + i) * ldy + p0 + tx] = tile[tx][i];
    __syncthreads();
  }
}

// The same for 16-bit elements with even P and Q: 64 x 64 tiles, rows of x read and rows of y
// written as 32-bit pairs (128 bytes per warp access on both sides).
__global__ void __launch_bounds__(256) k_transpose_pairs(const uint32_t* __restrict__ x,
                                                         int64_t P, int64_t Q,
                                                         uint32_t* __restrict__ y, int64_t ldyh) {
  __shared__ uint16_t tile[64][66];
  const int64_t tp = (P + 63) / 64, tq = (Q + 63) / 64, Ph = P / 2, Qh = Q / 2;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int64_t t = blockIdx.x; t < tp * tq; t += gridDim.x) {
    const int64_t p0 = (t / tq) * 64, q0 = (t % tq) * 64;
#pragma unroll
    for (int i = ty; i < 64; i += 8) {  // row p0 + i of x, columns q0 + 2 tx, q0 + 2 tx + 1
      const int64_t qp = q0 / 2 + tx;
      if (p0 + i < P && qp < Qh) {
        const uint32_t v = x[(p0 + i) * Qh + qp];
        tile[i][2 * tx] = static_cast<uint16_t>(v & 0xFFFFu);
        tile[i][2 * tx + 1] = static_cast<uint16_t>(v >> 16);
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = ty; i < 64; i += 8) {  // row q0 + i of y, columns p0 + 2 tx, p0 + 2 tx + 1
      const int64_t pp = p0 / 2 + tx;
      if (q0 + i < Q && pp < Ph)
        y[(q0 + i) * ldyh + pp] =
            static_cast<uint32_t>(tile[2 * tx][i]) | (static_cast<uint32_t>(tile[2 * tx + 1][i]) << 16);
    }
    __syncthreads();
  }
}

// Padded copy of the tensor: y[p, q] = x[p, q] for q < Q, 0 for Q <= q < ldy.
template <typename T>
__global__ void k_pad_rows(const T* __restrict__ x, int64_t P, int64_t Q, T* __restrict__ y,
                           int64_t ldy) {
  const int64_t n = P * ldy;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t p = i / ldy, q = i - p * ldy;
    y[i] = q < Q ? x[p * Q + q] : T(0);
  }
}

cudaError_t launch_pad_rows(const void* x, int es, int64_t P, int64_t Q, void* y, int64_t ldy,
                            cudaStream_t st) {
  if (P < 1 || Q < 1 || ldy < Q || (es != 2 && es != 4)) return cudaErrorInvalidValue;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const unsigned blocks =
      static_cast<unsigned>(std::min<int64_t>((P * ldy + 255) / 256, int64_t{16} * sms));
  if (es == 4)
    k_pad_rows<float><<<blocks, 256, 0, st>>>(static_cast<const float*>(x), P, Q,
                                               static_cast<float*>(y), ldy);
  else
    k_pad_rows<uint16_t><<<blocks, 256, 0, st>>>(static_cast<const uint16_t*>(x), P, Q,
                                                  static_cast<uint16_t*>(y), ldy);
  return cudaGetLastError();
}

cudaError_t launch_transpose(const void* x, int es, int64_t P, int64_t Q, void* y,
                             cudaStream_t st, int64_t ldy) {
  if (ldy == 0) ldy = P;
  if (P < 1 || Q < 1 || ldy < P || (es != 2 && es != 4)) return cudaErrorInvalidValue;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const bool pairs = es == 2 && P % 2 == 0 && Q % 2 == 0 && ldy % 2 == 0 &&
                     reinterpret_cast<uintptr_t>(x) % 4 == 0 && reinterpret_cast<uintptr_t>(y) % 4 == 0;
  if (pairs) {
    const int64_t tiles = ((P + 63) / 64) * ((Q + 63) / 64);
    const unsigned blocks = static_cast<unsigned>(std::min<int64_t>(tiles, int64_t{8} * sms));
    k_transpose_pairs<<<blocks, 256, 0, st>>>(static_cast<const uint32_t*>(x), P, Q,
                                               static_cast<uint32_t*>(y), ldy / 2);
    return cudaGetLastError();
  }
  const int64_t tiles = ((P + 31) / 32) * ((Q + 31) / 32);
  const unsigned blocks = static_cast<unsigned>(std::min<int64_t>(tiles, int64_t{8} * sms));
  if (es == 4)
    k_transpose<float><<<blocks, 256, 0, st>>>(static_cast<const float*>(x), P, Q,
                                                static_cast<float*>(y), ldy);
  else
    k_transpose<uint16_t><<<blocks, 256, 0, st>>>(static_cast<const uint16_t*>(x), P, Q,
                                                   static_cast<uint16_t*>(y), ldy);
  return cudaGetLastError();
}

cudaError_t launch_sum_splits(const float* partial, int splits, int64_t n, float* out,
                              cudaStream_t st) {
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);
  prefer_shared_carveout<k_sum_splits>();
  k_sum_splits<<<static_cast<unsigned>(std::max<int64_t>(blocks, 1)), 256, 0, st>>>(partial, splits, n, out);
  return cudaGetLastError();
}

cudaError_t launch_post_fast(const float* T, int64_t Ia, int64_t Ib, int R, const float* F,
                             float* out, cudaStream_t st) {
  const unsigned blocks = static_cast<unsigned>(std::min<int64_t>(Ia, 65535));
  prefer_shared_carveout<k_post_fast>();
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
  prefer_shared_carveout<k_post_slow>();
  k_post_slow<<<grid, 256, 0, st>>>(T, Ia, Ib, R, F, splits, dst);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || splits == 1) return e;
  return launch_sum_splits(partial, splits, Ib * R, out, st);
}

namespace {
// the vector type by the rank alone: float4 when R % 4 == 0, else float2 (even R)
bool post_vec4(int R) { return R % 4 == 0; }
int post_bb(int R) { return post_vec4(R) ? kPostBB : kPostBB2; }
}  // namespace

bool post4_ok(int R, const void* T, const void* F, const void* out) {
  const uintptr_t m = post_vec4(R) ? 15 : 7;
  const auto al = [m](const void* p) { return (reinterpret_cast<uintptr_t>(p) & m) == 0; };
  return (post_vec4(R) ? R <= 128 : R % 2 == 0 && R <= 64) && al(T) && al(F) && al(out);
}

cudaError_t launch_post_fast4(const float* T, int64_t Ia, int64_t Ib, int R, const float* F,
                              float* out, cudaStream_t st) {
  const unsigned blocks = static_cast<unsigned>(std::min<int64_t>(Ia, 65535));
  if (post_vec4(R)) {
    const int Q = R / 4;
    prefer_shared_carveout<k_post_fast4>();
    k_post_fast4<<<blocks, 32 * Q, 0, st>>>(reinterpret_cast<const float4*>(T), Ia, Ib, Q,
                                            reinterpret_cast<const float4*>(F),
                                            reinterpret_cast<float4*>(out));
  } else {
    const int Q = R / 2;
    prefer_shared_carveout<k_post_fastv<float2>>();
    k_post_fastv<float2><<<blocks, 32 * Q, 0, st>>>(reinterpret_cast<const float2*>(T), Ia,
                                                    Ib, Q, reinterpret_cast<const float2*>(F),
                                                    reinterpret_cast<float2*>(out));
  }
  return cudaGetLastError();
}

cudaError_t launch_post_part(const float* part, int64_t Ia, int64_t Ib, int R, float* out,
                             cudaStream_t st) {
  if (R > 32 || Ia < 1 || Ib < 32) return cudaErrorInvalidValue;
  const int64_t blocks = (Ia + 8 / kPartWarps - 1) / (8 / kPartWarps);
  if (blocks > 0x7FFFFFFF) return cudaErrorInvalidValue;
  prefer_shared_carveout<k_post_part>();
  k_post_part<<<static_cast<unsigned>(blocks), 256, 0, st>>>(part, Ia, Ib, R, out);
  return cudaGetLastError();
}

int post_slow4_splits(int64_t Ia, int64_t Ib, int R, int num_sms) {
  // As many splits of the reduced range as keep every CTA resident at once: a second,
  // partial wave of CTAs would take as long as the first (at 1000 x 1000, R = 32: 320 CTAs
  // at 2 per SM were 1.05 waves and took twice the time of 288).
  const int64_t bblocks = post_slow4_blocks(Ib, R);
  int per_sm = 0;
  const cudaError_t oe =
      R % 4 == 0 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_post_slow4,
                                                                 kPostBB * (R / 4), 0)
                 : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_post_slowv<float2>,
                                                                 kPostBB2 * (R / 2), 0);
  if (oe != cudaSuccess || per_sm < 1) {
    (void)cudaGetLastError();
    per_sm = 1;
  }
  int64_t splits = static_cast<int64_t>(per_sm) * num_sms / bblocks;
  splits = std::max<int64_t>(1, std::min<int64_t>(splits, std::max<int64_t>(1, Ia / 16)));
  return static_cast<int>(std::min<int64_t>(splits, 64));
}

int64_t post_slow4_blocks(int64_t Ib, int R) { return (Ib + post_bb(R) - 1) / post_bb(R); }

cudaError_t launch_post_slow4(const float* T, int64_t Ia, int64_t Ib, int R, const float* F,
                              int splits, float* partial, unsigned* count, float* out,
                              cudaStream_t st) {
  dim3 grid(static_cast<unsigned>(post_slow4_blocks(Ib, R)), static_cast<unsigned>(splits));
  if (post_vec4(R)) {
    const int Q = R / 4;
    prefer_shared_carveout<k_post_slow4>();
    k_post_slow4<<<grid, kPostBB * Q, 0, st>>>(
        reinterpret_cast<const float4*>(T), Ia, Ib, Q, reinterpret_cast<const float4*>(F),
        splits, reinterpret_cast<float4*>(partial), count, reinterpret_cast<float4*>(out));
  } else {
    const int Q = R / 2;
    prefer_shared_carveout<k_post_slowv<float2>>();
    k_post_slowv<float2><<<grid, kPostBB2 * Q, 0, st>>>(
        reinterpret_cast<const float2*>(T), Ia, Ib, Q, reinterpret_cast<const float2*>(F),
        splits, reinterpret_cast<float2*>(partial), count, reinterpret_cast<float2*>(out));
  }
  return cudaGetLastError();
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
