// Templated MTTKRP contraction kernels (see mttkrp.cu for the method).  Included by the
// per-type instantiation units gemm_{n,t}_{f32,bf16}.cu so that the unrolled variants
// compile in parallel.
#pragma once
#include <algorithm>

#include "ntf_internal.cuh"

namespace ntf {
namespace detail {


__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
  const int n = valid ? 16 : 0;  // n == 0: nothing is read, 16 zero bytes are written
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_addr(dst)),
               "l"(src), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

// Storage element traits: how many elements one 16-byte chunk holds and their FP32 values.
template <typename T>
struct Elem;
template <>
struct Elem<float> {
  static constexpr int kPer16 = 4;
  __device__ static __forceinline__ void unpack16(const uint4& v, float* f) {
    f[0] = __uint_as_float(v.x); f[1] = __uint_as_float(v.y);
    f[2] = __uint_as_float(v.z); f[3] = __uint_as_float(v.w);
  }
  __device__ static __forceinline__ float load1(const float* p) { return __ldg(p); }
};
template <>
struct Elem<__nv_bfloat16> {
  static constexpr int kPer16 = 8;
  // bf16 -> f32 is exact: the 16 stored bits become the high half of the float.
  __device__ static __forceinline__ void unpack16(const uint4& v, float* f) {
    f[0] = __uint_as_float(v.x << 16); f[1] = __uint_as_float(v.x & 0xffff0000u);
    f[2] = __uint_as_float(v.y << 16); f[3] = __uint_as_float(v.y & 0xffff0000u);
    f[4] = __uint_as_float(v.z << 16); f[5] = __uint_as_float(v.z & 0xffff0000u);
    f[6] = __uint_as_float(v.w << 16); f[7] = __uint_as_float(v.w & 0xffff0000u);
  }
  __device__ static __forceinline__ float load1(const __nv_bfloat16* p) {
    return __bfloat162float(*p);
  }
};

// Entry r of Khatri-Rao row q of a group (last mode fastest).  r >= R gives 0.
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

// ------------------------------------------------------------------------- GEMM-N
// CTA: WARPS warps; warp w owns 32-row groups w, w+WARPS, ... (up to GROUPS of them) of a
// row block; each thread accumulates all RP columns of its rows.  Per stage the CTA stages a
// [rows x 32 bytes] slab of X (48-byte smem pitch: conflict-free 16-byte reads by 8
// consecutive rows) and the matching [TQ x RP] Khatri-Rao tile.
template <typename T, int RP, int WARPS, int GROUPS>
struct GN {
  static constexpr int kThreads = WARPS * 32;
  static constexpr int kRows = WARPS * GROUPS * 32;
  static constexpr int kChunks = 2;
  static constexpr int kTQ = kChunks * Elem<T>::kPer16;
  static constexpr int kPitch = 48;
  static constexpr int kStages = 4;
  static constexpr int kXBytes = kRows * kPitch;
  static constexpr int kWFloats = kTQ * RP;
  static constexpr int kStageBytes = kXBytes + kWFloats * 4;
  static constexpr int kSmem = kStages * kStageBytes;
};

template <typename T, int RP, int WARPS, int GROUPS, int NG>
__device__ __forceinline__ void gn_compute(const char* xs, const float* ws, int warp, int lane,
                                           float (&acc)[GROUPS][RP]) {
  using C = GN<T, RP, WARPS, GROUPS>;
  constexpr int E = Elem<T>::kPer16;
#pragma unroll
  for (int c = 0; c < C::kChunks; ++c) {
    float xv[NG][E];
#pragma unroll
    for (int g = 0; g < NG; ++g) {
      const int lr = (warp + g * WARPS) * 32 + lane;
      const uint4 v = *reinterpret_cast<const uint4*>(xs + lr * C::kPitch + c * 16);
      Elem<T>::unpack16(v, xv[g]);
    }
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const float* wr = ws + (c * E + e) * RP;
#pragma unroll
      for (int r4 = 0; r4 < RP / 4; ++r4) {
        const float4 w = *reinterpret_cast<const float4*>(wr + r4 * 4);
#pragma unroll
        for (int g = 0; g < NG; ++g) {
          acc[g][r4 * 4 + 0] = fmaf(xv[g][e], w.x, acc[g][r4 * 4 + 0]);
          acc[g][r4 * 4 + 1] = fmaf(xv[g][e], w.y, acc[g][r4 * 4 + 1]);
          acc[g][r4 * 4 + 2] = fmaf(xv[g][e], w.z, acc[g][r4 * 4 + 2]);
          acc[g][r4 * 4 + 3] = fmaf(xv[g][e], w.w, acc[g][r4 * 4 + 3]);
        }
      }
    }
  }
}

template <typename T, int RP, int WARPS, int GROUPS>
__global__ void __launch_bounds__(WARPS * 32)
    k_gemm_n(const T* __restrict__ X, int64_t P, int64_t Q, int R, Group g, int rows_per_blk,
             int splits, float* __restrict__ out) {
  using C = GN<T, RP, WARPS, GROUPS>;
  extern __shared__ __align__(16) char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int split = blockIdx.x;
  const int64_t row0 = static_cast<int64_t>(blockIdx.y) * rows_per_blk;
  const int nrows = static_cast<int>((P - row0 < rows_per_blk ? P - row0 : (int64_t)rows_per_blk));
  const int64_t ntile_all = (Q + C::kTQ - 1) / C::kTQ;
  const int64_t t0 = ntile_all * split / splits, t1 = ntile_all * (split + 1) / splits;
  const int ntile = static_cast<int>(t1 - t0);

  // warp-uniform number of row groups this warp owns
  int ng = 0;
#pragma unroll
  for (int gi = 0; gi < GROUPS; ++gi) ng += ((warp + gi * WARPS) * 32 < nrows) ? 1 : 0;

  float acc[GROUPS][RP];
#pragma unroll
  for (int a = 0; a < GROUPS; ++a)
#pragma unroll
    for (int r = 0; r < RP; ++r) acc[a][r] = 0.0f;

  auto load = [&](int it, int slot) {
    char* xs = smem + slot * C::kStageBytes;
    float* ws = reinterpret_cast<float*>(xs + C::kXBytes);
    const int64_t q0 = (t0 + it) * C::kTQ;
    for (int i = tid; i < nrows * C::kChunks; i += C::kThreads) {
      const int row = i / C::kChunks, c = i % C::kChunks;
      const int64_t qc = q0 + c * Elem<T>::kPer16;
      const bool valid = qc < Q;
      const T* src = valid ? X + (row0 + row) * Q + qc : X;
      cp_async16(xs + row * C::kPitch + c * 16, src, valid);
    }
    for (int i = tid; i < C::kWFloats; i += C::kThreads) {
      const int q = i / RP, r = i % RP;
      const int64_t qq = q0 + q;
      ws[i] = (r < R && qq < Q) ? kr_entry(g, qq, r, R) : 0.0f;
    }
  };

#pragma unroll
  for (int s = 0; s < C::kStages - 1; ++s) {
    if (s < ntile) load(s, s);
    cp_async_commit();
  }
  for (int it = 0; it < ntile; ++it) {
    cp_async_wait<C::kStages - 2>();
    __syncthreads();
    const int nx = it + C::kStages - 1;
    if (nx < ntile) load(nx, nx % C::kStages);
    cp_async_commit();
    const int slot = it % C::kStages;
    const char* xs = smem + slot * C::kStageBytes;
    const float* ws = reinterpret_cast<const float*>(xs + C::kXBytes);
    if (ng == GROUPS) {
      gn_compute<T, RP, WARPS, GROUPS, GROUPS>(xs, ws, warp, lane, acc);
    } else if (GROUPS > 1 && ng >= 1) {
      if constexpr (GROUPS == 4) {
        if (ng == 3) gn_compute<T, RP, WARPS, GROUPS, 3>(xs, ws, warp, lane, acc);
        else if (ng == 2) gn_compute<T, RP, WARPS, GROUPS, 2>(xs, ws, warp, lane, acc);
        else gn_compute<T, RP, WARPS, GROUPS, 1>(xs, ws, warp, lane, acc);
      } else if constexpr (GROUPS == 2) {
        gn_compute<T, RP, WARPS, GROUPS, 1>(xs, ws, warp, lane, acc);
      }
    }
  }
  cp_async_wait<0>();

  float* o = out + static_cast<int64_t>(split) * P * R;
#pragma unroll
  for (int gi = 0; gi < GROUPS; ++gi) {
    const int lr = (warp + gi * WARPS) * 32 + lane;
    if (gi < ng && lr < nrows) {
      float* dst = o + (row0 + lr) * R;
#pragma unroll
      for (int r = 0; r < RP; ++r)
        if (r < R) dst[r] = acc[gi][r];
    }
  }
}

// ------------------------------------------------------------------------- GEMM-T
// CTA: 128 threads; thread t owns CPT consecutive columns; the CTA's column block is
// 128*CPT wide.  Per stage: TP rows of the block (contiguous row segments) and the matching
// [TP x RP] Khatri-Rao tile; the contraction runs over the rows.
template <typename T, int RP>
struct GT {
  static constexpr int kThreads = 128;
  static constexpr int kCPT = RP <= 32 ? 4 : 2;
  static constexpr int kCols = kThreads * kCPT;
  static constexpr int kRowBytes = kCols * static_cast<int>(sizeof(T));
  static constexpr int kTP = 8192 / kRowBytes;  // 8 KB of X per stage
  static constexpr int kStages = 6;
  static constexpr int kXBytes = kTP * kRowBytes;
  static constexpr int kWFloats = kTP * RP;
  static constexpr int kStageBytes = kXBytes + kWFloats * 4;
  static constexpr int kSmem = kStages * kStageBytes;
};

template <int CPT, typename T>
__device__ __forceinline__ void gt_load_cols(const char* p, float* f);
template <>
__device__ __forceinline__ void gt_load_cols<4, float>(const char* p, float* f) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  f[0] = v.x; f[1] = v.y; f[2] = v.z; f[3] = v.w;
}
template <>
__device__ __forceinline__ void gt_load_cols<2, float>(const char* p, float* f) {
  const float2 v = *reinterpret_cast<const float2*>(p);
  f[0] = v.x; f[1] = v.y;
}
template <>
__device__ __forceinline__ void gt_load_cols<4, __nv_bfloat16>(const char* p, float* f) {
  const uint2 v = *reinterpret_cast<const uint2*>(p);
  f[0] = __uint_as_float(v.x << 16); f[1] = __uint_as_float(v.x & 0xffff0000u);
  f[2] = __uint_as_float(v.y << 16); f[3] = __uint_as_float(v.y & 0xffff0000u);
}
template <>
__device__ __forceinline__ void gt_load_cols<2, __nv_bfloat16>(const char* p, float* f) {
  const uint32_t v = *reinterpret_cast<const uint32_t*>(p);
  f[0] = __uint_as_float(v << 16); f[1] = __uint_as_float(v & 0xffff0000u);
}

template <typename T, int RP>
__global__ void __launch_bounds__(128)
    k_gemm_t(const T* __restrict__ X, int64_t P, int64_t Q, int R, Group g, int splits,
             float* __restrict__ out) {
  using C = GT<T, RP>;
  constexpr int CPT = C::kCPT;
  extern __shared__ __align__(16) char smem[];
  const int tid = threadIdx.x;
  const int split = blockIdx.x;
  const int64_t c0 = static_cast<int64_t>(blockIdx.y) * C::kCols;
  const int ncols = static_cast<int>((Q - c0 < C::kCols ? Q - c0 : (int64_t)C::kCols));
  const int64_t p_beg = P * split / splits, p_end = P * (split + 1) / splits;
  const int ntile = static_cast<int>((p_end - p_beg + C::kTP - 1) / C::kTP);
  const bool active = (tid & ~31) * CPT < ncols;  // warp-uniform

  float acc[CPT][RP];
#pragma unroll
  for (int a = 0; a < CPT; ++a)
#pragma unroll
    for (int r = 0; r < RP; ++r) acc[a][r] = 0.0f;

  constexpr int kChunksPerRow = C::kRowBytes / 16;
  auto load = [&](int it, int slot) {
    char* xs = smem + slot * C::kStageBytes;
    float* ws = reinterpret_cast<float*>(xs + C::kXBytes);
    const int64_t p0 = p_beg + static_cast<int64_t>(it) * C::kTP;
    for (int i = tid; i < C::kTP * kChunksPerRow; i += C::kThreads) {
      const int pr = i / kChunksPerRow, c = i % kChunksPerRow;
      const int64_t col = c0 + c * Elem<T>::kPer16;
      const bool valid = (p0 + pr < p_end) && (col < Q);
      const T* src = valid ? X + (p0 + pr) * Q + col : X;
      cp_async16(xs + pr * C::kRowBytes + c * 16, src, valid);
    }
    for (int i = tid; i < C::kWFloats; i += C::kThreads) {
      const int pr = i / RP, r = i % RP;
      const int64_t pp = p0 + pr;
      ws[i] = (r < R && pp < p_end) ? kr_entry(g, pp, r, R) : 0.0f;
    }
  };

#pragma unroll
  for (int s = 0; s < C::kStages - 1; ++s) {
    if (s < ntile) load(s, s);
    cp_async_commit();
  }
  for (int it = 0; it < ntile; ++it) {
    cp_async_wait<C::kStages - 2>();
    __syncthreads();
    const int nx = it + C::kStages - 1;
    if (nx < ntile) load(nx, nx % C::kStages);
    cp_async_commit();
    if (active) {
      const int slot = it % C::kStages;
      const char* xs = smem + slot * C::kStageBytes;
      const float* ws = reinterpret_cast<const float*>(xs + C::kXBytes);
#pragma unroll
      for (int pr = 0; pr < C::kTP; ++pr) {
        float xv[CPT];
        gt_load_cols<CPT, T>(xs + pr * C::kRowBytes + tid * CPT * sizeof(T), xv);
        const float* wr = ws + pr * RP;
#pragma unroll
        for (int r4 = 0; r4 < RP / 4; ++r4) {
          const float4 w = *reinterpret_cast<const float4*>(wr + r4 * 4);
#pragma unroll
          for (int c = 0; c < CPT; ++c) {
            acc[c][r4 * 4 + 0] = fmaf(xv[c], w.x, acc[c][r4 * 4 + 0]);
            acc[c][r4 * 4 + 1] = fmaf(xv[c], w.y, acc[c][r4 * 4 + 1]);
            acc[c][r4 * 4 + 2] = fmaf(xv[c], w.z, acc[c][r4 * 4 + 2]);
            acc[c][r4 * 4 + 3] = fmaf(xv[c], w.w, acc[c][r4 * 4 + 3]);
          }
        }
      }
    }
  }
  cp_async_wait<0>();

  float* o = out + static_cast<int64_t>(split) * Q * R;
#pragma unroll
  for (int c = 0; c < CPT; ++c) {
    const int lc = tid * CPT + c;
    if (lc < ncols) {
      float* dst = o + (c0 + lc) * R;
#pragma unroll
      for (int r = 0; r < RP; ++r)
        if (r < R) dst[r] = acc[c][r];
    }
  }
}

// ------------------------------------------------------------- unaligned fallbacks
// Plain-load versions for shapes whose rows are not 16-byte aligned (odd extents): one
// thread per output entry block, no staging.  Correct for any shape; used only when the
// fast path's alignment preconditions fail.
template <typename T>
__global__ void k_gemm_n_plain(const T* __restrict__ X, int64_t P, int64_t Q, int R, Group g,
                               int splits, float* __restrict__ out) {
  const int split = blockIdx.y;
  const int64_t q_beg = Q * split / splits, q_end = Q * (split + 1) / splits;
  for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < P * R;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t p = idx / R;
    const int r = static_cast<int>(idx % R);
    float acc = 0.0f;
    for (int64_t q = q_beg; q < q_end; ++q)
      acc = fmaf(Elem<T>::load1(X + p * Q + q), kr_entry(g, q, r, R), acc);
    out[split * P * R + idx] = acc;
  }
}

template <typename T>
__global__ void k_gemm_t_plain(const T* __restrict__ X, int64_t P, int64_t Q, int R, Group g,
                               int splits, float* __restrict__ out) {
  const int split = blockIdx.y;
  const int64_t p_beg = P * split / splits, p_end = P * (split + 1) / splits;
  for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < Q * R;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t q = idx / R;
    const int r = static_cast<int>(idx % R);
    float acc = 0.0f;
    for (int64_t p = p_beg; p < p_end; ++p)
      acc = fmaf(Elem<T>::load1(X + p * Q + q), kr_entry(g, p, r, R), acc);
    out[split * Q * R + idx] = acc;
  }
}

// ------------------------------------------------------------------ dispatch helpers
// Padded rank for the register tiles (a multiple of 4; coarser steps above 24 keep the
// number of compiled variants small).
inline int round_rp(int R) {
  return R <= 24 ? ((R + 3) / 4) * 4 : R <= 32 ? 32 : R <= 48 ? ((R + 7) / 8) * 8 : R <= 52 ? 52 : 64;
}

template <typename T, int RP, int WARPS, int GROUPS>
cudaError_t run_gemm_n(const T* X, int64_t P, int64_t Q, int R, const Group& g,
                       const GemmPlan& plan, float* out, cudaStream_t st) {
  using C = GN<T, RP, WARPS, GROUPS>;
  auto kern = k_gemm_n<T, RP, WARPS, GROUPS>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmem);
  if (e != cudaSuccess) return e;
  dim3 grid(plan.splits, plan.blocks);
  kern<<<grid, C::kThreads, C::kSmem, st>>>(X, P, Q, R, g, plan.rows_per_blk, plan.splits, out);
  return cudaGetLastError();
}

template <typename T, int RP>
cudaError_t run_gemm_t(const T* X, int64_t P, int64_t Q, int R, const Group& g,
                       const GemmPlan& plan, float* out, cudaStream_t st) {
  using C = GT<T, RP>;
  auto kern = k_gemm_t<T, RP>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmem);
  if (e != cudaSuccess) return e;
  dim3 grid(plan.splits, plan.blocks);
  kern<<<grid, C::kThreads, C::kSmem, st>>>(X, P, Q, R, g, plan.splits, out);
  return cudaGetLastError();
}

// RP dispatch: every multiple of 4 up to 64.
#define NTF_RP_CASES(M) M(4) M(8) M(12) M(16) M(20) M(24) M(32) M(40) M(48) M(52) M(64)

template <typename T, int RP>
cudaError_t gemm_n_rp(const T* X, int64_t P, int64_t Q, int R, const Group& g,
                      const GemmPlan& plan, float* out, cudaStream_t st, bool small) {
  if constexpr (RP <= 24) {
    if (small) return run_gemm_n<T, RP, 4, 4>(X, P, Q, R, g, plan, out, st);
  }
  return run_gemm_n<T, RP, 8, 2>(X, P, Q, R, g, plan, out, st);
}

template <typename T>
cudaError_t gemm_n_typed(const T* X, int64_t P, int64_t Q, int R, const Group& g,
                         const GemmPlan& plan, float* out, cudaStream_t st) {
  if (!plan.vec16) {
    dim3 grid(static_cast<unsigned>(std::min<int64_t>((P * R + 255) / 256, 4096)), plan.splits);
    k_gemm_n_plain<T><<<grid, 256, 0, st>>>(X, P, Q, R, g, plan.splits, out);
    return cudaGetLastError();
  }
  const int rp = round_rp(R);
  // Few rows and a small rank: 4 warps x 4 row groups per warp (more FMAs per shared-memory
  // load); otherwise 8 warps x 2 row groups (fits the register file up to RP = 64).
  const bool small = P <= 512 && rp <= 24;
  switch (rp) {
#define NTF_CASE(V) \
  case V:           \
    return gemm_n_rp<T, V>(X, P, Q, R, g, plan, out, st, small);
    NTF_RP_CASES(NTF_CASE)
#undef NTF_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t gemm_t_typed(const T* X, int64_t P, int64_t Q, int R, const Group& g,
                         const GemmPlan& plan, float* out, cudaStream_t st) {
  if (!plan.vec16) {
    dim3 grid(static_cast<unsigned>(std::min<int64_t>((Q * R + 255) / 256, 4096)), plan.splits);
    k_gemm_t_plain<T><<<grid, 256, 0, st>>>(X, P, Q, R, g, plan.splits, out);
    return cudaGetLastError();
  }
  switch (round_rp(R)) {
#define NTF_CASE(V) \
  case V:           \
    return run_gemm_t<T, V>(X, P, Q, R, g, plan, out, st);
    NTF_RP_CASES(NTF_CASE)
#undef NTF_CASE
    default:
      return cudaErrorInvalidValue;
  }
}


}  // namespace detail
}  // namespace ntf
