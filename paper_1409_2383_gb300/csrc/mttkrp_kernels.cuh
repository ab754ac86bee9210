// Templated MTTKRP contraction kernels (the method is described in mttkrp.cu).  Included by
// the per-type instantiation units gemm_{n,t}_{f32,bf16}.cu so that the unrolled variants
// compile in parallel.
//
// Both kernels stream one tile of the matricized tensor X[P, Q] per CTA.  The 4 warps of a
// CTA split the contraction range of the tile; each warp runs its own 2-stage ring of 16-byte
// cp.async copies -- the tensor slab and the matching rows of the Khatri-Rao operand W (a
// precomputed, zero-padded [K_pad, RP] table) -- and synchronises only itself (no CTA barrier
// until the end); W rows are read as shared-memory broadcasts.  The 4 warp partial sums are
// added in a fixed order through shared memory at the end.
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

// Storage element traits: elements per 16-byte chunk and their FP32 values.
template <typename T>
struct Elem;
template <>
struct Elem<float> {
  static constexpr int kPer16 = 4;
  __device__ static __forceinline__ void unpack16(const uint4& v, float* f) {
    f[0] = __uint_as_float(v.x); f[1] = __uint_as_float(v.y);
    f[2] = __uint_as_float(v.z); f[3] = __uint_as_float(v.w);
  }
  __device__ static __forceinline__ void load2(const char* p, float* f) {
    const float2 v = *reinterpret_cast<const float2*>(p);
    f[0] = v.x; f[1] = v.y;
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
  __device__ static __forceinline__ void load2(const char* p, float* f) {
    const uint32_t v = *reinterpret_cast<const uint32_t*>(p);
    f[0] = __uint_as_float(v << 16); f[1] = __uint_as_float(v & 0xffff0000u);
  }
  __device__ static __forceinline__ float load1(const __nv_bfloat16* p) {
    return __bfloat162float(*p);
  }
};

// Padded rank of the register tiles (a multiple of 4; coarser steps above 24 keep the number
// of compiled variants small).
inline int round_rp(int R) {
  return R <= 24 ? ((R + 3) / 4) * 4 : R <= 32 ? 32 : R <= 48 ? ((R + 7) / 8) * 8 : R <= 52 ? 52 : 64;
}

constexpr int kWarps = 4;          // warps per CTA, splitting the contraction range of a tile
constexpr int kStages = 2;         // per-warp cp.async ring depth
constexpr int kTileRows = 64;      // GEMM-N rows per CTA (2 per lane)
constexpr int kTileCols = 64;      // GEMM-T columns per CTA (2 per lane)

// acc[r4*2 .. r4*2+1] += x * (w.x, w.y, w.z, w.w) as two packed FP32x2 FMAs (each lane of a
// packed FMA is an ordinary IEEE fused multiply-add: the same results as four fmaf, half the
// instructions).  xx = (x, x).
__device__ __forceinline__ void fma4(float2* acc, int r4, float2 xx, const float4& w) {
  acc[r4 * 2 + 0] = __ffma2_rn(xx, make_float2(w.x, w.y), acc[r4 * 2 + 0]);
  acc[r4 * 2 + 1] = __ffma2_rn(xx, make_float2(w.z, w.w), acc[r4 * 2 + 1]);
}

// Adds the (2 x RP) accumulators of the 4 warps in the fixed order (w0 + w2) + (w1 + w3); the
// sum ends in warp 0.  buf: 2 * 64 * (RP + 1) floats (padded rows: conflict-free).
template <int RP>
__device__ __forceinline__ void reduce_warps(float2 (&acc)[2][RP / 2], float* buf, int warp,
                                             int lane) {
  constexpr int LD = RP + 1;
  constexpr int H = RP / 2;
  __syncthreads();  // every warp has finished with its ring; buf may alias it
  if (warp >= 2) {
    float* b = buf + (warp - 2) * 64 * LD;
#pragma unroll
    for (int g = 0; g < 2; ++g)
#pragma unroll
      for (int r = 0; r < H; ++r) {
        b[(g * 32 + lane) * LD + 2 * r] = acc[g][r].x;
        b[(g * 32 + lane) * LD + 2 * r + 1] = acc[g][r].y;
      }
  }
  __syncthreads();
  if (warp < 2) {
    const float* b = buf + warp * 64 * LD;
#pragma unroll
    for (int g = 0; g < 2; ++g)
#pragma unroll
      for (int r = 0; r < H; ++r) {
        acc[g][r].x += b[(g * 32 + lane) * LD + 2 * r];
        acc[g][r].y += b[(g * 32 + lane) * LD + 2 * r + 1];
      }
  }
  __syncthreads();
  if (warp == 1) {
#pragma unroll
    for (int g = 0; g < 2; ++g)
#pragma unroll
      for (int r = 0; r < H; ++r) {
        buf[(g * 32 + lane) * LD + 2 * r] = acc[g][r].x;
        buf[(g * 32 + lane) * LD + 2 * r + 1] = acc[g][r].y;
      }
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int g = 0; g < 2; ++g)
#pragma unroll
      for (int r = 0; r < H; ++r) {
        acc[g][r].x += buf[(g * 32 + lane) * LD + 2 * r];
        acc[g][r].y += buf[(g * 32 + lane) * LD + 2 * r + 1];
      }
  }
}

// Writes acc (2 x RP, padded) as R floats per output row.
template <int RP>
__device__ __forceinline__ void store_row(float* dst, const float2 (&a)[RP / 2], int R) {
#pragma unroll
  for (int r = 0; r < RP / 2; ++r) {
    if (2 * r < R) dst[2 * r] = a[r].x;
    if (2 * r + 1 < R) dst[2 * r + 1] = a[r].y;
  }
}

// ------------------------------------------------------------------------- GEMM-N
// out[p, r] = sum_{q in chunk} X[p, q] W[q, r] for the 64 rows of blockIdx.x and the column
// chunk blockIdx.y.  Lane l of every warp owns rows l and l + 32; warp w streams the w-th
// quarter of the chunk, 64 bytes of each row per stage (80-byte smem pitch: the 16-byte reads
// of 8 consecutive rows fall in distinct bank groups).
template <typename T, int RP>
struct GN2 {
  static constexpr int kE = Elem<T>::kPer16;
  static constexpr int kCh = 4;                  // 16-byte chunks per row per stage
  static constexpr int kTQ = kCh * kE;           // columns per stage
  static constexpr int kPitch = kCh * 16 + 16;
  static constexpr int kXBytes = kTileRows * kPitch;
  static constexpr int kWBytes = kTQ * RP * 4;   // W rows of the stage
  static constexpr int kStageBytes = kXBytes + kWBytes;
  static constexpr int kRingBytes = kWarps * kStages * kStageBytes;
};

template <typename T, int RP>
__global__ void __launch_bounds__(kWarps * 32)
    k_gemm_n2(const T* __restrict__ X, int64_t P, int64_t Q, int R, const float* __restrict__ W,
              int64_t chunk, float* __restrict__ out) {
  using C = GN2<T, RP>;
  extern __shared__ __align__(16) char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t row0 = static_cast<int64_t>(blockIdx.x) * kTileRows;
  const int nrows = static_cast<int>(P - row0 < kTileRows ? P - row0 : kTileRows);
  const int64_t c0 = static_cast<int64_t>(blockIdx.y) * chunk;
  const int64_t c1 = Q < c0 + chunk ? Q : c0 + chunk;
  const int64_t nst_all = (c1 - c0 + C::kTQ - 1) / C::kTQ;
  const int64_t s_beg = nst_all * warp / kWarps;
  const int nst = static_cast<int>(nst_all * (warp + 1) / kWarps - s_beg);
  char* ring = smem + warp * kStages * C::kStageBytes;

  auto issue = [&](int i, int slot) {
    char* dst = ring + slot * C::kStageBytes;
    const int64_t q0 = c0 + (s_beg + i) * C::kTQ;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int r = (lane >> 2) + 8 * k, c = lane & 3;
      const int64_t qc = q0 + c * C::kE;
      const bool valid = r < nrows && qc < c1;
      cp_async16(dst + r * C::kPitch + c * 16, valid ? X + (row0 + r) * Q + qc : X, valid);
    }
    // W rows q0 .. q0 + kTQ (inside the padded table)
    const char* wsrc = reinterpret_cast<const char*>(W + q0 * RP);
    for (int k = lane; k < C::kWBytes / 16; k += 32)
      cp_async16(dst + C::kXBytes + k * 16, wsrc + k * 16, true);
  };

  float2 acc[2][RP / 2];
#pragma unroll
  for (int g = 0; g < 2; ++g)
#pragma unroll
    for (int r = 0; r < RP / 2; ++r) acc[g][r] = make_float2(0.0f, 0.0f);

#pragma unroll
  for (int s = 0; s < kStages - 1; ++s) {
    if (s < nst) issue(s, s);
    cp_async_commit();
  }
  for (int i = 0; i < nst; ++i) {
    cp_async_wait<kStages - 2>();
    __syncwarp();
    const int nx = i + kStages - 1;
    if (nx < nst) issue(nx, nx % kStages);
    cp_async_commit();
    const char* xs = ring + (i % kStages) * C::kStageBytes;
    const float* wq = reinterpret_cast<const float*>(xs + C::kXBytes);
#pragma unroll
    for (int c = 0; c < C::kCh; ++c) {
      float x0[C::kE], x1[C::kE];
      Elem<T>::unpack16(*reinterpret_cast<const uint4*>(xs + lane * C::kPitch + c * 16), x0);
      Elem<T>::unpack16(*reinterpret_cast<const uint4*>(xs + (lane + 32) * C::kPitch + c * 16), x1);
#pragma unroll
      for (int e = 0; e < C::kE; ++e) {
        const float4* wr = reinterpret_cast<const float4*>(wq + (c * C::kE + e) * RP);
        const float2 xa = make_float2(x0[e], x0[e]), xb = make_float2(x1[e], x1[e]);
#pragma unroll
        for (int r4 = 0; r4 < RP / 4; ++r4) {
          const float4 w = wr[r4];
          fma4(acc[0], r4, xa, w);
          fma4(acc[1], r4, xb, w);
        }
      }
    }
  }
  cp_async_wait<0>();
  reduce_warps<RP>(acc, reinterpret_cast<float*>(smem), warp, lane);
  if (warp == 0) {
    float* o = out + static_cast<int64_t>(blockIdx.y) * P * R;
#pragma unroll
    for (int g = 0; g < 2; ++g) {
      const int lr = g * 32 + lane;
      if (lr < nrows) store_row<RP>(o + (row0 + lr) * R, acc[g], R);
    }
  }
}

// ------------------------------------------------------------------------- GEMM-T
// out[q, r] = sum_{p in chunk} X[p, q] W[p, r] for the 64 columns of blockIdx.x and the row
// chunk blockIdx.y.  Lane l owns columns 2l, 2l + 1; warp w streams the w-th quarter of the
// chunk, whole 64-column row segments (consecutive lanes read consecutive addresses).
template <typename T, int RP>
struct GT2 {
  static constexpr int kE = Elem<T>::kPer16;
  static constexpr int kRowBytes = kTileCols * static_cast<int>(sizeof(T));  // 256 / 128
  static constexpr int kChunksPerRow = kRowBytes / 16;
  static constexpr int kTP = 4096 / kRowBytes;                                // rows per stage
  static constexpr int kXBytes = kTP * kRowBytes;
  static constexpr int kWBytes = kTP * RP * 4;                                // W rows
  static constexpr int kStageBytes = kXBytes + kWBytes;
  static constexpr int kRingBytes = kWarps * kStages * kStageBytes;
};

template <typename T, int RP>
__global__ void __launch_bounds__(kWarps * 32)
    k_gemm_t2(const T* __restrict__ X, int64_t P, int64_t Q, int R, const float* __restrict__ W,
              int64_t chunk, float* __restrict__ out) {
  using C = GT2<T, RP>;
  extern __shared__ __align__(16) char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t q0 = static_cast<int64_t>(blockIdx.x) * kTileCols;
  const int ncols = static_cast<int>(Q - q0 < kTileCols ? Q - q0 : kTileCols);
  const int64_t p0 = static_cast<int64_t>(blockIdx.y) * chunk;
  const int64_t p1 = P < p0 + chunk ? P : p0 + chunk;
  const int64_t nst_all = (p1 - p0 + C::kTP - 1) / C::kTP;
  const int64_t s_beg = nst_all * warp / kWarps;
  const int nst = static_cast<int>(nst_all * (warp + 1) / kWarps - s_beg);
  char* ring = smem + warp * kStages * C::kStageBytes;

  auto issue = [&](int i, int slot) {
    char* dst = ring + slot * C::kStageBytes;
    const int64_t pr0 = p0 + (s_beg + i) * C::kTP;
    constexpr int kCopies = C::kTP * C::kChunksPerRow / 32;  // 8
#pragma unroll
    for (int k = 0; k < kCopies; ++k) {
      const int idx = lane + 32 * k;
      const int rr = idx / C::kChunksPerRow, c = idx % C::kChunksPerRow;
      const int64_t p = pr0 + rr, col = q0 + c * C::kE;
      const bool valid = p < p1 && col < Q;
      cp_async16(dst + rr * C::kRowBytes + c * 16, valid ? X + p * Q + col : X, valid);
    }
    const char* wsrc = reinterpret_cast<const char*>(W + pr0 * RP);
    for (int k = lane; k < C::kWBytes / 16; k += 32)
      cp_async16(dst + C::kXBytes + k * 16, wsrc + k * 16, true);
  };

  float2 acc[2][RP / 2];
#pragma unroll
  for (int g = 0; g < 2; ++g)
#pragma unroll
    for (int r = 0; r < RP / 2; ++r) acc[g][r] = make_float2(0.0f, 0.0f);

#pragma unroll
  for (int s = 0; s < kStages - 1; ++s) {
    if (s < nst) issue(s, s);
    cp_async_commit();
  }
  for (int i = 0; i < nst; ++i) {
    cp_async_wait<kStages - 2>();
    __syncwarp();
    const int nx = i + kStages - 1;
    if (nx < nst) issue(nx, nx % kStages);
    cp_async_commit();
    const char* xs = ring + (i % kStages) * C::kStageBytes;
    const float* wp = reinterpret_cast<const float*>(xs + C::kXBytes);
#pragma unroll 4
    for (int rr = 0; rr < C::kTP; ++rr) {
      float xv[2];
      Elem<T>::load2(xs + rr * C::kRowBytes + lane * 2 * static_cast<int>(sizeof(T)), xv);
      const float4* wr = reinterpret_cast<const float4*>(wp + rr * RP);
      const float2 xa = make_float2(xv[0], xv[0]), xb = make_float2(xv[1], xv[1]);
#pragma unroll
      for (int r4 = 0; r4 < RP / 4; ++r4) {
        const float4 w = wr[r4];
        fma4(acc[0], r4, xa, w);
        fma4(acc[1], r4, xb, w);
      }
    }
  }
  cp_async_wait<0>();
  reduce_warps<RP>(acc, reinterpret_cast<float*>(smem), warp, lane);
  if (warp == 0) {
    float* o = out + static_cast<int64_t>(blockIdx.y) * Q * R;
#pragma unroll
    for (int g = 0; g < 2; ++g) {
      const int lc = lane * 2 + g;
      if (lc < ncols) store_row<RP>(o + (q0 + lc) * R, acc[g], R);
    }
  }
}

// ------------------------------------------------------------- unaligned fallbacks
// Plain-load versions for shapes whose rows are not 16-byte aligned (odd extents): one thread
// per output entry, whole contraction, no staging.  Correct for any shape; used only when the
// fast path's alignment preconditions fail.
template <typename T>
__global__ void k_gemm_n_plain(const T* __restrict__ X, int64_t P, int64_t Q, int R,
                               const float* __restrict__ W, int RP, float* __restrict__ out) {
  for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < P * R;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t p = idx / R;
    const int r = static_cast<int>(idx % R);
    float acc = 0.0f;
    for (int64_t q = 0; q < Q; ++q) acc = fmaf(Elem<T>::load1(X + p * Q + q), W[q * RP + r], acc);
    out[idx] = acc;
  }
}

template <typename T>
__global__ void k_gemm_t_plain(const T* __restrict__ X, int64_t P, int64_t Q, int R,
                               const float* __restrict__ W, int RP, float* __restrict__ out) {
  for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < Q * R;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t q = idx / R;
    const int r = static_cast<int>(idx % R);
    float acc = 0.0f;
    for (int64_t p = 0; p < P; ++p) acc = fmaf(Elem<T>::load1(X + p * Q + q), W[p * RP + r], acc);
    out[idx] = acc;
  }
}

// ------------------------------------------------------------------ dispatch helpers
template <int RP>
constexpr int reduce_bytes() { return 2 * 64 * (RP + 1) * 4; }

template <typename T, int RP>
cudaError_t run_gemm_n2(const T* X, int64_t P, int64_t Q, int R, const float* W,
                        const GemmPlan& plan, float* out, cudaStream_t st) {
  constexpr int smem = GN2<T, RP>::kRingBytes > reduce_bytes<RP>() ? GN2<T, RP>::kRingBytes
                                                                   : reduce_bytes<RP>();
  auto kern = k_gemm_n2<T, RP>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  dim3 grid(plan.tiles, plan.chunks);
  kern<<<grid, kWarps * 32, smem, st>>>(X, P, Q, R, W, plan.chunk_len, out);
  return cudaGetLastError();
}

template <typename T, int RP>
cudaError_t run_gemm_t2(const T* X, int64_t P, int64_t Q, int R, const float* W,
                        const GemmPlan& plan, float* out, cudaStream_t st) {
  constexpr int smem = GT2<T, RP>::kRingBytes > reduce_bytes<RP>() ? GT2<T, RP>::kRingBytes
                                                                   : reduce_bytes<RP>();
  auto kern = k_gemm_t2<T, RP>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  dim3 grid(plan.tiles, plan.chunks);
  kern<<<grid, kWarps * 32, smem, st>>>(X, P, Q, R, W, plan.chunk_len, out);
  return cudaGetLastError();
}

#define NTF_RP_CASES(M) M(4) M(8) M(12) M(16) M(20) M(24) M(32) M(40) M(48) M(52) M(64)

template <typename T>
cudaError_t gemm_n_typed(const T* X, int64_t P, int64_t Q, int R, const float* W,
                         const GemmPlan& plan, float* out, cudaStream_t st) {
  const int rp = round_rp(R);
  if (!plan.vec16) {
    const unsigned g = static_cast<unsigned>(std::min<int64_t>((P * R + 255) / 256, 8192));
    k_gemm_n_plain<T><<<g, 256, 0, st>>>(X, P, Q, R, W, rp, out);
    return cudaGetLastError();
  }
  switch (rp) {
#define NTF_CASE(V) \
  case V:           \
    return run_gemm_n2<T, V>(X, P, Q, R, W, plan, out, st);
    NTF_RP_CASES(NTF_CASE)
#undef NTF_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t gemm_t_typed(const T* X, int64_t P, int64_t Q, int R, const float* W,
                         const GemmPlan& plan, float* out, cudaStream_t st) {
  const int rp = round_rp(R);
  if (!plan.vec16) {
    const unsigned g = static_cast<unsigned>(std::min<int64_t>((Q * R + 255) / 256, 8192));
    k_gemm_t_plain<T><<<g, 256, 0, st>>>(X, P, Q, R, W, rp, out);
    return cudaGetLastError();
  }
  switch (rp) {
#define NTF_CASE(V) \
  case V:           \
    return run_gemm_t2<T, V>(X, P, Q, R, W, plan, out, st);
    NTF_RP_CASES(NTF_CASE)
#undef NTF_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace detail
}  // namespace ntf
