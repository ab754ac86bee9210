// MTTKRP of a sparse tensor in coordinate form (the sparse case of Sec. IV-A: with n nonzeros
// the product X^(n) (Khatri-Rao) costs 3nF flops for a 3-way tensor and never forms the
// Khatri-Rao matrix).  Entry (i_1, ..., i_N) with value v adds v prod_{m != n} F_m[i_m, :] to
// row i_n of M.
//
// Layout, built once by ntf_sptensor_create: for every mode n, the nonzeros sorted by i_n and,
// within a row, by the index of the first other mode (equal pairs keep their input order), as
// packed words (i_n, the other modes' indices, the value's bits) -- N + 1 words, one 16-byte
// load for a 3-way tensor -- plus row offsets [I_n + 1], so that an MTTKRP streams each
// nonzero once, in order, and the nonzeros of a row that share that index come together (their
// factor row is gathered once from L2, then from L1).  The sort is a
// least-significant-digit radix sort, 8 bits per pass, each pass a stable counting sort over
// tiles of 4096 nonzeros: per-tile digit histograms, their prefix over (digit, tile), and a
// scatter in which each tile ranks its nonzeros in order (warp match on the digit, then
// per-warp counts).
//
// MTTKRP: warp c takes the sorted nonzeros [128 c, 128 (c + 1)) (balanced whatever the row
// lengths); its lanes load 32 nonzeros at a time (coalesced), the warp walks them by broadcast
// with the factor-row gathers of 8 nonzeros in flight (lanes over the rank: r = lane,
// lane + 32; the factors are L2-resident at these sizes); products and sums in FP32
// registers, row by row.  Rows inside a chunk are written to M; the segments of rows cut
// by a chunk boundary go to per-chunk slots that a fix-up kernel adds in chunk order (no
// atomics: the result does not depend on scheduling).
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <string>

#include "ntf_internal.cuh"

struct ntf_sptensor {
  int N = 0;
  int64_t dims[ntf::kMaxOrder] = {};
  int64_t nnz = 0;
  cudaStream_t st = nullptr;
  // per mode: this mode's index, the other modes' indices and the value of each nonzero,
  // sorted by this mode's index ([nnz][N + 1] 32-bit words), and row offsets
  uint32_t* packed[ntf::kMaxOrder] = {};
  int64_t* rowptr[ntf::kMaxOrder] = {};
  float* partial = nullptr;  // [chunks][2][64] segments of rows cut by chunk boundaries
  void* arena = nullptr;
};

namespace {

thread_local std::string g_sp_err;

ntf_status spfail(ntf_status s, const char* fmt, ...) {
  char buf[256];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_sp_err = buf;
  return s;
}

constexpr int kTile = 4096;           // nonzeros per tile of a sort pass
constexpr int kSortThreads = 256;     // 16 rounds of 256 per tile
constexpr int kRounds = kTile / kSortThreads;

// Per-tile histogram of the digit (key >> shift) & 255 of the keys in tile order.
__global__ void __launch_bounds__(kSortThreads) k_digit_hist(const uint32_t* __restrict__ key,
                                                           int64_t n, int shift,
                                                           uint32_t* __restrict__ hist) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kTile;
  for (int r = 0; r < kRounds; ++r) {
    const int64_t e = base + r * kSortThreads + threadIdx.x;
    if (e < n) atomicAdd(&h[(key[e] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[static_cast<int64_t>(blockIdx.x) * 256 + threadIdx.x] = h[threadIdx.x];
}

// offsets[t][d] = (nonzeros with a smaller digit) + (nonzeros with digit d in tiles < t).
// One CTA of 256 threads, thread d walks the tiles of digit d.
__global__ void __launch_bounds__(256) k_digit_offsets(uint32_t* __restrict__ hist, int tiles) {
  __shared__ uint32_t tot[256];
  const int d = threadIdx.x;
  uint32_t run = 0;
  for (int t = 0; t < tiles; ++t) {
    const uint32_t c = hist[static_cast<int64_t>(t) * 256 + d];
    hist[static_cast<int64_t>(t) * 256 + d] = run;
    run += c;
  }
  tot[d] = run;
  __syncthreads();
  if (d == 0) {  // exclusive scan of the digit totals
    uint32_t acc = 0;
    for (int b = 0; b < 256; ++b) {
      const uint32_t c = tot[b];
      tot[b] = acc;
      acc += c;
    }
  }
  __syncthreads();
  for (int t = 0; t < tiles; ++t) hist[static_cast<int64_t>(t) * 256 + d] += tot[d];
}

// Stable scatter of (key, payload) by the digit: each tile places its nonzeros in order.
__global__ void __launch_bounds__(kSortThreads) k_digit_scatter(
    const uint32_t* __restrict__ key, const uint32_t* __restrict__ pay, int64_t n, int shift,
    const uint32_t* __restrict__ offsets, uint32_t* __restrict__ key_out,
    uint32_t* __restrict__ pay_out) {
  constexpr int kW = kSortThreads / 32;
  __shared__ uint32_t run[256];             // placed so far in this tile, per digit
  __shared__ uint32_t wcount[kW][256];      // this round's count per warp and digit
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  run[tid] = offsets[static_cast<int64_t>(blockIdx.x) * 256 + tid];
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kTile;
  for (int r = 0; r < kRounds; ++r) {
    for (int i = tid; i < kW * 256; i += kSortThreads) (&wcount[0][0])[i] = 0;
    __syncthreads();
    const int64_t e = base + r * kSortThreads + tid;
    const bool live = e < n;
    const uint32_t k = live ? key[e] : 0u;
    const uint32_t d = live ? (k >> shift) & 255u : 256u + lane;  // dead lanes: no match
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const uint32_t below = __popc(peers & ((1u << lane) - 1u));  // same digit, lower lane
    const int leader = __ffs(peers) - 1;
    if (live && lane == leader) wcount[warp][d] = __popc(peers);
    __syncthreads();
    if (live) {
      uint32_t pos = run[d] + below;
      for (int w = 0; w < warp; ++w) pos += wcount[w][d];
      key_out[pos] = k;
      pay_out[pos] = pay[e];
    }
    __syncthreads();
    // advance the per-digit counters by this round's counts (thread = digit)
    uint32_t c = 0;
    for (int w = 0; w < kW; ++w) c += wcount[w][tid];
    run[tid] += c;
    __syncthreads();
  }
}

// key[p] = the mode-`mode` index of nonzero pay[p] (the second key of a two-key sort).
__global__ void k_gather_keys(const int32_t* __restrict__ idx, int N, int mode, int64_t n,
                              const uint32_t* __restrict__ pay, uint32_t* __restrict__ key) {
  for (int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; p < n;
       p += static_cast<int64_t>(gridDim.x) * blockDim.x)
    key[p] = static_cast<uint32_t>(idx[static_cast<int64_t>(pay[p]) * N + mode]);
}

__global__ void k_iota_keys(const int32_t* __restrict__ idx, int N, int mode, int64_t n,
                            uint32_t* __restrict__ key, uint32_t* __restrict__ pay) {
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < n;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    key[e] = static_cast<uint32_t>(idx[e * N + mode]);
    pay[e] = static_cast<uint32_t>(e);
  }
}

// packed[p] = (key, other indices of nonzero perm[p], its value bits); rowptr by binary
// search of the sorted keys: rowptr[i] = number of nonzeros whose key is below i.
__global__ void k_pack(const int32_t* __restrict__ idx, const float* __restrict__ vals, int N,
                       int mode, int64_t n, const uint32_t* __restrict__ perm,
                       uint32_t* __restrict__ packed) {
  for (int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; p < n;
       p += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t e = perm[p];
    uint32_t* o = packed + p * (N + 1);
    o[0] = static_cast<uint32_t>(idx[e * N + mode]);
    int j = 1;
    for (int m = 0; m < N; ++m)
      if (m != mode) o[j++] = static_cast<uint32_t>(idx[e * N + m]);
    o[N] = __float_as_uint(vals[e]);
  }
}

__global__ void k_rowptr(const uint32_t* __restrict__ sorted_key, int64_t n, int64_t I,
                         int64_t* __restrict__ rowptr) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i <= I;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    int64_t lo = 0, hi = n;  // first position with key >= i
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (static_cast<int64_t>(sorted_key[mid]) < i) lo = mid + 1;
      else hi = mid;
    }
    rowptr[i] = lo;
  }
}

struct SpF {
  const float* F[ntf::kMaxOrder - 1];  // the other modes' factors, in mode order
};

constexpr int kChunk = 128;  // sorted nonzeros per warp

// One nonzero of a mode-sorted layout (N = 3: one 16-byte load).
template <int N>
__device__ __forceinline__ void load_nz(const uint32_t* __restrict__ q, uint32_t (&w)[N + 1]) {
  if constexpr (N == 3) {
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(q));
    w[0] = v.x;
    w[1] = v.y;
    w[2] = v.z;
    w[3] = v.w;
  } else {
#pragma unroll
    for (int k = 0; k <= N; ++k) w[k] = __ldg(q + k);
  }
}

// Chunk kernel: warp c sums the products of the sorted nonzeros [c kChunk, (c + 1) kChunk)
// row by row.  Lane l loads nonzero base + l of each group of 32 (one coalesced load for the
// warp); the warp then walks the group by broadcast, kUnroll nonzeros at a time with their
// factor-row gathers issued together (lanes over the rank: columns lane, lane + 32).  A row
// wholly inside the chunk is written to M; the segment of a row that began before the chunk
// goes to partial[c][0], that of a row continuing past it to partial[c][1] (the fix-up
// kernel adds the segments of such rows in chunk order).
template <int N>
__global__ void __launch_bounds__(256) k_sp_chunks(const uint32_t* __restrict__ packed,
                                                   int64_t nnz, int R, SpF f,
                                                   float* __restrict__ M,
                                                   float* __restrict__ partial) {
  constexpr int kUnroll = 8;
  const int lane = threadIdx.x & 31;
  const bool h0 = lane < R, h1 = lane + 32 < R;
  const int64_t chunks = (nnz + kChunk - 1) / kChunk;
  const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
  for (int64_t c = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
       c < chunks; c += warps) {
    const int64_t p0 = c * kChunk, p1 = p0 + kChunk < nnz ? p0 + kChunk : nnz;
    uint32_t row = __ldg(packed + p0 * (N + 1));
    bool before = p0 > 0 && __ldg(packed + (p0 - 1) * (N + 1)) == row;
    float a0 = 0.0f, a1 = 0.0f;
    float* const part = partial + c * 2 * 64;
    auto flush = [&](bool cont) {
      float* o = before ? part : cont ? part + 64 : M + static_cast<int64_t>(row) * R;
      if (h0) o[lane] = a0;
      if (h1) o[lane + 32] = a1;
    };
    for (int64_t base = p0; base < p1; base += 32) {
      const int cnt = p1 - base < 32 ? static_cast<int>(p1 - base) : 32;
      uint32_t mine[N + 1];
      if (lane < cnt) {
        load_nz<N>(packed + (base + lane) * (N + 1), mine);
      } else {
#pragma unroll
        for (int k = 0; k <= N; ++k) mine[k] = 0;
      }
      for (int j0 = 0; j0 < cnt; j0 += kUnroll) {
        uint32_t key[kUnroll];
        float t0[kUnroll], t1[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {  // broadcast nonzero j0 + u, gather its rows
          const int j = j0 + u < cnt ? j0 + u : cnt - 1;
          key[u] = __shfl_sync(0xffffffffu, mine[0], j);
          const float v = __uint_as_float(__shfl_sync(0xffffffffu, mine[N], j));
          float c0 = v, c1 = v;
#pragma unroll
          for (int m = 0; m < N - 1; ++m) {
            const uint32_t im = __shfl_sync(0xffffffffu, mine[1 + m], j);
            const float* fr = f.F[m] + static_cast<int64_t>(im) * R;
            if (h0) c0 *= __ldg(fr + lane);
            if (h1) c1 *= __ldg(fr + lane + 32);
          }
          t0[u] = c0;
          t1[u] = c1;
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {  // accumulate in order, row by row
          if (j0 + u >= cnt) break;           // warp-uniform
          if (key[u] != row) {
            flush(false);
            before = false;
            row = key[u];
            a0 = a1 = 0.0f;
          }
          a0 += t0[u];
          a1 += t1[u];
        }
      }
    }
    flush(p1 < nnz && __ldg(packed + p1 * (N + 1)) == row);
  }
}

// The same chunks for R <= 32 (one column per lane), with fewer instructions per nonzero: each
// group of 32 nonzeros is loaded coalesced (the next group's load issued before the current
// group is walked) and staged in shared memory, from which every lane reads the nonzero it
// walks as one broadcast load (instead of a shuffle per field); the row of the first other
// mode, whose equal indices the layout keeps together within a row, stays in a register while
// the index repeats; the rows of the other modes are gathered kUnroll nonzeros at a time.
template <int N>
__global__ void __launch_bounds__(256) k_sp_chunks32(const uint32_t* __restrict__ packed,
                                                     int64_t nnz, int R, SpF f,
                                                     float* __restrict__ M,
                                                     float* __restrict__ partial) {
  constexpr int kUnroll = 8, kW = N + 1;
  __shared__ __align__(16) uint32_t s_nz[8][32 * kW + 4];  // per warp: 32 nonzeros (N + 1 words)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t* const sw = s_nz[warp];
  const bool h = lane < R;
  const int64_t chunks = (nnz + kChunk - 1) / kChunk;
  const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
  for (int64_t c = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + warp; c < chunks;
       c += warps) {
    const int64_t p0 = c * kChunk, p1 = p0 + kChunk < nnz ? p0 + kChunk : nnz;
    uint32_t row = __ldg(packed + p0 * kW);
    bool before = p0 > 0 && __ldg(packed + (p0 - 1) * kW) == row;
    float acc = 0.0f;
    uint32_t cur = 0xFFFFFFFFu;  // index of the first other mode's row held in g
    float g = 0.0f;
    float* const part = partial + c * 2 * 64;
    auto flush = [&](bool cont) {
      float* o = before ? part : cont ? part + 64 : M + static_cast<int64_t>(row) * R;
      if (h) o[lane] = acc;
    };
    uint32_t nxt[kW];
    if (lane < p1 - p0) {
      load_nz<N>(packed + (p0 + lane) * kW, nxt);
    } else {
#pragma unroll
      for (int k = 0; k < kW; ++k) nxt[k] = 0;
    }
    for (int64_t base = p0; base < p1; base += 32) {
      const int cnt = p1 - base < 32 ? static_cast<int>(p1 - base) : 32;
      __syncwarp();
      if constexpr (N == 3) {
        *reinterpret_cast<uint4*>(sw + lane * 4) = make_uint4(nxt[0], nxt[1], nxt[2], nxt[3]);
      } else {
#pragma unroll
        for (int k = 0; k < kW; ++k) sw[lane * kW + k] = nxt[k];
      }
      __syncwarp();
      if (base + 32 + lane < p1) load_nz<N>(packed + (base + 32 + lane) * kW, nxt);
      for (int j0 = 0; j0 < cnt; j0 += kUnroll) {
        float t[kUnroll];
        uint32_t key[kUnroll], i1[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {  // value times the rows of modes 2 .. N-1
          const int j = j0 + u < cnt ? j0 + u : cnt - 1;
          uint32_t q[kW];
          if constexpr (N == 3) {
            const uint4 w = *reinterpret_cast<const uint4*>(sw + j * 4);  // broadcast
            q[0] = w.x;
            q[1] = w.y;
            q[2] = w.z;
            q[3] = w.w;
          } else {
#pragma unroll
            for (int k = 0; k < kW; ++k) q[k] = sw[j * kW + k];
          }
          key[u] = q[0];
          i1[u] = q[1];
          float v = __uint_as_float(q[N]);
#pragma unroll
          for (int m = 1; m < N - 1; ++m)
            v *= h ? __ldg(f.F[m] + static_cast<int64_t>(q[1 + m]) * R + lane) : 0.0f;
          t[u] = v;
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {  // in order: row changes, the first mode's row
          if (j0 + u >= cnt) break;           // warp-uniform
          if (key[u] != row) {
            flush(false);
            before = false;
            row = key[u];
            acc = 0.0f;
          }
          if (i1[u] != cur) {  // warp-uniform
            cur = i1[u];
            g = h ? __ldg(f.F[0] + static_cast<int64_t>(cur) * R + lane) : 0.0f;
          }
          acc = fmaf(t[u], g, acc);
        }
      }
    }
    flush(p1 < nnz && __ldg(packed + p1 * kW) == row);
  }
}

// Rows cut by chunk boundaries: the sum of their segments in chunk order; rows without
// nonzeros: zero.  One warp per row.
__global__ void __launch_bounds__(256) k_sp_fixup(const int64_t* __restrict__ rowptr, int64_t I,
                                                  int R, const float* __restrict__ partial,
                                                  float* __restrict__ M) {
  const int lane = threadIdx.x & 31;
  const bool h0 = lane < R, h1 = lane + 32 < R;
  const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
       i < I; i += warps) {
    const int64_t s = rowptr[i], e = rowptr[i + 1];
    float a0 = 0.0f, a1 = 0.0f;
    if (s < e) {
      const int64_t c0 = s / kChunk, c1 = (e - 1) / kChunk;
      if (c0 == c1) continue;  // written by its chunk
      const float* q = partial + c0 * 2 * 64 + 64;  // the row continues past chunk c0
      if (h0) a0 = q[lane];
      if (h1) a1 = q[lane + 32];
      for (int64_t c = c0 + 1; c <= c1; ++c) {   // began before chunks c0+1 .. c1
        const float* r = partial + c * 2 * 64;
        if (h0) a0 += r[lane];
        if (h1) a1 += r[lane + 32];
      }
    }
    if (h0) M[i * R + lane] = a0;
    if (h1) M[i * R + lane + 32] = a1;
  }
}

unsigned grid_for(int64_t n, int threads) {
  return static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads,
                                                                       8 * ntf::kNumSM)));
}

bool misaligned(const void* p, uintptr_t elem) { return reinterpret_cast<uintptr_t>(p) % elem != 0; }

}  // namespace

extern "C" {

ntf_status ntf_sptensor_create(ntf_sptensor** out, int order, const int64_t* dims, int64_t nnz,
                               const int32_t* d_idx, const float* d_vals, void* stream) {
  if (!out) return spfail(NTF_ERR_INVALID_ARG, "null output pointer");
  *out = nullptr;
  if (order < 3 || order > ntf::kMaxOrder || !dims)
    return spfail(NTF_ERR_INVALID_ARG, "order must be 3 or 4");
  if (nnz < 1 || nnz >= (int64_t{1} << 31) || !d_idx || !d_vals)
    return spfail(NTF_ERR_INVALID_ARG, "need 1 <= nnz < 2^31 and non-null indices and values");
  if (misaligned(d_idx, 4) || misaligned(d_vals, 4))
    return spfail(NTF_ERR_INVALID_ARG, "indices and values must be 4-byte aligned");
  for (int m = 0; m < order; ++m)
    if (dims[m] < 1 || dims[m] > (int64_t{1} << 30))
      return spfail(NTF_ERR_INVALID_ARG, "dims[%d] out of range", m);
  ntf_sptensor* s = new ntf_sptensor();
  s->N = order;
  s->nnz = nnz;
  s->st = static_cast<cudaStream_t>(stream);
  int64_t maxdim = 0;
  for (int m = 0; m < order; ++m) {
    s->dims[m] = dims[m];
    maxdim = std::max(maxdim, dims[m]);
  }
  const int64_t tiles = (nnz + kTile - 1) / kTile;
  // arena: per mode packed [nnz][N] + rowptr [I+1]; sort scratch: keys, payloads (x2),
  // tile histograms
  size_t off = 0;
  auto take = [&](size_t b) { const size_t o = off; off += (b + 255) / 256 * 256; return o; };
  size_t oP[ntf::kMaxOrder], oR[ntf::kMaxOrder];
  for (int m = 0; m < order; ++m) {
    oP[m] = take(static_cast<size_t>(nnz) * (order + 1) * 4);
    oR[m] = take(static_cast<size_t>(dims[m] + 1) * 8);
  }
  const int64_t chunks = (nnz + kChunk - 1) / kChunk;
  const size_t oK0 = take(nnz * 4), oK1 = take(nnz * 4), oQ0 = take(nnz * 4),
               oQ1 = take(nnz * 4), oH = take(static_cast<size_t>(tiles) * 256 * 4),
               oPart = take(static_cast<size_t>(chunks) * 2 * 64 * 4);
  cudaError_t e = cudaMalloc(&s->arena, off);
  if (e != cudaSuccess) {
    delete s;
    return spfail(NTF_ERR_OOM, "sparse tensor layout: %s", cudaGetErrorString(e));
  }
  char* b = static_cast<char*>(s->arena);
  for (int m = 0; m < order; ++m) {
    s->packed[m] = reinterpret_cast<uint32_t*>(b + oP[m]);
    s->rowptr[m] = reinterpret_cast<int64_t*>(b + oR[m]);
  }
  uint32_t* key[2] = {reinterpret_cast<uint32_t*>(b + oK0), reinterpret_cast<uint32_t*>(b + oK1)};
  uint32_t* pay[2] = {reinterpret_cast<uint32_t*>(b + oQ0), reinterpret_cast<uint32_t*>(b + oQ1)};
  uint32_t* hist = reinterpret_cast<uint32_t*>(b + oH);
  s->partial = reinterpret_cast<float*>(b + oPart);
  cudaStream_t st = s->st;
  for (int m = 0; m < order && e == cudaSuccess; ++m) {
    // two stable passes of the radix sort: by the first other mode's index, then by this
    // mode's (the order of the first survives among equal i_n)
    const int m2 = m == 0 ? 1 : 0;
    k_iota_keys<<<grid_for(nnz, 256), 256, 0, st>>>(d_idx, order, m2, nnz, key[0], pay[0]);
    int cur = 0;
    for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {
      const int64_t I = pass == 0 ? dims[m2] : dims[m];
      if (pass == 1) {
        k_gather_keys<<<grid_for(nnz, 256), 256, 0, st>>>(d_idx, order, m, nnz, pay[cur],
                                                          key[cur]);
      }
      for (int shift = 0; shift < 32 && e == cudaSuccess; shift += 8) {
        if (shift > 0 && (I - 1) >> shift == 0) break;  // the remaining digits are zero
        k_digit_hist<<<static_cast<unsigned>(tiles), kSortThreads, 0, st>>>(key[cur], nnz,
                                                                           shift, hist);
        k_digit_offsets<<<1, 256, 0, st>>>(hist, static_cast<int>(tiles));
        k_digit_scatter<<<static_cast<unsigned>(tiles), kSortThreads, 0, st>>>(
            key[cur], pay[cur], nnz, shift, hist, key[cur ^ 1], pay[cur ^ 1]);
        cur ^= 1;
        e = cudaGetLastError();
      }
    }
    if (e != cudaSuccess) break;
    k_pack<<<grid_for(nnz, 256), 256, 0, st>>>(d_idx, d_vals, order, m, nnz, pay[cur],
                                                s->packed[m]);
    k_rowptr<<<grid_for(dims[m] + 1, 256), 256, 0, st>>>(key[cur], nnz, dims[m], s->rowptr[m]);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaFree(s->arena);
    delete s;
    return spfail(NTF_ERR_CUDA, "sparse tensor layout: %s", cudaGetErrorString(e));
  }
  *out = s;
  return NTF_OK;
}

ntf_status ntf_sptensor_destroy(ntf_sptensor* s) {
  if (s) {
    cudaStreamSynchronize(s->st);
    cudaFree(s->arena);
    delete s;
  }
  return NTF_OK;
}

ntf_status ntf_sptensor_mttkrp(ntf_sptensor* s, int mode, int rank,
                               const float* const* d_factors, float* d_M) {
  (void)cudaGetLastError();  // a stale non-sticky error is not this call's
  if (!s) return spfail(NTF_ERR_INVALID_ARG, "null sparse tensor");
  if (mode < 0 || mode >= s->N) return spfail(NTF_ERR_INVALID_ARG, "mode %d out of range", mode);
  if (rank < 1 || rank > ntf::kMaxRank)
    return spfail(NTF_ERR_INVALID_ARG, "rank %d not in [1, %d]", rank, ntf::kMaxRank);
  if (!d_factors || !d_M || misaligned(d_M, 4))
    return spfail(NTF_ERR_INVALID_ARG, "null factors or null / misaligned output");
  SpF f{};
  int j = 0;
  for (int m = 0; m < s->N; ++m) {
    if (m == mode) continue;
    if (!d_factors[m] || misaligned(d_factors[m], 4))
      return spfail(NTF_ERR_INVALID_ARG, "null or misaligned factor %d", m);
    f.F[j++] = d_factors[m];
  }
  const int64_t I = s->dims[mode];
  const int64_t chunks = (s->nnz + kChunk - 1) / kChunk;
  const unsigned gc = grid_for(chunks * 32, 256), gf = grid_for(I * 32, 256);
  if (rank <= 32 && s->N == 3)
    k_sp_chunks32<3><<<gc, 256, 0, s->st>>>(s->packed[mode], s->nnz, rank, f, d_M, s->partial);
  else if (rank <= 32)
    k_sp_chunks32<4><<<gc, 256, 0, s->st>>>(s->packed[mode], s->nnz, rank, f, d_M, s->partial);
  else if (s->N == 3)
    k_sp_chunks<3><<<gc, 256, 0, s->st>>>(s->packed[mode], s->nnz, rank, f, d_M, s->partial);
  else
    k_sp_chunks<4><<<gc, 256, 0, s->st>>>(s->packed[mode], s->nnz, rank, f, d_M, s->partial);
  k_sp_fixup<<<gf, 256, 0, s->st>>>(s->rowptr[mode], I, rank, s->partial, d_M);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return spfail(NTF_ERR_CUDA, "sparse MTTKRP: %s", cudaGetErrorString(e));
  return NTF_OK;
}

int64_t ntf_sptensor_nnz(const ntf_sptensor* s) { return s ? s->nnz : -1; }

const char* ntf_sptensor_last_error(void) { return g_sp_err.c_str(); }

}  // extern "C"
