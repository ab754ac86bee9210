// Tensor-core MTTKRP contractions (tcgen05 + TMA).  Included by umma_{bf16,f32}.cu.
//
// The two skinny contractions of the sweep (mttkrp.cu)
//
//   GEMM-N:  out[p, r] = sum_q X[p, q] W[q, r]        (A = X tile, K-major)
//   GEMM-T:  out[q, r] = sum_p X[p, q] W[p, r]        (A = X^T tile, M-contiguous)
//
// run as D[128 x N] += A[128 x K] * B[K x N] on the 5th-generation tensor cores, with the
// output rows (M = 128 per tile) on the TMEM lanes and the padded rank N on TMEM columns.
//
// Precision.  The tensor cores multiply 16-bit or TF32 operands exactly into FP32 sums, so
// the FP32 contract is kept by splitting operands into sums of narrower parts:
//   BF16 storage: X is exact in BF16; W = w1 + w2 + w3 with w1 = bf16(W),
//                 w2 = bf16(W - w1), w3 = bf16(W - w1 - w2) (24 significant bits), and
//                 X W = X w1 + X w2 + X w3 (one kind::f16 MMA per K step with the three
//                 parts side by side in N, summed by the epilogue).
//   FP32 storage: X = xh + xl and W = wh + wl with xh, wh = the value truncated to TF32
//                 (10 stored mantissa bits) and xl, wl = the exact remainders; X W is formed
//                 as xh wh + xh wl + xl wh (two kind::tf32 MMAs), dropping xl wl
//                 (relative size 2^-22).  A kind::tf32 MMA reads an FP32 operand by its
//                 sign, exponent and 10 leading mantissa bits, so a tensor value serves as
//                 its own xh: converter warps write xl beside the K-major tensor tile (and,
//                 for GEMM-T, first transpose the tile in place), between the TMA load and
//                 the MMA.
//
// CTA roles (persistent: one CTA per SM walks the (tile, K-chunk) work items):
//   warps 0-3  epilogue: TMEM -> registers -> global, warp w owns TMEM lanes 32w..32w+31
//   warp 4     TMA producer (one thread): X tile + all W split rows of the stage
//   warp 5     MMA issuer (one thread): tcgen05.mma into a double-buffered accumulator; a
//              tile's contraction range is accumulated in segments of 8 stages, each in a
//              fresh accumulator that the epilogue adds into FP32 registers
//   warps 6-9  (FP32 only) converters: the lo operand tile xl (GEMM-T: and the transpose)
// Stages form a ring guarded by mbarriers (full: TMA bytes landed; ready: converted; empty:
// the MMAs reading the stage completed).  Every wait is bounded: on timeout the kernel sets
// the timeout bit in *err, every role leaves its loop, outstanding copies and MMAs are
// drained (bounded), and the TMEM is freed before the CTA exits.
#pragma once
#include <cuda.h>

#include "ntf_internal.cuh"

namespace ntf {
namespace umma {

constexpr int kTileM = 128;
constexpr int kItemQ = 4;  // work-item slots between the producer and the other roles
constexpr int kSmemBudget = 200 * 1024;
constexpr uint64_t kWaitNs = 2000000000ull;  // a wait gives up after 2 s

// kWRes (BF16 only): the whole split Khatri-Rao table of the contraction (at most kWBlocks
// 64-deep K blocks) is loaded into shared memory once per CTA, and the stages carry the
// tensor tile only -- more tensor bytes in flight and half the L2 -> SM traffic.
template <bool kT, bool kF32, int kN, bool kWRes = false>
struct Cfg {
  static_assert(!(kWRes && kF32), "resident tables are for BF16 storage");
  static constexpr int kStageK = kF32 ? 32 : 64;   // K per stage: 128 bytes of one row
  static constexpr int kSplits = kF32 ? 2 : 3;     // W parts
  static constexpr int kABytes = kTileM * 128;     // tensor tile (the hi part for FP32)
  static constexpr int kLoBytes = kF32 ? kTileM * 128 : 0;
  static constexpr int kWBlockBytes = kSplits * kN * 128;            // W rows of one K block
  static constexpr int kWBytes = kWRes ? 0 : kWBlockBytes;           // W per stage
  static constexpr int kWBlocks = kWRes ? (kN <= 16 ? 8 : 7) : 0;    // resident K blocks
  static constexpr int kWResBytes = kWBlocks * kWBlockBytes;
  // (FP32 GEMM-T: the untransposed X rows land in the operand tile and are transposed there)
  static constexpr int kStageBytes = kABytes + kLoBytes + kWBytes;
  static constexpr int kStagesRaw =
      ((kWRes ? 224 * 1024 : kSmemBudget) - kWResBytes) / kStageBytes;
  static constexpr int kStagesMax = kWRes ? 8 : 6;
  static constexpr int kStages = kStagesRaw > kStagesMax ? kStagesMax : kStagesRaw;
  static constexpr int kTxBytes = kABytes + kWBytes;
  static constexpr int kWarps = kF32 ? 10 : 6;
  static constexpr int kThreads = kWarps * 32;
  // Accumulator of one segment: one N-column block per W part (x w1 | x w2 | x w3 for BF16,
  // xh wh | xh wl + xl wh for FP32); two of them alternate between MMA and epilogue.
  static constexpr int kAccCols = kSplits * kN;
  static constexpr int kAccStride = kAccCols <= 32 ? 32 : kAccCols <= 64 ? 64 : kAccCols <= 128 ? 128 : 256;
  static constexpr int kTmemCols = 2 * kAccStride;
  // Stages accumulated in TMEM before the epilogue takes the partial sum into FP32 registers.
  // The tensor-core accumulation does not round to nearest (each MMA adds a small one-sided
  // error, ~2^-24 of the sum); capping the number of MMAs per accumulator caps that bias
  // at 32 main-block additions (~2e-6 relative), and the register sums round to nearest.
  static constexpr int kSegStages = 8;
  static constexpr int kSmemBytes = kWResBytes + kStages * kStageBytes + 1024;  // + alignment
  static_assert(kStages >= 2, "stage does not fit");
  static_assert(kStageBytes % 1024 == 0, "stage pieces must stay 1024-byte aligned");
  static_assert(kWBlockBytes % 1024 == 0, "W blocks must stay 1024-byte aligned");
  static_assert(kN % 16 == 0 && kN >= 16 && kN <= 64, "N must be 16..64 in steps of 16");
  static_assert(kTmemCols <= 512, "accumulators exceed the tensor memory");
};

// Args (the work-item description shared with the host) is declared in ntf_internal.cuh.

// ----------------------------------------------------------------------------- PTX
__device__ __forceinline__ uint32_t saddr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void bar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(saddr(b)), "r"(count));
}

__device__ __forceinline__ void bar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(saddr(b)) : "memory");
}

__device__ __forceinline__ void bar_arrive_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(saddr(b)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool bar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.b32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(saddr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
  return t;
}

// Bounded wait for the phase of parity `parity` to complete; false after limit_ns or, when
// abort_flag is given, once another role has given up.
__device__ __forceinline__ bool bar_wait(uint64_t* b, uint32_t parity,
                                         volatile int* abort_flag,
                                         uint64_t limit_ns = kWaitNs) {
  uint64_t t0 = 0;
  for (uint32_t n = 0;; ++n) {
    if (bar_try(b, parity)) return true;
    if (abort_flag && *abort_flag) return false;
    if ((n & 255u) == 0) {
      const uint64_t t = now_ns();
      if (n == 0) t0 = t;
      else if (t - t0 > limit_ns) return false;
    }
  }
}

// The same for waits that last a whole accumulation segment (the epilogue's): a short sleep
// between tests leaves the SM's issue slots to the kernels that share it.
__device__ __forceinline__ bool bar_wait_patient(uint64_t* b, uint32_t parity,
                                                 volatile int* abort_flag) {
  uint64_t t0 = 0;
  for (uint32_t n = 0;; ++n) {
    if (bar_try(b, parity)) return true;
    if (abort_flag && *abort_flag) return false;
    const uint64_t t = now_ns();
    if (n == 0) t0 = t;
    else if (t - t0 > kWaitNs) return false;
    __nanosleep(256);
  }
}

__device__ __forceinline__ void tma_2d(void* dst, const CUtensorMap* map, int x, int y,
                                       uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];\n" ::"r"(saddr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(saddr(bar))
      : "memory");
}

// Shared-memory matrix descriptor (tcgen05): start address, leading / stride byte offsets,
// the fixed version bits 46-48 = 0b001, 128-byte swizzle (mode 2 in bits 61-63).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = static_cast<uint64_t>((addr & 0x3FFFFu) >> 4);
  d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16;
  d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32;
  d |= 1ull << 46;
  d |= 2ull << 61;
  return d;
}

// Instruction descriptor: FP32 accumulator, operand formats (f16 kind: 1 = BF16; tf32 kind:
// 2 = TF32), A major-ness (0 = K-major, 1 = M-contiguous), N >> 3, M >> 4.
__host__ __device__ constexpr uint32_t idesc(uint32_t fmt, uint32_t a_mn, int n, int m) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | (a_mn << 15) |
         (static_cast<uint32_t>(n >> 3) << 17) | (static_cast<uint32_t>(m >> 4) << 24);
}

template <bool kF32>
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id,
                                    uint32_t acc) {
  if constexpr (kF32)
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(id), "r"(acc));
  else
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(id), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* b) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
          saddr(b))
      : "memory");
}

__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}

// 16 consecutive FP32 accumulator columns of this warp's 32 TMEM lanes (one row per lane).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

// TF32 split remainder: hi = x with its 13 trailing mantissa bits cleared (sign, exponent and
// the 10 leading mantissa bits, what a kind::tf32 MMA reads of x); lo = x - hi, exact.
__device__ __forceinline__ float tf32_rem(float x) {
  return x - __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
}

// Sums over the 32 lanes of a warp of x[0..31], one column per lane: lane l returns the sum
// of the lanes' x[l].  Halves are exchanged at distances 16, 8, 4, 2, 1 (a lane keeps the
// half its lane bit selects and adds its partner's copy of it): 31 shuffles, a fixed order.
__device__ __forceinline__ float warp_colsum(float (&x)[32], int lane) {
#pragma unroll
  for (int h = 16; h >= 1; h >>= 1) {
    const bool up = (lane & h) != 0;
#pragma unroll
    for (int j = 0; j < h; ++j) {
      const float send = up ? x[j] : x[j + h];
      const float keep = up ? x[j + h] : x[j];
      x[j] = keep + __shfl_xor_sync(0xffffffffu, send, h);
    }
  }
  return x[0];
}

// The leading mode's second tree level for this warp's 32 output rows (group g): row
// p = a Ib + b weighs its row v by F[b]; the group's rows belong to at most two values of a
// (Ib >= 32), a0 = 32 g / Ib and a0 + 1, whose column sums go to part[g][0] and part[g][1]
// (the second only when the group reaches a0 + 1: no other slot is read).  v is consumed.
template <int kN>
__device__ __forceinline__ void post_group(const Args& a, float (&v)[kN], int tile, int warp,
                                           int lane) {
  const int64_t g = static_cast<int64_t>(tile) * (kTileM / 32) + warp;
  if (g * 32 >= a.M) return;  // warp-uniform: no rows
  const int64_t p = g * 32 + lane;
  const bool live = p < a.M;
  const int64_t a0 = (g * 32) / a.post_Ib;
  const int64_t ar = live ? p / a.post_Ib : a0;
  const int seg = static_cast<int>(ar - a0);
  const float* f = a.post_F + (live ? p - ar * a.post_Ib : 0) * a.R;
  if ((a.R & 3) == 0) {  // rows of F 16-byte aligned: four columns per load
#pragma unroll
    for (int c = 0; c < kN; c += 4) {
      const float4 q = live && c < a.R ? __ldg(reinterpret_cast<const float4*>(f + c))
                                       : make_float4(0.f, 0.f, 0.f, 0.f);
      v[c] *= q.x;
      v[c + 1] *= q.y;
      v[c + 2] *= q.z;
      v[c + 3] *= q.w;
    }
  } else {
#pragma unroll
    for (int c = 0; c < kN; ++c) v[c] = live && c < a.R ? v[c] * __ldg(f + c) : 0.0f;
  }
  const int segs = __any_sync(0xffffffffu, seg == 1) ? 2 : 1;
  for (int sg = 0; sg < segs; ++sg) {
    float* dst = a.post_part + (g * 2 + sg) * a.R;
#pragma unroll
    for (int blk = 0; blk < kN; blk += 32) {
      float x[32];
#pragma unroll
      for (int j = 0; j < 32; ++j)
        x[j] = blk + j < kN && seg == sg ? v[blk + j < kN ? blk + j : 0] : 0.0f;
      const float sum = warp_colsum(x, lane);
      if (blk + lane < a.R) dst[blk + lane] = sum;
    }
  }
}

// ---------------------------------------------------------------------------- kernel
// Register cap: the sweep's other kernels (factor updates, reductions, coefficient systems,
// second tree levels) run beside the persistent contraction, and one of their 8-warp CTAs
// shares an SM with a contraction CTA only if two of its warps fit next to the contraction's
// two warps in a scheduler's 16384 registers.  At N = 64 the uncapped kernel takes 202
// registers (13312 of a scheduler's registers for two warps) and nothing fits; capped at 168
// (10752) the reductions and second tree levels (80-84 registers) do, for a few spilled bytes.
// FP32 (ten warps): capped at 112 at N <= 32, so that two warps of a second tree level (84
// registers) fit beside the three contraction warps a scheduler holds.
template <int kN, bool kF32>
constexpr int kUmmaMaxRegs = kN > 32 ? 168 : kF32 ? 112 : 144;

template <bool kT, bool kF32, int kN, bool kWRes>
__global__ void __maxnreg__((kUmmaMaxRegs<kN, kF32>))
    k_umma(const __grid_constant__ CUtensorMap tx, const __grid_constant__ CUtensorMap tw,
           Args a) {
  using C = Cfg<kT, kF32, kN, kWRes>;
  constexpr int S = C::kStages;
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t full[S], ready[S], empty[S], tfull[2], tempty[2], drain, wfull;
  __shared__ uint64_t cread[S];  // FP32 GEMM-T: every converter warp has read the raw tile
  __shared__ uint64_t ifull[kItemQ], iempty[kItemQ];
  __shared__ int s_item[kItemQ];
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  __shared__ int skip_flag;

  // No work (a sweep of a run that has stopped): the CTA only takes part in the counter
  // protocol.  The flag is read once per CTA; CTAs that read it before it was set take every
  // item between them through the work-item counter.
  if (threadIdx.x == 0) skip_flag = a.skip ? *reinterpret_cast<const volatile int*>(a.skip) : 0;
  __syncthreads();
  if (skip_flag) {
    if (threadIdx.x == 0 && atomicAdd(a.sched + 1, 1u) == gridDim.x - 1) {
      a.sched[0] = 0;
      a.sched[1] = 0;
    }
    return;
  }

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t base_s = (saddr(smem_raw) + 1023u) & ~1023u;
  uint8_t* base = smem_raw + (base_s - saddr(smem_raw));
  const int items = a.tiles * a.chunks;
  const int nks_all = static_cast<int>((a.K + C::kStageK - 1) / C::kStageK);  // K blocks

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      bar_init(&full[s], 1);
      bar_init(&ready[s], 4);
      bar_init(&cread[s], 4);
      bar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      bar_init(&tfull[b], 1);
      bar_init(&tempty[b], 4);
    }
    bar_init(&drain, 1);
    bar_init(&wfull, 1);
    for (int q = 0; q < kItemQ; ++q) {
      bar_init(&ifull[q], 1);
      bar_init(&iempty[q], kF32 ? 9 : 5);  // MMA thread, 4 epilogue (+ 4 converter) warps
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     saddr(&tmem_base)),
                 "r"(C::kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_base;
  volatile int* abrt = &abort_flag;
  auto give_up = [&]() {
    if (!*abrt) {
      *abrt = 1;
      atomicOr(a.err, kStTimeout);
    }
  };

  // Work items come from a global counter (dynamic scheduling: a CTA that shares its SM with
  // another kernel takes fewer items).  The producer fetches them and hands them to the other
  // roles through a small ring of item slots; every role sees the same sequence, ending with
  // the sentinel `items`.
  auto next_item = [&](uint32_t u, int& it) -> bool {  // consumers; false on timeout
    const int q = u % kItemQ;
    if (!bar_wait(&ifull[q], (u / kItemQ) & 1, abrt)) return false;
    it = s_item[q];
    return true;
  };
  // shared memory: [resident W blocks (kWRes)] [stages]
  uint8_t* const wres = base;
  const uint32_t wres_s = base_s;
  const uint32_t stages_s = base_s + C::kWResBytes;
  auto stage_ptr = [&](int slot) { return base + C::kWResBytes + slot * C::kStageBytes; };
  // piece offsets within a stage
  constexpr int kOffA = 0, kOffLo = C::kABytes, kOffW = kOffLo + C::kLoBytes;

  if (warp == 4) {
    // ------------------------------------------------------------------ TMA producer
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&tx)) : "memory");
      asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&tw)) : "memory");
      if constexpr (kWRes) {  // the whole split table, once
        bar_arrive_tx(&wfull, static_cast<uint32_t>(nks_all * C::kWBlockBytes));
        for (int kb = 0; kb < nks_all; ++kb)
          tma_2d(wres + kb * C::kWBlockBytes, &tw, kb * C::kStageK, 0, &wfull);
      }
      uint32_t g = 0;
      bool ok = true;
      for (uint32_t u = 0; ok; ++u) {
        const int q = u % kItemQ;
        if (!bar_wait(&iempty[q], ((u / kItemQ) & 1) ^ 1, abrt)) {
          give_up();
          ok = false;
          break;
        }
        int it = static_cast<int>(atomicAdd(a.sched, 1u));
        if (it > items) it = items;
        s_item[q] = it;
        bar_arrive(&ifull[q]);
        if (it >= items) break;
        const int tile = it % a.tiles, ch = it / a.tiles;
        const int64_t k0 = ch * a.chunk_len;
        const int64_t k1 = a.K < k0 + a.chunk_len ? a.K : k0 + a.chunk_len;
        const int nks = static_cast<int>((k1 - k0 + C::kStageK - 1) / C::kStageK);
        for (int ks = 0; ks < nks; ++ks, ++g) {
          const int slot = g % S;
          if (!bar_wait(&empty[slot], ((g / S) & 1) ^ 1, abrt)) {
            give_up();
            ok = false;
            break;
          }
          uint8_t* st = stage_ptr(slot);
          bar_arrive_tx(&full[slot], C::kTxBytes);
          const int kx = static_cast<int>(k0 + ks * C::kStageK);
          const int m0 = tile * kTileM;
          if constexpr (!kT) {
            tma_2d(st + kOffA, &tx, kx, m0, &full[slot]);
          } else if constexpr (!kF32) {
            tma_2d(st + kOffA, &tx, m0, kx, &full[slot]);
            tma_2d(st + kOffA + kTileM * 64, &tx, m0 + 64, kx, &full[slot]);
          } else {
            tma_2d(st + kOffA, &tx, m0, kx, &full[slot]);  // raw rows, transposed in place
          }
          if constexpr (!kWRes) tma_2d(st + kOffW, &tw, kx, 0, &full[slot]);
        }
      }
      // copies still in flight (only possible after a timeout) land before the CTA exits:
      // the last use of every slot has completed its phase
      if (!ok) {
        for (uint32_t h = g > S ? g - S : 0; h < g; ++h) bar_wait(&full[h % S], (h / S) & 1, nullptr);
        if constexpr (kWRes) bar_wait(&wfull, 0, nullptr);
      }
    }
  } else if (warp == 5) {
    // ------------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      // BF16: one MMA per K step, B = [w1 | w2 | w3] (N' = 3N) -> the three column blocks.
      // FP32: xh [wh | wl] (N' = 2N) -> blocks 0 and 1, then xl wh -> block 1.
      constexpr uint32_t kIdWide =
          idesc(kF32 ? 2u : 1u, (kT && !kF32) ? 1u : 0u, C::kAccCols, kTileM);
      constexpr uint32_t kIdLo = idesc(2u, 0u, kN, kTileM);
      uint32_t g = 0, u = 0;
      bool ok = true, issued = false;
      if constexpr (kWRes) {
        if (!bar_wait(&wfull, 0, abrt)) {
          give_up();
          ok = false;
        }
      }
      for (uint32_t v = 0; ok; ++v) {
        int it;
        if (!next_item(v, it)) {
          give_up();
          ok = false;
          break;
        }
        bar_arrive(&iempty[v % kItemQ]);
        if (it >= items) break;
        const int ch = it / a.tiles;
        const int64_t k0 = ch * a.chunk_len;
        const int64_t k1 = a.K < k0 + a.chunk_len ? a.K : k0 + a.chunk_len;
        const int nks = static_cast<int>((k1 - k0 + C::kStageK - 1) / C::kStageK);
        for (int s0 = 0; s0 < nks && ok; s0 += C::kSegStages, ++u) {
          const int s1 = nks < s0 + C::kSegStages ? nks : s0 + C::kSegStages;
          const uint32_t b = u & 1;
          if (!bar_wait(&tempty[b], ((u >> 1) & 1) ^ 1, abrt)) {
            give_up();
            ok = false;
            break;
          }
          fence_after();
          const uint32_t d = tmem + b * C::kAccStride;
          for (int ks = s0; ks < s1; ++ks, ++g) {
            const int slot = g % S;
            if (!bar_wait(kF32 ? &ready[slot] : &full[slot], (g / S) & 1, abrt)) {
              give_up();
              ok = false;
              break;
            }
            fence_after();
            const uint32_t st = stages_s + slot * C::kStageBytes;
            // W block of this stage: in the stage, or resident at its K-block index
            const uint32_t wblk = kWRes ? wres_s + static_cast<uint32_t>(k0 / C::kStageK + ks) *
                                                       C::kWBlockBytes
                                        : st + kOffW;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const uint32_t acc = (ks != s0 || k != 0);
              const uint64_t w = sdesc(wblk + k * 32, 16, 1024);
              if constexpr (kF32) {
                const uint64_t ah = sdesc(st + kOffA + k * 32, 16, 1024);
                const uint64_t al = sdesc(st + kOffLo + k * 32, 16, 1024);
                mma<true>(d, ah, w, kIdWide, acc);
                mma<true>(d + kN, al, w, kIdLo, 1);
              } else {
                // K-major A: 32 bytes per K step inside the swizzled row; M-contiguous A:
                // 16 K rows of 128 bytes per step, the two 64-column halves 8 KB apart.
                const uint64_t aa = kT ? sdesc(st + kOffA + k * 2048, kTileM * 64, 1024)
                                       : sdesc(st + kOffA + k * 32, 16, 1024);
                mma<false>(d, aa, w, kIdWide, acc);
              }
            }
            issued = true;
            mma_commit(&empty[slot]);
          }
          if (!ok) break;
          mma_commit(&tfull[b]);
        }
      }
      if (!ok && issued) {  // let every issued MMA finish before the TMEM is released
        mma_commit(&drain);
        bar_wait(&drain, 0, nullptr);
      }
    }
  } else if (warp < 4) {
    // --------------------------------------------------------------------- epilogue
    uint32_t u = 0;
    bool ok = true;
    for (uint32_t w = 0; ok; ++w) {
      int it = 0;
      ok = __all_sync(0xffffffffu, next_item(w, it));
      if (!ok) {
        if (lane == 0) give_up();
        break;
      }
      __syncwarp();
      if (lane == 0) bar_arrive(&iempty[w % kItemQ]);
      if (it >= items) break;
      const int tile = it % a.tiles, ch = it / a.tiles;
      const int64_t k0 = ch * a.chunk_len;
      const int64_t k1 = a.K < k0 + a.chunk_len ? a.K : k0 + a.chunk_len;
      const int nks = static_cast<int>((k1 - k0 + C::kStageK - 1) / C::kStageK);
      float v[kN];
#pragma unroll
      for (int c = 0; c < kN; ++c) v[c] = 0.0f;
      for (int s0 = 0; s0 < nks; s0 += C::kSegStages, ++u) {
        const uint32_t b = u & 1;
        ok = __all_sync(0xffffffffu, bar_wait_patient(&tfull[b], (u >> 1) & 1, abrt));
        if (!ok) {
          if (lane == 0) give_up();
          break;
        }
        fence_after();
        const uint32_t taddr =
            tmem + (static_cast<uint32_t>(warp * 32) << 16) + b * C::kAccStride;
#pragma unroll
        for (int c = 0; c < kN; c += 16) {
          float p0[16], p1[16], p2[16];
          tmem_ld16(taddr + c, p0);
          tmem_ld16(taddr + kN + c, p1);
          if constexpr (C::kSplits == 3) tmem_ld16(taddr + 2 * kN + c, p2);
          tmem_wait_ld();
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const float corr = C::kSplits == 3 ? p1[i] + p2[i] : p1[i];
            v[c + i] += p0[i] + corr;
          }
        }
        fence_before();
        __syncwarp();
        if (lane == 0) bar_arrive(&tempty[b]);
      }
      if (!ok) break;
      const int64_t row = static_cast<int64_t>(tile) * kTileM + warp * 32 + lane;
      if (row < a.M) {
        float* o = a.out + (static_cast<int64_t>(ch) * a.M + row) * a.R;
        if ((a.R & 3) == 0) {
#pragma unroll
          for (int c = 0; c < kN; c += 4)
            if (c < a.R)
              *reinterpret_cast<float4*>(o + c) = make_float4(v[c], v[c + 1], v[c + 2], v[c + 3]);
        } else {
#pragma unroll
          for (int c = 0; c < kN; ++c)
            if (c < a.R) o[c] = v[c];
        }
      }
      if constexpr (!kT && kN <= 32) {  // (wider rows: the level runs as its own kernel)
        if (a.post_F) post_group<kN>(a, v, tile, warp, lane);
      }
    }
  } else if constexpr (kF32) {
    // ------------------------------------------------------------------- converters
    const int t = threadIdx.x - 6 * 32;  // 0..127
    uint32_t g = 0;
    bool ok = true;
    for (uint32_t w = 0; ok; ++w) {
      int it = 0;
      ok = __all_sync(0xffffffffu, next_item(w, it));
      if (!ok) {
        if (lane == 0) give_up();
        break;
      }
      __syncwarp();
      if (lane == 0) bar_arrive(&iempty[w % kItemQ]);
      if (it >= items) break;
      const int ch = it / a.tiles;
      const int64_t k0 = ch * a.chunk_len;
      const int64_t k1 = a.K < k0 + a.chunk_len ? a.K : k0 + a.chunk_len;
      const int nks = static_cast<int>((k1 - k0 + C::kStageK - 1) / C::kStageK);
      for (int ks = 0; ks < nks; ++ks, ++g) {
        const int slot = g % S;
        ok = __all_sync(0xffffffffu, bar_wait(&full[slot], (g / S) & 1, abrt));
        if (!ok) {
          if (lane == 0) give_up();
          break;
        }
        uint8_t* st = stage_ptr(slot);
        if constexpr (!kT) {
          // the tile stays as the hi part; the lo part goes to the same offset of the lo
          // tile, so it keeps the swizzled layout the TMA wrote
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int off = (t + 128 * i) * 16;
            const float4 x = *reinterpret_cast<const float4*>(st + kOffA + off);
            *reinterpret_cast<float4*>(st + kOffLo + off) =
                make_float4(tf32_rem(x.x), tf32_rem(x.y), tf32_rem(x.z), tf32_rem(x.w));
          }
        } else {
          // transpose in place: thread m reads column m of the raw rows [32 K][128 M] (plain
          // layout) into registers; once all four converter warps have read the tile (cread:
          // one arrival per warp, a bounded wait) the K-major operand rows overwrite it, 128
          // bytes (32 K values) per M row, 16-byte chunk c at chunk position c ^ (m & 7) (the
          // 128-byte swizzle): the values themselves (the hi parts) to the operand tile, the
          // lo parts to the lo tile.  (A separate raw buffer
          // would cost two of the five stages.)
          const float* raw = reinterpret_cast<const float*>(st + kOffA);
          const int m = t;
          float xv[32];
#pragma unroll
          for (int k = 0; k < 32; ++k) xv[k] = raw[k * kTileM + m];
          __syncwarp();
          if (lane == 0) bar_arrive(&cread[slot]);
          ok = __all_sync(0xffffffffu, bar_wait(&cread[slot], (g / S) & 1, abrt));
          if (!ok) {
            if (lane == 0) give_up();
            break;
          }
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const float4 h = make_float4(xv[4 * c], xv[4 * c + 1], xv[4 * c + 2], xv[4 * c + 3]);
            const int off = m * 128 + ((c ^ (m & 7)) << 4);
            *reinterpret_cast<float4*>(st + kOffA + off) = h;
            *reinterpret_cast<float4*>(st + kOffLo + off) =
                make_float4(tf32_rem(h.x), tf32_rem(h.y), tf32_rem(h.z), tf32_rem(h.w));
          }
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncwarp();
        if (lane == 0) bar_arrive(&ready[slot]);
      }
    }
  }

  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"(C::kTmemCols));
  }
  // the last CTA to leave resets the item counter for the next launch (every producer has
  // stopped fetching by then)
  if (threadIdx.x == 0 && atomicAdd(a.sched + 1, 1u) == gridDim.x - 1) {
    a.sched[0] = 0;
    a.sched[1] = 0;
  }
}

}  // namespace umma
}  // namespace ntf

namespace ntf {
namespace umma {

template <bool kT, bool kF32, int kN, bool kWRes>
cudaError_t run(const UmmaPlan& p, const Args& a, cudaStream_t st) {
  using C = Cfg<kT, kF32, kN, kWRes>;
  auto kern = k_umma<kT, kF32, kN, kWRes>;
  cudaError_t e =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmemBytes);
  if (e != cudaSuccess) return e;
  kern<<<p.grid, C::kThreads, C::kSmemBytes, st>>>(p.tx, p.tw, a);
  return cudaGetLastError();
}

// K blocks of the split table that fit in shared memory for the resident-table kernel
inline int wres_blocks(int N) { return N <= 16 ? 8 : N <= 32 ? 7 : 0; }

template <bool kF32>
cudaError_t dispatch(const UmmaPlan& p, const Args& a, cudaStream_t st) {
  if constexpr (!kF32) {
    if (p.wres) {
      switch (p.N * 2 + (p.transposed ? 1 : 0)) {
        case 32: return run<false, false, 16, true>(p, a, st);
        case 33: return run<true, false, 16, true>(p, a, st);
        case 64: return run<false, false, 32, true>(p, a, st);
        case 65: return run<true, false, 32, true>(p, a, st);
        default: return cudaErrorInvalidValue;
      }
    }
  }
  switch (p.N * 2 + (p.transposed ? 1 : 0)) {
    case 32: return run<false, kF32, 16, false>(p, a, st);
    case 33: return run<true, kF32, 16, false>(p, a, st);
    case 64: return run<false, kF32, 32, false>(p, a, st);
    case 65: return run<true, kF32, 32, false>(p, a, st);
    case 96: return run<false, kF32, 48, false>(p, a, st);
    case 97: return run<true, kF32, 48, false>(p, a, st);
    case 128: return run<false, kF32, 64, false>(p, a, st);
    case 129: return run<true, kF32, 64, false>(p, a, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace umma
}  // namespace ntf
