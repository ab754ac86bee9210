// Host side of the tensor-core contractions (kernels in umma_kernels.cuh): work split over
// persistent CTAs, TMA tensor maps of the tensor and of the split Khatri-Rao table.
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "ntf_internal.cuh"

namespace ntf {
namespace umma {
cudaError_t launch_bf16(const UmmaPlan& p, const Args& a, cudaStream_t st);
cudaError_t launch_f32(const UmmaPlan& p, const Args& a, cudaStream_t st);
}  // namespace umma

namespace {

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link to libcuda).
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    (void)cudaGetLastError();
  });
  return fn;
}

// 2-D row-major map: `inner` elements per row (contiguous), `outer` rows of `row_bytes`.
bool encode(CUtensorMap* map, CUtensorMapDataType type, const void* base, uint64_t inner,
            uint64_t outer, uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer,
            bool swizzle128) {
  const PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {inner, outer};
  const cuuint64_t strides[1] = {row_bytes};
  const cuuint32_t box[2] = {box_inner, box_outer};
  const cuuint32_t elem_strides[2] = {1, 1};
  const CUresult r =
      fn(map, type, 2, const_cast<void*>(base), dims, strides, box, elem_strides,
         CU_TENSOR_MAP_INTERLEAVE_NONE,
         swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

int umma_n(int R) { return ((R + 15) / 16) * 16; }
int64_t pad64(int64_t K) { return ((K + 63) / 64) * 64; }

}  // namespace

size_t umma_wsplit_bytes(int64_t K, int R, int dtype) {
  const int splits = dtype == NTF_BF16 ? 3 : 2;
  const int es = dtype == NTF_BF16 ? 2 : 4;
  return static_cast<size_t>(splits) * umma_n(R) * pad64(K) * es;
}

bool umma_plan(UmmaPlan* p, bool transposed, int dtype, const void* X, int64_t P, int64_t Q,
               int R, void* Wsplit, int num_sms, int64_t ld) {
  *p = UmmaPlan{};
  if (ld == 0) ld = Q;
  if (R < 1 || R > 64 || !X || !Wsplit || P < 1 || Q < 1 || ld < Q || num_sms < 1) return false;
  const bool f32 = dtype != NTF_BF16;
  const int es = f32 ? 4 : 2;
  // TMA: 16-byte aligned base and row pitch (the tensor map's extent is Q: columns Q .. ld-1
  // of a padded copy are never read)
  if (reinterpret_cast<uintptr_t>(X) % 16 != 0 || (ld * es) % 16 != 0) return false;
  const int64_t M = transposed ? Q : P, K = transposed ? P : Q;
  if (M >= (int64_t{1} << 31) || K >= (int64_t{1} << 31)) return false;
  p->transposed = transposed;
  p->f32 = f32;
  p->N = umma_n(R);
  p->splits = f32 ? 2 : 3;
  p->K_pad = pad64(K);
  const int stage_k = f32 ? 32 : 64;
  const int64_t tiles = (M + 127) / 128;
  // Persistent CTAs, one per SM, but two SMs fewer than the GPU has: the sweep runs small
  // kernels (coefficient systems, reductions) on other streams at the same time, and a CTA
  // that cannot become resident until such a kernel leaves its SM would hold back its whole
  // share of tiles.
  const int64_t ctas = num_sms > 8 ? num_sms - 2 : num_sms;
  // Fewer than four rounds of tiles: split the contraction range into chunks (multiples of
  // 64, at least 4 stages long) so that the work items, tiles x chunks, fill the grid's
  // rounds evenly.  The split minimises the contraction length that the busiest CTA covers,
  // rounds x (chunk length + 512 for an item's start-up), over at most 16 rounds; one chunk
  // where that is as good (4-way 200 x 200 x 200 x 50: 313 row tiles, 3 chunks, 939 items).
  int64_t chunks = 1, len = pad64(K);
  if (tiles < 4 * ctas) {
    int64_t best = -1;
    const int64_t cmax = std::max<int64_t>(1, std::min<int64_t>(K / 256, 16 * ctas / tiles));
    for (int64_t c = 1; c <= cmax; ++c) {
      const int64_t l = pad64((K + c - 1) / c);
      const int64_t ce = (K + l - 1) / l;
      const int64_t cost = (tiles * ce + ctas - 1) / ctas * (l + 512);
      if (best < 0 || cost < best) {
        best = cost;
        chunks = ce;
        len = l;
      }
    }
  }
  p->args.M = M;
  p->args.K = K;
  p->args.chunk_len = len;
  p->args.R = R;
  p->args.tiles = static_cast<int>(tiles);
  p->args.chunks = static_cast<int>(chunks);
  p->grid = static_cast<int>(std::min<int64_t>(tiles * chunks, ctas));
  const CUtensorMapDataType t =
      f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  const uint64_t pitch = static_cast<uint64_t>(ld) * es;
  bool ok;
  if (!transposed)  // K-major X tile: 128 rows x 128 bytes of the row
    ok = encode(&p->tx, t, X, Q, P, pitch, stage_k, 128, true);
  else if (!f32)    // M-contiguous tile halves: 64 rows (K) x 64 columns (M)
    ok = encode(&p->tx, t, X, Q, P, pitch, 64, 64, true);
  else              // raw FP32 rows for the transposing split: 32 rows (K) x 128 columns (M)
    ok = encode(&p->tx, t, X, Q, P, pitch, 128, 32, false);
  ok = ok && encode(&p->tw, t, Wsplit, p->K_pad, static_cast<uint64_t>(p->splits) * p->N,
                    p->K_pad * es, stage_k, p->splits * p->N, true);
  // BF16 with N <= 32: keep the whole split table in shared memory when it has few enough
  // 64-deep K blocks (8 for N = 16, 7 for N = 32)
  const int64_t nks_all = (K + stage_k - 1) / stage_k;
  p->wres = !f32 && ((p->N <= 16 && nks_all <= 8) || (p->N == 32 && nks_all <= 7));
  p->on = ok;
  return ok;
}

cudaError_t launch_umma(const UmmaPlan& p, float* out, int* err, unsigned* sched,
                        const int* skip, cudaStream_t st, const float* post_F, int64_t post_Ib,
                        float* post_part) {
  if (!p.on || !sched) return cudaErrorInvalidValue;
  if (post_F && (p.transposed || p.args.chunks != 1 || p.N > 32 || post_Ib < 32 || !post_part))
    return cudaErrorInvalidValue;
  umma::Args a = p.args;
  a.post_F = post_F;
  a.post_Ib = post_Ib;
  a.post_part = post_part;
  a.out = out;
  a.err = err;
  a.sched = sched;
  a.skip = skip;
  return p.f32 ? umma::launch_f32(p, a, st) : umma::launch_bf16(p, a, st);
}

}  // namespace ntf
