// One factor update of eq. (ADMM_NTF_ALS_C) followed by the projection and dual steps of
// eq. (ADMoM_NTF), repeated inner_iters times, as three launches:
//
//  k_update_system  one CTA: H = Hadamard_{m != n} Gram_m + rho I (FP64) and H^{-1} (FP64,
//                   symmetric sweep operator: Gauss-Jordan in symmetric form, the SPD
//                   counterpart of factoring H once) -- the coefficient matrix common to all
//                   rows (App. B).  Stored as FP64 and FP32.
//  k_update_rows    one warp per row: x = H^{-1}(m + rho At - Y), At = (x + Y/rho)_+,
//                   Y += rho (x - At); per-CTA partial sums of the residual norms of
//                   Sec. IV-C, of the new factor's Gram (FP64), of the fit terms
//                   <M_i, f_i>, f_i^T G f_i and of the KKT measures of the row problems
//                   (eq. KKT_NTF, gradient At G - M).  The row arithmetic is FP32 under the trace
//                   penalty policy (then cond(H) <= R + 1) and FP64 otherwise.
//  k_update_reduce  fixed-order sums of the partials: the stored Gram of the factor, the
//                   residuals, the penalty rule (Sec. IV-D) and, for the last factor of a
//                   sweep, the relative error ||X||^2 - 2<M, F> + sum_i f_i^T G f_i.
//
// Inside a sweep the reduction and the next factor's coefficient system are one kernel
// (k_update_reduce_system: its last CTA builds the system); a small set of partials is
// reduced by the rows kernel's own last CTA instead.  The last factor's reduction also
// evaluates the run's stopping rules and writes the sweep's outcome; the rows kernel of a
// factor that alone forms a contraction's Khatri-Rao operand writes that contraction's split
// table from the new rows.
#include <cmath>

#include "ntf_internal.cuh"

namespace ntf {
namespace {

constexpr int kRowWarps = 8;  // rows per CTA
constexpr int kRowThreads = kRowWarps * 32;
// Scalar partials per CTA: [0, kSumScal) are summed over CTAs -- squared norms of the
// residuals (0-4), the fit terms <M, f> and f^T G f (5, 6), the complementarity sum
// sum |At (At G - M)| (7) -- and [kSumScal, kScal) are maxima -- max(-(At G - M)) (8),
// max |At| (9), max |M| (10), max(-At) (11) -- for the KKT measures of eq. (KKT_NTF).
constexpr int kScal = 12;
constexpr int kSumScal = 8;
// The rows kernel reduces its own partials (in its last CTA) when there are at most this many
// Gram partial entries to add; larger sets go to the separate multi-CTA reduction.
constexpr int64_t kFusedReduceMax = 2048;
constexpr int kRedEntries = 32;  // packed Gram entries per CTA of the separate reduction
                                 // (256 threads, 8 per entry)

// Per-mode system slot: H^{-1} in FP64, H^{-1} and H (without rho) in FP32.
struct SysView {
  double* hinv64;
  float* hinv32;
  float* h32;
};
__host__ __device__ inline SysView sys_view(double* base, int mode, int R) {
  const int RR = R * R;
  char* p = reinterpret_cast<char*>(base) + static_cast<size_t>(mode) * RR * 16;
  SysView v;
  v.hinv64 = reinterpret_cast<double*>(p);
  v.hinv32 = reinterpret_cast<float*>(p + static_cast<size_t>(RR) * 8);
  v.h32 = reinterpret_cast<float*>(p + static_cast<size_t>(RR) * 12);
  return v;
}

struct UpdArgs {
  const double* grams;  // [N, R, R]
  double* sys;          // N system slots
  const float* M;       // [I, R]
  float* A;
  float* At;
  float* Y;
  Ctrl* ctrl;
  double* gram_part;    // [blocks, R (R + 1) / 2] packed lower triangles
  double* scal_part;    // [blocks, kScal]
  double* gram_out;     // [R, R] stored Gram of this factor
  SweepSnap* snap;      // a sweep of ntf_run: its outcome slots (host-mapped), else null
  void* wsplit;         // split Khatri-Rao table to write from the new rows (or null)
  int64_t ws_kpad;
  int ws_n, ws_bf16;
  int64_t I;
  int N, mode, R, inner, rho_policy, kr_aux, want_fit;
  int fused;            // rows kernel also reduces (last CTA)
  double mu, tau_incr, tau_decr;
  double inv_r;          // 1 / R, formed on the host (an FP64 division is slow on this GPU)
  float box_lo, box_hi;  // projection of the auxiliary: onto [box_lo, box_hi] ((.)_+: [0, inf))
  int tail_only;         // the inner iterations ran elsewhere: x, At, Y as stored, At before
  const float* t_before; // the update in t_before (the partial sums and reductions only)
};

// 1/p for p > 0: the single-precision estimate refined by two Newton-Raphson steps for
// f(y) = 1/y - p (y <- y + y (1 - p y)), each of which squares the relative error.
__device__ __forceinline__ double recip_newton(double p) {
  const float pf = static_cast<float>(p);
  if (!(pf > 1e-30f) || !(pf < 1e30f)) return 1.0 / p;
  double y = static_cast<double>(__frcp_rn(pf));
  y = fma(y, fma(-p, y, 1.0), y);
  return fma(y, fma(-p, y, 1.0), y);
}

// H = Hadamard_{m != n} Gram_m + rho I and H^{-1} by the symmetric sweep operator
// (Goodnight 1979) on every diagonal entry: sweeping pivot k with d = a_kk replaces
//   a_ij -> a_ij - a_ik a_kj / d  (i, j != k),   a_ik -> a_ik / d,   a_kk -> -1 / d,
// keeps the matrix symmetric, and after all R sweeps the matrix is -H^{-1}.  This is
// Gauss-Jordan elimination without pivoting in symmetric form: valid and stable for SPD H,
// where every pivot is a Schur-complement diagonal entry, positive exactly when H is SPD.
//
// Division-free form: the kernel holds B = c A for a tracked scalar c > 0 and applies the
// sweep to B as
//   b_ij -> 2^e (b_ij b_kk - b_ik b_kj),   b_ik -> 2^e c b_ik,   b_kk -> -2^e c^2,
//   c -> 2^e c b_kk,
// with 2^e the power of two that brings b_kk into [1, 2) (exact scaling, so the entries stay
// of the size of H); at the end H^{-1} = -B / c with the only reciprocal.  No reciprocal sits
// on the per-step dependency chain.  Every entry takes the same two FP64 instructions per
// step, 2^e fma(-u_i, u_j, b_ij g), where u is column k of B with its pivot entry replaced by
// zero and g = b_kk off row/column k, g = c on it: on row/column k one of u_i, u_j is that
// zero, and the pivot's owner has replaced its entry by -c beforehand.  (FP64 runs at a small
// fraction of the FP32 rate on this GPU, and a warp whose lanes took different branches
// would issue each branch's FP64 instructions in turn, so operands are selected, not
// branched on.)  Only the lower triangle is kept, in registers (S packed entries per thread);
// u, b_kk and c are published through shared memory (double-buffered, one barrier per step).
constexpr int kSysThreads = 256;

// x 2^e for the scale factor of a pivot, e in [-1023, 1022], on the exponent field alone
// (integer instructions and selects: on this GPU every FP64 instruction, even one whose
// predicate is off, holds the small FP64 unit, and a library scaling call on the rare path
// was issued with every entry).  Exact when x and the result are normal numbers; zero,
// subnormals, infinities and NaN stay what they are; a result below the normal range becomes
// a signed zero and one above it a signed infinity (for an SPD matrix scaled by its pivots
// neither happens short of entries 10^300 apart).
__device__ __forceinline__ double scale_pow2(double x, int e) {
  const int hi = __double2hiint(x);
  const int lo = __double2loint(x);
  const int ex = (hi >> 20) & 0x7FF;
  const int ne = ex + e;
  const int sign = hi & static_cast<int>(0x80000000u);
  int rhi = static_cast<int>(static_cast<unsigned>(hi) + (static_cast<unsigned>(e) << 20));
  int rlo = lo;
  if (ex == 0 || ex == 0x7FF) {  // zero, subnormal, infinity, NaN: unchanged
    rhi = hi;
  } else if (ne <= 0) {          // below the normal range: signed zero
    rhi = sign;
    rlo = 0;
  } else if (ne >= 0x7FF) {      // above it: signed infinity
    rhi = sign | 0x7FF00000;
    rlo = 0;
  }
  return __hiloint2double(rhi, rlo);
}

template <int S, int NT>
__device__ void system_body(const UpdArgs& a) {
  __shared__ double s_col[2][64];  // u: column k of B, zero at the pivot
  __shared__ double s_piv[2], s_c[2];
  __shared__ double s_red[NT / 32], s_gmax[NT / 32];
  const int R = a.R, RR = R * R, T = R * (R + 1) / 2;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const SysView sv = sys_view(a.sys, a.mode, R);
  double v[S];
  int ii[S], jj[S];
  double tr = 0.0, gmax = 0.0;
#pragma unroll
  for (int q = 0; q < S; ++q) {
    const int p = tid + NT * q;
    int i = static_cast<int>((sqrtf(8.0f * p + 1.0f) - 1.0f) * 0.5f);
    while (i * (i + 1) / 2 > p) --i;
    while ((i + 1) * (i + 2) / 2 <= p) ++i;
    const int j = p - i * (i + 1) / 2;
    ii[q] = p < T ? i : -1;
    jj[q] = p < T ? j : -1;
    double h = 0.0;
    if (p < T) {
      double g[kMaxOrder];  // loads first, then the product
#pragma unroll
      for (int m = 0; m < kMaxOrder; ++m)
        g[m] = m < a.N && m != a.mode ? a.grams[m * RR + i * R + j] : 1.0;
      h = g[0];
#pragma unroll
      for (int m = 1; m < kMaxOrder; ++m) h *= g[m];
      sv.h32[i * R + j] = static_cast<float>(h);
      sv.h32[j * R + i] = static_cast<float>(h);
      if (i == j) tr += h;
      gmax = fmax(gmax, fabs(h));
    }
    v[q] = h;
  }
  for (int off = 16; off > 0; off >>= 1) {
    tr += __shfl_xor_sync(0xffffffffu, tr, off);
    gmax = fmax(gmax, __shfl_xor_sync(0xffffffffu, gmax, off));
  }
  if (lane == 0) {
    s_red[warp] = tr;
    s_gmax[warp] = gmax;
  }
  __syncthreads();
  if (tid == 0) {
    double g = 0.0;
    for (int w = 0; w < NT / 32; ++w) g = fmax(g, s_gmax[w]);
    a.ctrl->kkt[a.mode][3] = g;  // max |G|: scale of the KKT measures
  }
  double rho;
  if (a.rho_policy == NTF_RHO_TRACE) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) t += s_red[w];
    rho = t * a.inv_r;
  } else {
    rho = a.ctrl->rho[a.mode];
  }
  bool fail = !(rho > 0.0) || !isfinite(rho);
#pragma unroll
  for (int q = 0; q < S; ++q)
    if (ii[q] >= 0 && ii[q] == jj[q]) v[q] += rho;

  double c = 1.0, piv = 1.0;  // c and b_kk of the current step (the same in every thread)
  int e = 0;
  for (int k = 0; k < R && !fail; ++k) {
    const int b = k & 1;
#pragma unroll
    for (int q = 0; q < S; ++q) {  // publish u (column k); the pivot's owner also b_kk, c
      const int i = ii[q], j = jj[q];
      if (i == k || j == k) {
        const bool pivot = i == j;
        s_col[b][i + j - k] = pivot ? 0.0 : v[q];
        if (pivot) {
          const double ck = k ? scale_pow2(c * piv, e) : 1.0;  // c after the previous step
          s_piv[b] = v[q];
          s_c[b] = ck;
          v[q] = -ck;
        }
      }
    }
    __syncthreads();  // one barrier per step: the next step writes the other buffers
    piv = s_piv[b];
    c = s_c[b];
    const int pex = __double2hiint(piv) >> 20;  // negative when the sign bit is set
    if (static_cast<unsigned>(pex - 1) >= 0x7FEu) {  // not SPD (or not a normal number)
      fail = true;  // the same shared value in every thread: a uniform exit
      break;
    }
    e = 1023 - pex;  // b_kk 2^e in [1, 2)
#pragma unroll
    for (int q = 0; q < S; ++q) {
      const int i = ii[q], j = jj[q];
      if (i < 0) continue;
      const double g = i == k || j == k ? c : piv;
      v[q] = scale_pow2(fma(-s_col[b][i], s_col[b][j], v[q] * g), e);
    }
  }
  if (fail) {  // uniform
    if (tid == 0) {
      a.ctrl->bad[a.mode] = 1;
      atomicOr(&a.ctrl->status, kStNotSpd);
    }
    return;
  }
  const double nic = -recip_newton(scale_pow2(c * piv, e));  // H^{-1} = -B / c
#pragma unroll
  for (int q = 0; q < S; ++q) {
    const int i = ii[q], j = jj[q];
    if (i < 0) continue;
    const double h = v[q] * nic;
    sv.hinv64[i * R + j] = h;
    sv.hinv64[j * R + i] = h;
    sv.hinv32[i * R + j] = static_cast<float>(h);
    sv.hinv32[j * R + i] = static_cast<float>(h);
  }
  if (tid == 0) {
    a.ctrl->bad[a.mode] = 0;
    a.ctrl->stats[a.mode][5] = rho;
  }
}

// Trace policy: H = Hadamard_{m != n} Gram_m + rho I with rho = trace(G)/R, so that
// cond(H) <= R + 1 (the eigenvalues of G lie in [0, trace G]).  H is factored once in FP64
// (App. B) as H = L D L^T by right-looking elimination, fraction-free: the trailing part is
// kept as B = c A for a tracked scalar c > 0 and step k maps
//   b_ij -> 2^e (b_ij b_kk - b_ik b_jk)  (i >= j > k),   c -> 2^e c b_kk,
// with 2^e the power of two that brings b_kk into [1, 2) (exact), so no reciprocal lies on
// the chain of dependent steps.  Column k is final after step k: l_ik = b_ik / b_kk and
// d_k = b_kk / c (c of step k cancels in l).  The lower triangle is packed column by column,
// so the trailing part of step k is a suffix of the packing and the threads that still have
// work at a step fill whole warps (FP64 instructions issue per warp at a small fraction of
// the FP32 rate on this GPU, so partly idle warps would cost as much as busy ones).  A pivot
// that is not a positive normal number reports NOT_SPD, where Cholesky would fail.
// H^{-1} = L^{-T} D^{-1} L^{-1} is then formed in FP32 from the FP64 factor: W = L^{-1} by
// forward substitution (one warp per set of columns, shuffles, no block barriers) and
// H^{-1}_ij = sum_{k >= max(i, j)} W_ki W_kj / d_k; with cond(H) <= R + 1 its error is a few
// FP32 roundings, the precision the rows kernel applies it in.  Only the FP32 inverse is
// written (the rows kernel of this policy reads nothing else).
__device__ __forceinline__ int col_start(int j, int R) { return j * R - j * (j - 1) / 2; }

// Largest rank whose packed lower triangle fits in n entries (at most kMaxRank).
__host__ __device__ constexpr int ldl_max_rank(int n) {
  int r = 0;
  while (r < kMaxRank && (r + 1) * (r + 2) / 2 <= n) ++r;
  return r;
}

template <int S, int NT>
__device__ void system_ldl(const UpdArgs& a) {
  constexpr int kRmax = ldl_max_rank(S * NT);
  constexpr int kVBuf = kRmax * (kRmax | 1);  // V with an odd row stride (R | 1 <= kRmax | 1)
  constexpr int kBuf = S * NT > kVBuf ? S * NT : kVBuf;
  __shared__ double s_col[2][kMaxRank];  // column k + 1 of B, published during step k
  __shared__ double s_piv[2], s_c[2];
  __shared__ double s_rho;
  __shared__ unsigned long long s_gmax[NT / 32];
  __shared__ double s_pk[kMaxRank], s_ck[kMaxRank];  // b_kk and c of every step
  __shared__ float s_l[kBuf];  // L (packed by column), then V = D^{-1/2} L^{-1} (by rows)
  __shared__ float s_dinv[kMaxRank];
  const int R = a.R, RR = R * R, T = R * (R + 1) / 2;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const SysView sv = sys_view(a.sys, a.mode, R);
  // FP64 instructions are scarce on this GPU (a small fraction of the FP32 rate), so the
  // prologue spends them only on the Hadamard products: |h| maxima on the bit patterns (the
  // order of non-negative doubles), the trace by one warp from the diagonals.
  // Slot q of thread t holds packed entry p = T - 1 - (t + NT q), the packing read backwards:
  // the trailing part of step k (p >= col_start(k + 1)) is then a prefix of the slots, and a
  // step runs only the slots that hold some of it (a count that is the same in every thread)
  // instead of issuing every slot's FP64 instructions under a predicate.
  const int nslot = (T + NT - 1) / NT;  // slots that hold entries
  double v[S];
  int ii[S], jj[S];
  unsigned long long gmax = 0;
#pragma unroll
  for (int q = 0; q < S; ++q) {
    const int p = T - 1 - (tid + NT * q);  // negative: no entry
    int j = -1, i = -1;
    if (p >= 0) {  // column j of the packing holds rows j .. R-1: col_start(j) <= p
      const float b2 = 2.0f * R + 1.0f;
      j = static_cast<int>((b2 - sqrtf(b2 * b2 - 8.0f * p)) * 0.5f);
      j = j < 0 ? 0 : j > R - 1 ? R - 1 : j;
      while (j > 0 && col_start(j, R) > p) --j;
      while (j + 1 < R && col_start(j + 1, R) <= p) ++j;
      i = j + (p - col_start(j, R));
    }
    ii[q] = i;
    jj[q] = j;
    double h = 0.0;
    if (p >= 0) {
      // the other factors' Grams: factors o = k (k < mode) or k + 1, k = 0 .. N-2; loads
      // first, then the N - 2 products
      const int e = i * R + j;
      const double g0 = a.grams[(0 < a.mode ? 0 : 1) * RR + e];
      const double g1 = a.grams[(1 < a.mode ? 1 : 2) * RR + e];
      const double g2 = a.N > 3 ? a.grams[(2 < a.mode ? 2 : 3) * RR + e] : 1.0;
      h = g0 * g1;
      if (a.N > 3) h *= g2;
      const float hf = static_cast<float>(h);
      sv.h32[i * R + j] = hf;
      sv.h32[j * R + i] = hf;
      const unsigned long long bits =
          static_cast<unsigned long long>(__double_as_longlong(h)) & 0x7FFFFFFFFFFFFFFFull;
      gmax = bits > gmax ? bits : gmax;
    }
    v[q] = h;
  }
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, gmax, off);
    gmax = o > gmax ? o : gmax;
  }
  if (lane == 0) s_gmax[warp] = gmax;
  if (warp == 0) {  // trace(G) = sum_j prod_m Gram_m[j, j]
    double t = 0.0;
    for (int j = lane; j < R; j += 32) {
      double d = 1.0;
      for (int m = 0; m < a.N; ++m)
        if (m != a.mode) d *= a.grams[m * RR + j * R + j];
      t += d;
    }
    for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
    if (lane == 0) s_rho = t * a.inv_r;
  }
  __syncthreads();
  const double rho = s_rho;
  if (tid == 0) {
    unsigned long long g = 0;
    for (int w = 0; w < NT / 32; ++w) g = s_gmax[w] > g ? s_gmax[w] : g;
    a.ctrl->kkt[a.mode][3] = __longlong_as_double(static_cast<long long>(g));  // max |G|
  }
  bool fail = !(rho > 0.0) || !isfinite(rho);
#pragma unroll
  for (int q = 0; q < S; ++q) {
    if (ii[q] >= 0 && ii[q] == jj[q]) v[q] += rho;
    if (jj[q] == 0) {  // publish column 0 (c = 1)
      s_col[0][ii[q]] = v[q];
      if (ii[q] == 0) {
        s_piv[0] = v[q];
        s_c[0] = 1.0;
      }
    }
  }
  __syncthreads();
  for (int k = 0; k < R && !fail; ++k) {
    const int b = k & 1;
    const double piv = s_piv[b], c = s_c[b];
    const int pex = __double2hiint(piv) >> 20;  // negative when the sign bit is set
    if (static_cast<unsigned>(pex - 1) >= 0x7FEu) {  // not SPD (or not a normal number)
      fail = true;  // the same shared value in every thread: a uniform exit
      break;
    }
    if (tid == 0) {
      s_pk[k] = piv;
      s_ck[k] = c;
    }
    const int e = 1023 - pex;   // b_kk 2^e in [1, 2)
    const int first = col_start(k + 1, R);  // the trailing part is p >= first: slots
    const int nact = (T - first + NT - 1) / NT;  // t + NT q < T - first, the first nact
#pragma unroll
    for (int q = 0; q < S; ++q) {
      if (q >= nact) break;                       // the same in every thread
      if (tid + NT * q >= T - first) continue;  // only in the last of them
      const int i = ii[q], j = jj[q];
      // b_ij b_kk - b_ik b_kj with the product of the loaded column entries formed here: a
      // product of register values alone (b_ij b_kk) would be computed ahead of the slot
      // test for every slot, each one a full FP64 instruction
      const double nv = scale_pow2(fma(v[q], piv, -(s_col[b][i] * s_col[b][j])), e);
      v[q] = nv;
      if (j == k + 1) {  // publish column k + 1 for the next step
        s_col[b ^ 1][i] = nv;
        if (i == j) {
          s_piv[b ^ 1] = nv;
          s_c[b ^ 1] = scale_pow2(c * piv, e);
        }
      }
    }
    __syncthreads();  // one barrier per step: the next step reads the other buffers
  }
  if (fail) {  // uniform
    if (tid == 0) {
      a.ctrl->bad[a.mode] = 1;
      atomicOr(&a.ctrl->status, kStNotSpd);
    }
    return;
  }
  // L (unit lower, FP32) and D^{-1}: l_ij = b_ij / b_jj, 1/d_j = c_j / b_jj
  if (tid < R) {
    const double rp = recip_newton(s_pk[tid]);
    s_pk[tid] = rp;
    s_dinv[tid] = static_cast<float>(s_ck[tid] * rp);
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < S; ++q) {
    if (q >= nslot) break;
    const int i = ii[q], j = jj[q];
    if (i < 0) continue;
    s_l[T - 1 - (tid + NT * q)] = i == j ? 1.0f : static_cast<float>(v[q] * s_pk[j]);
  }
  __syncthreads();
  // W = L^{-1}: warp w forms the columns j = w, w + NT/32, ...; lane l holds rows l, l + 32
  constexpr int kCols = kMaxRank / (NT / 32);
  float w0[kCols], w1[kCols];
#pragma unroll
  for (int cc = 0; cc < kCols; ++cc) {
    const int j = warp + (NT / 32) * cc;
    w0[cc] = lane == j ? 1.0f : 0.0f;
    w1[cc] = lane + 32 == j ? 1.0f : 0.0f;
  }
  for (int k = 0; k + 1 < R; ++k) {
    const int ck = col_start(k, R) - k;  // s_l[ck + i] = L_ik
    const float l0 = lane > k && lane < R ? s_l[ck + lane] : 0.0f;
    const float l1 = lane + 32 > k && lane + 32 < R ? s_l[ck + lane + 32] : 0.0f;
    // every column, without a test: for j > k the entry w_kj is still zero and the update
    // changes nothing, and columns j >= R are never stored; branch-free, the columns'
    // shuffles and multiply-adds interleave
#pragma unroll
    for (int cc = 0; cc < kCols; ++cc) {
      const float y = __shfl_sync(0xffffffffu, k < 32 ? w0[cc] : w1[cc], k & 31);
      w0[cc] = fmaf(-l0, y, w0[cc]);
      w1[cc] = fmaf(-l1, y, w1[cc]);
    }
  }
  __syncthreads();  // every warp has read L
  // V = D^{-1/2} W by rows (row k at k vs; vs = R | 1 is odd, so a warp's column store and
  // its reads of a row's consecutive entries are free of bank conflicts); H^{-1} = V^T V
  const int vs = R | 1;
  const float d0 = lane < R ? sqrtf(s_dinv[lane]) : 0.0f;
  const float d1 = lane + 32 < R ? sqrtf(s_dinv[lane + 32]) : 0.0f;
#pragma unroll
  for (int cc = 0; cc < kCols; ++cc) {
    const int j = warp + (NT / 32) * cc;
    if (j >= R) continue;
    if (lane < R) s_l[lane * vs + j] = w0[cc] * d0;
    if (lane + 32 < R) s_l[(lane + 32) * vs + j] = w1[cc] * d1;
  }
  __syncthreads();
  // H^{-1}_ij = sum_{k >= i} V_ki V_kj (i >= j; V_ki = 0 for k < i): the lanes of a warp hold
  // consecutive i of one column j, so V_ki is a contiguous read and V_kj a broadcast
#pragma unroll
  for (int q = 0; q < S; ++q) {
    if (q >= nslot) break;
    const int i = ii[q], j = jj[q];
    if (i < 0) continue;
    float acc0 = 0.0f, acc1 = 0.0f;
    int k = i;
    for (; k + 1 < R; k += 2) {
      acc0 = fmaf(s_l[k * vs + i], s_l[k * vs + j], acc0);
      acc1 = fmaf(s_l[(k + 1) * vs + i], s_l[(k + 1) * vs + j], acc1);
    }
    if (k < R) acc0 = fmaf(s_l[k * vs + i], s_l[k * vs + j], acc0);
    const float h = acc0 + acc1;
    sv.hinv32[i * R + j] = h;
    sv.hinv32[j * R + i] = h;
  }
  if (tid == 0) {
    a.ctrl->bad[a.mode] = 0;
    a.ctrl->stats[a.mode][5] = rho;
  }
}

// The coefficient system of a factor update: the FP64 factorization above under the trace
// policy for R >= kLdlMinRank, the FP64 sweep operator otherwise (under the other policies the
// rows then run in FP64 from its FP64 inverse).  Measured per launch on GB300 (alone): sweep
// operator R = 20: 13.5 us, R = 32: 34 us, R = 40: 48 us; LDL^T R = 32: 26 us, R = 50: 51 us,
// R = 64: 83 us.
constexpr int kLdlMinRank = 28;
template <int S, int NT>
__device__ __forceinline__ void system_any(const UpdArgs& a) {
  if constexpr (S >= 2) {  // R >= kLdlMinRank takes at least two slots per thread
    if (a.rho_policy == NTF_RHO_TRACE && a.R >= kLdlMinRank) {
      system_ldl<S, NT>(a);
      return;
    }
  }
  system_body<S, NT>(a);
}

__device__ void update_reduce_cta(const UpdArgs& a, int nblocks);

// (r, s), r >= s, of packed lower-triangle entry e = r (r + 1) / 2 + s.
__device__ __forceinline__ void tri_index(int e, int& r, int& s) {
  int i = static_cast<int>((sqrtf(8.0f * e + 1.0f) - 1.0f) * 0.5f);
  while (i * (i + 1) / 2 > e) --i;
  while ((i + 1) * (i + 2) / 2 <= e) ++i;
  r = i;
  s = e - i * (i + 1) / 2;
}

// End of a rows CTA: the CTA's scalar partials (per-warp values part[] in registers) and its
// share of the new Gram (packed lower triangle; FP64 accumulation of products of the stored
// FP32 values, each exact in FP64) from frow [kRowWarps][ld] (zero for absent rows; FP64
// copies of the FP32 values, or the FP32 values themselves); then, when the reduction is
// fused, the last CTA reduces.
__device__ void update_reduce_cta(const UpdArgs& a, int nblocks);

template <typename F>
__device__ __forceinline__ void rows_cta_tail(const UpdArgs& a, float (&part)[kScal],
                                              const F* frow, int ld,
                                              double (*red)[kScal]) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int R = a.R, T = R * (R + 1) / 2;
#pragma unroll
  for (int q = 0; q < kScal; ++q)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const float o = __shfl_xor_sync(0xffffffffu, part[q], off);
      part[q] = q < kSumScal ? part[q] + o : fmaxf(part[q], o);
    }
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < kScal; ++q) red[warp][q] = part[q];
  __syncthreads();
  if (tid < kScal) {
    double v = 0.0;  // maxima: every entry is >= 0 (the measures are clamped at zero)
    for (int w = 0; w < kRowWarps; ++w)
      v = tid < kSumScal ? v + red[w][tid] : fmax(v, red[w][tid]);
    a.scal_part[blockIdx.x * kScal + tid] = v;
  }
  double* gp = a.gram_part + static_cast<int64_t>(blockIdx.x) * T;
  for (int e = tid; e < T; e += kRowThreads) {
    int r, c;
    tri_index(e, r, c);
    double g0 = 0.0, g1 = 0.0;
#pragma unroll
    for (int w = 0; w < kRowWarps; w += 2) {
      g0 = fma(static_cast<double>(frow[w * ld + r]), static_cast<double>(frow[w * ld + c]), g0);
      g1 = fma(static_cast<double>(frow[(w + 1) * ld + r]),
               static_cast<double>(frow[(w + 1) * ld + c]), g1);
    }
    gp[e] = g0 + g1;
  }
  if (!a.fused) return;
  // the last CTA to finish sums every CTA's partials (fixed order, so the result does not
  // depend on which CTA that is) and resets the counter for the next launch
  __shared__ int s_last;
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = atomicAdd(&a.ctrl->red_count[a.mode], 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  update_reduce_cta(a, gridDim.x);
  if (tid == 0) {
    a.ctrl->red_count[a.mode] = 0;
    // every CTA of this kernel has read stop by now
    if (a.snap && a.want_fit) a.ctrl->stop = a.ctrl->stop_next;
  }
}

template <int S>
__global__ void __launch_bounds__(kSysThreads) k_update_system(UpdArgs a) {
  if (a.ctrl->stop) return;  // the run has stopped
  system_any<S, kSysThreads>(a);
}

// Rows for R <= 32.  Real = float (trace policy) or double.  One warp per row, lane j owns
// element j and holds column j of H^{-1} (= row j: symmetric) in registers for the whole
// update; x = H^{-1} v takes v_k from lane k by shuffles.  kR = R rounded up to a multiple of
// 4 fixes the loop lengths at compile time (the padding lanes and columns hold zeros).
// Register cap of the FP32 rows kernel: the factor updates run while a persistent
// contraction CTA (6 warps, 144 registers each at rank <= 32) holds each SM, and a rows CTA
// (8 warps, two on each of the SM's four schedulers) shares an SM with it only if two of its
// warps fit in what the contraction's two warps leave of a scheduler's 16384 registers:
// 2 x 32 x 112 + 2 x 32 x 144 = 16384.  (The FP64 rows of the other penalty policies spill at
// that cap and keep their registers.)
template <typename Real>
constexpr int kRows32MaxRegs = sizeof(Real) == 4 ? 112 : 168;

template <typename Real, int kR>
__global__ void __maxnreg__(kRows32MaxRegs<Real>) k_update_rows32(UpdArgs a) {
  __shared__ double frow[kRowWarps][32];  // FP64 copies: one conversion per element
  __shared__ double red[kRowWarps][kScal];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int R = a.R;
  const bool h = lane < R;
  const SysView sv = sys_view(a.sys, a.mode, R);
  // every load is issued before the status test, so that their latencies overlap (the
  // system slot and the rows are valid memory either way)
  const int bad = a.ctrl->bad[a.mode] | a.ctrl->stop;
  Real hc[kR];
  float gc[kR];  // column of the FP32 coefficient matrix G (no rho): fit and KKT terms
#pragma unroll
  for (int k = 0; k < kR; ++k) {
    Real v = 0;
    float gv = 0.0f;
    if (k < R && h) {
      if constexpr (sizeof(Real) == 4) v = __ldg(sv.hinv32 + k * R + lane);
      else v = __ldg(sv.hinv64 + k * R + lane);
      gv = __ldg(sv.h32 + k * R + lane);
    }
    hc[k] = v;
    gc[k] = gv;
  }
  const Real rho = static_cast<Real>(a.ctrl->stats[a.mode][5]);
  const int64_t row = static_cast<int64_t>(blockIdx.x) * kRowWarps + warp;
  const bool live = row < a.I && h;
  const int64_t idx = row * R + lane;
  const Real m = live ? static_cast<Real>(a.M[idx]) : Real(0);
  Real t = live ? static_cast<Real>(a.At[idx]) : Real(0);
  Real y = live ? static_cast<Real>(a.Y[idx]) : Real(0);
  const bool tail = a.tail_only != 0;
  const Real x_st = tail && live ? static_cast<Real>(a.A[idx]) : Real(0);
  const Real t_st = tail && live ? static_cast<Real>(a.t_before[idx]) : t;
  if (bad) return;  // uniform: the system of this factor failed, or the run has stopped; the
                    // state is kept
  const Real rinv = Real(1) / rho;
  const Real lo = a.box_lo, hi = a.box_hi;
  float part[kScal] = {};
  float f = 0.0f;
  if (row < a.I) {
    const Real t_in = t_st;
    Real x = x_st;
    for (int it = 0; it < (tail ? 0 : a.inner); ++it) {
      const Real v = m + rho * t - y;  // zero in the padding lanes
      Real p0 = 0, p1 = 0, p2 = 0, p3 = 0;
#pragma unroll
      for (int k = 0; k < kR; k += 4) {
        p0 = fma(hc[k], __shfl_sync(0xffffffffu, v, k), p0);
        p1 = fma(hc[k + 1], __shfl_sync(0xffffffffu, v, k + 1), p1);
        p2 = fma(hc[k + 2], __shfl_sync(0xffffffffu, v, k + 2), p2);
        p3 = fma(hc[k + 3], __shfl_sync(0xffffffffu, v, k + 3), p3);
      }
      x = h ? (p0 + p1) + (p2 + p3) : Real(0);
      const Real n = fmin(fmax(lo, x + y * rinv), hi);
      y += rho * (x - n);
      t = n;
    }
    if (!h) x = t = y = 0;
    const float fx = static_cast<float>(x), ft = static_cast<float>(t);
    if (h) {
      a.A[idx] = fx;
      a.At[idx] = ft;
      a.Y[idx] = static_cast<float>(y);
    }
    part[0] = static_cast<float>((x - t) * (x - t));
    part[1] = static_cast<float>((t - t_in) * (t - t_in));
    part[2] = static_cast<float>(x * x);
    part[3] = static_cast<float>(t * t);
    part[4] = static_cast<float>(y * y);
    // the factor that feeds the next Khatri-Rao products, as stored (FP32)
    f = a.kr_aux ? ft : fx;
    if (a.wsplit && h)  // its entry (row, lane) of the next contraction's split table
      split_store(a.wsplit, static_cast<int64_t>(a.ws_n) * a.ws_kpad,
                  static_cast<int64_t>(lane) * a.ws_kpad + row, f, a.ws_bf16);
    float g = 0.0f;  // (G f)_j with the FP32 coefficient matrix (no rho)
    if (a.want_fit) {
      part[5] = static_cast<float>(m) * f;
#pragma unroll
      for (int k = 0; k < kR; ++k) g = fmaf(gc[k], __shfl_sync(0xffffffffu, f, k), g);
      part[6] = f * g;
    }
    // KKT of the row problem min_{x >= 0} 1/2 x^T G x - m^T x at x = At (eq. KKT_NTF):
    // gradient (G At)_j - m_j; (G At)_j is the fit's (G f)_j when f = At
    float gt = g;
    if (!(a.want_fit && a.kr_aux)) {
      gt = 0.0f;
#pragma unroll
      for (int k = 0; k < kR; ++k) gt = fmaf(gc[k], __shfl_sync(0xffffffffu, ft, k), gt);
    }
    if (h) {
      const float gr = gt - static_cast<float>(m);
      part[7] = fabsf(ft * gr);
      part[8] = fmaxf(0.0f, -gr);
      part[9] = fabsf(ft);
      part[10] = fabsf(static_cast<float>(m));
      part[11] = fmaxf(0.0f, -ft);
    }
  }
  frow[warp][lane] = h ? static_cast<double>(f) : 0.0;
  rows_cta_tail(a, part, &frow[0][0], 32, red);
}

// Rows for any R <= 64.  Real = float (trace policy) or double.  One warp per row, lanes own
// elements lane and lane + 32; v and f are broadcast through a per-warp shared buffer.
template <typename Real>
__global__ void __launch_bounds__(kRowThreads) k_update_rows(UpdArgs a) {
  extern __shared__ double shd[];
  const int R = a.R, RR = R * R;
  Real* Hi = reinterpret_cast<Real*>(shd);                       // [RR] H^{-1}
  float* Hf = reinterpret_cast<float*>(Hi + RR);                 // [RR] H (fit and KKT)
  Real* vbuf = reinterpret_cast<Real*>(shd + ((RR * sizeof(Real) + RR * 4 + 15) / 16) * 2);
  float* frow = reinterpret_cast<float*>(vbuf + kRowWarps * 64); // [kRowWarps][64]
  __shared__ double red[kRowWarps][kScal];
  if (a.ctrl->bad[a.mode] || a.ctrl->stop) return;  // uniform
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const SysView sv = sys_view(a.sys, a.mode, R);
  for (int idx = tid; idx < RR; idx += kRowThreads) {
    if constexpr (sizeof(Real) == 4) Hi[idx] = sv.hinv32[idx];
    else Hi[idx] = sv.hinv64[idx];
    Hf[idx] = sv.h32[idx];
  }
  __syncthreads();
  const Real rho = static_cast<Real>(a.ctrl->stats[a.mode][5]);
  const Real rinv = Real(1) / rho;
  const int64_t row = static_cast<int64_t>(blockIdx.x) * kRowWarps + warp;
  float part[kScal] = {};
  const int j0 = lane, j1 = lane + 32;
  const bool h0 = j0 < R, h1 = j1 < R;
  Real* vb = vbuf + warp * 64;
  float* fr = frow + warp * 64;
  if (row < a.I) {
    const int64_t base = row * R;
    const Real m0 = h0 ? a.M[base + j0] : 0, m1 = h1 ? a.M[base + j1] : 0;
    Real t0 = h0 ? a.At[base + j0] : 0, t1 = h1 ? a.At[base + j1] : 0;
    Real y0 = h0 ? a.Y[base + j0] : 0, y1 = h1 ? a.Y[base + j1] : 0;
    const bool tail = a.tail_only != 0;
    const Real s0 = tail && h0 ? a.t_before[base + j0] : t0;
    const Real s1 = tail && h1 ? a.t_before[base + j1] : t1;
    Real x0 = tail && h0 ? a.A[base + j0] : 0, x1 = tail && h1 ? a.A[base + j1] : 0;
    const Real lo = a.box_lo, hi = a.box_hi;
    for (int it = 0; it < (tail ? 0 : a.inner); ++it) {
      if (h0) vb[j0] = m0 + rho * t0 - y0;
      if (h1) vb[j1] = m1 + rho * t1 - y1;
      __syncwarp();
      // x = H^{-1} v; H^{-1} is symmetric, so lane j reads row k (consecutive addresses)
      Real p0 = 0, q0 = 0, p1 = 0, q1 = 0;
      int k = 0;
      for (; k + 1 < R; k += 2) {
        const Real va = vb[k], vc = vb[k + 1];
        if (h0) {
          p0 = fma(Hi[k * R + j0], va, p0);
          q0 = fma(Hi[(k + 1) * R + j0], vc, q0);
        }
        if (h1) {
          p1 = fma(Hi[k * R + j1], va, p1);
          q1 = fma(Hi[(k + 1) * R + j1], vc, q1);
        }
      }
      if (k < R) {
        const Real va = vb[k];
        if (h0) p0 = fma(Hi[k * R + j0], va, p0);
        if (h1) p1 = fma(Hi[k * R + j1], va, p1);
      }
      __syncwarp();
      x0 = p0 + q0;
      x1 = p1 + q1;
      const Real n0 = fmin(fmax(lo, x0 + y0 * rinv), hi);
      const Real n1 = fmin(fmax(lo, x1 + y1 * rinv), hi);
      y0 += rho * (x0 - n0);
      y1 += rho * (x1 - n1);
      t0 = n0;
      t1 = n1;
    }
    if (!h0) { x0 = t0 = y0 = 0; }
    if (!h1) { x1 = t1 = y1 = 0; }
    const float fx0 = static_cast<float>(x0), fx1 = static_cast<float>(x1);
    const float ft0 = static_cast<float>(t0), ft1 = static_cast<float>(t1);
    if (h0) {
      a.A[base + j0] = fx0;
      a.At[base + j0] = ft0;
      a.Y[base + j0] = static_cast<float>(y0);
    }
    if (h1) {
      a.A[base + j1] = fx1;
      a.At[base + j1] = ft1;
      a.Y[base + j1] = static_cast<float>(y1);
    }
    part[0] = static_cast<float>((x0 - t0) * (x0 - t0) + (x1 - t1) * (x1 - t1));
    part[1] = static_cast<float>((t0 - s0) * (t0 - s0) + (t1 - s1) * (t1 - s1));
    part[2] = static_cast<float>(x0 * x0 + x1 * x1);
    part[3] = static_cast<float>(t0 * t0 + t1 * t1);
    part[4] = static_cast<float>(y0 * y0 + y1 * y1);
    // the factor that feeds the next Khatri-Rao products, as stored (FP32)
    const float f0 = a.kr_aux ? ft0 : fx0, f1 = a.kr_aux ? ft1 : fx1;
    if (h0) fr[j0] = f0;
    if (h1) fr[j1] = f1;
    if (a.wsplit) {  // entries (row, j) of the next contraction's split table
      const int64_t nt = static_cast<int64_t>(a.ws_n) * a.ws_kpad;
      if (h0) split_store(a.wsplit, nt, static_cast<int64_t>(j0) * a.ws_kpad + row, f0, a.ws_bf16);
      if (h1) split_store(a.wsplit, nt, static_cast<int64_t>(j1) * a.ws_kpad + row, f1, a.ws_bf16);
    }
    float g0 = 0.0f, g1 = 0.0f;  // (G f)_j with the FP32 coefficient matrix (no rho)
    __syncwarp();
    if (a.want_fit) {
      part[5] = static_cast<float>(m0) * f0 + static_cast<float>(m1) * f1;
      for (int kk = 0; kk < R; ++kk) {
        const float fk = fr[kk];
        if (h0) g0 = fmaf(Hf[kk * R + j0], fk, g0);
        if (h1) g1 = fmaf(Hf[kk * R + j1], fk, g1);
      }
      part[6] = f0 * g0 + f1 * g1;
    }
    // KKT of the row problem at x = At (eq. KKT_NTF): gradient (G At)_j - m_j
    if (!(a.want_fit && a.kr_aux)) {
      float* tb = reinterpret_cast<float*>(vb);  // this warp's v buffer is free now
      __syncwarp();
      if (h0) tb[j0] = ft0;
      if (h1) tb[j1] = ft1;
      __syncwarp();
      g0 = g1 = 0.0f;
      for (int kk = 0; kk < R; ++kk) {
        const float tk = tb[kk];
        if (h0) g0 = fmaf(Hf[kk * R + j0], tk, g0);
        if (h1) g1 = fmaf(Hf[kk * R + j1], tk, g1);
      }
      __syncwarp();
    }
    const float gr0 = h0 ? g0 - static_cast<float>(m0) : 0.0f;
    const float gr1 = h1 ? g1 - static_cast<float>(m1) : 0.0f;
    part[7] = fabsf(ft0 * gr0) + fabsf(ft1 * gr1);
    part[8] = fmaxf(0.0f, fmaxf(-gr0, -gr1));
    part[9] = fmaxf(fabsf(ft0), fabsf(ft1));
    part[10] = fmaxf(fabsf(static_cast<float>(m0)), fabsf(static_cast<float>(m1)));
    part[11] = fmaxf(0.0f, fmaxf(-ft0, -ft1));
  } else {
    if (h0) fr[j0] = 0.0f;
    if (h1) fr[j1] = 0.0f;
  }
  rows_cta_tail(a, part, frow, 64, red);
}

// Residual norms, penalty rule (Sec. IV-D) and, for the last factor of a sweep, the fit,
// from the fixed-order sums of the scalar partials (one thread).
// Called by one whole warp (lane-parallel arithmetic; lane 0 writes).  FP64 division and
// square root are long instruction sequences on this GPU, so the quotients of the update's
// measures are formed in one division (lane q: quotient q) and the roots in one square root
// (lane q: root q) instead of one after the other.
__device__ void update_finalize(const UpdArgs& a, const double* sum, int lane) {
  Ctrl* c = a.ctrl;
  const double rho = c->stats[a.mode][5];
  // KKT measures of the factor's row problems at At (eq. KKT_NTF), scaled as
  // s_x = max |At|, s_g = max |G| s_x + max |M|
  const double sx = fmax(sum[9], 1e-30);
  const double sg = c->kkt[a.mode][3] * sx + sum[10];
  const double e2 = a.want_fit ? c->x_norm2 - 2.0 * sum[5] + sum[6] : 0.0;
  // quotients: lane 0 the relative squared error, 1 the negativity, 2 the dual infeasibility,
  // 3 the complementarity
  double num = 0.0, den = 1.0;
  if (lane == 0 && a.want_fit) {
    num = fmax(e2, 0.0);
    den = c->x_norm2;
  } else if (lane == 1) {
    num = fmax(0.0, sum[11]);
    den = sx;
  } else if (lane == 2 && sg > 0.0) {
    num = fmax(0.0, sum[8]);
    den = sg;
  } else if (lane == 3 && sg > 0.0) {
    num = sum[7];
    den = sg * sx * static_cast<double>(a.I) * a.R;
  }
  const double quo = num / den;
  // roots: lanes 0-4 the norms of sum[0..4], lane 5 the relative error
  const double q0 = __shfl_sync(0xffffffffu, quo, 0);
  const double rad = lane < 5 ? sum[lane < 5 ? lane : 0] : lane == 5 ? q0 : 0.0;
  const double root = sqrt(rad);
  double q[4], r[6];
#pragma unroll
  for (int k = 0; k < 4; ++k) q[k] = __shfl_sync(0xffffffffu, quo, k);
#pragma unroll
  for (int k = 0; k < 6; ++k) r[k] = __shfl_sync(0xffffffffu, root, k);
  if (lane != 0) return;
  const double P = r[0], D = rho * r[1];
  c->stats[a.mode][0] = P;
  c->stats[a.mode][1] = D;
  c->stats[a.mode][2] = r[2];
  c->stats[a.mode][3] = r[3];
  c->stats[a.mode][4] = r[4];
  bool finite = true;
  for (int k = 0; k < 5; ++k) finite = finite && isfinite(sum[k]);
  if (a.rho_policy == NTF_RHO_ADAPTIVE) {
    // eq. (varying_penalty_rule); the cases exclude each other because mu > 1
    double rr = rho;
    if (P > a.mu * D) rr = a.tau_incr * rho;
    else if (D > a.mu * P) rr = rho / a.tau_decr;
    c->rho[a.mode] = rr;
  } else if (a.rho_policy == NTF_RHO_TRACE) {
    c->rho[a.mode] = rho;
  }
  c->kkt[a.mode][0] = q[1];
  c->kkt[a.mode][1] = q[2];
  c->kkt[a.mode][2] = q[3];
  if (a.want_fit) {
    c->fit_inner = sum[5];
    c->fit_gram = sum[6];
    c->rel_err = r[5];
    finite = finite && isfinite(e2);
  }
  if (!finite) atomicOr(&c->status, kStNonFinite);
  if (a.snap && a.want_fit) {
    // the last factor of a sweep of ntf_run: at a checked sweep, the stopping rules (the fit
    // target; the residual criteria of Sec. IV-C over every factor's norms of this sweep)
    const int k = c->sweep;
    int stop = 0;
    if ((k + 1) % c->check_every == 0 || k + 1 == c->max_outer) {
      if (c->use_tgt && c->rel_err <= c->target_rfe) stop |= 1;
      if (c->use_res) {
        bool all = true;
        for (int m = 0; m < a.N && all; ++m) {
          const double* s = c->stats[m];
          all = s[0] <= c->res_base[m] + c->eps_rel * fmax(s[2], s[3]) &&
                s[1] <= c->res_base[m] + c->eps_rel * s[4];
        }
        if (all) stop |= 2;
      }
      if (c->use_kkt) {
        bool all = true;
        for (int m = 0; m < a.N && all; ++m) {
          const double* q = c->kkt[m];
          all = (c->kkt_dual_tol <= 0.0 || q[1] <= c->kkt_dual_tol) &&
                (c->kkt_comp_tol <= 0.0 || q[2] <= c->kkt_comp_tol);
        }
        if (all) stop |= 4;
      }
    }
    const int status = c->status;
    SweepSnap* sn = a.snap + (k & 1);
    sn->sweep = k + 1;
    sn->status = status;
    sn->stop = stop;
    sn->rel_err = c->rel_err;
    double kd = 0.0, kc = 0.0;
    for (int m = 0; m < a.N; ++m) {
      kd = fmax(kd, c->kkt[m][1]);
      kc = fmax(kc, c->kkt[m][2]);
    }
    sn->kkt_dual = kd;
    sn->kkt_comp = kc;
    c->stop_next = stop != 0 || status != 0;
    c->sweep = k + 1;
  }
}

// Packed Gram entry e of the updated factor: the per-CTA partials summed over blocks in a
// fixed order, read from L2 sixteen blocks at a time (the loads of a batch are independent, so
// they are in flight together; consecutive threads read consecutive entries).
__device__ __forceinline__ double gram_entry_sum(const UpdArgs& a, int nblocks, int e) {
  const int T = a.R * (a.R + 1) / 2;
  constexpr int kB = 16;
  double s = 0.0;
  int b = 0;
  for (; b + kB <= nblocks; b += kB) {
    double t[kB];
#pragma unroll
    for (int u = 0; u < kB; ++u) t[u] = __ldcg(a.gram_part + static_cast<int64_t>(b + u) * T + e);
#pragma unroll
    for (int w = kB / 2; w > 0; w >>= 1)
#pragma unroll
      for (int u = 0; u < w; ++u) t[u] += t[u + w];
    s += t[0];
  }
  if (b < nblocks) {
    double t[kB];
#pragma unroll
    for (int u = 0; u < kB; ++u)
      t[u] = b + u < nblocks ? __ldcg(a.gram_part + static_cast<int64_t>(b + u) * T + e) : 0.0;
#pragma unroll
    for (int w = kB / 2; w > 0; w >>= 1)
#pragma unroll
      for (int u = 0; u < w; ++u) t[u] += t[u + w];
    s += t[0];
  }
  return s;
}

// The same sum by the 8 lanes of a group (lanes 8g .. 8g+7 of a warp, called by the whole
// warp): lane s of the group takes blocks s, s + 8, ... (eight loads in flight per batch), and
// a fixed butterfly over the group gives every lane of it the same sum.  Entries e >= T read
// nothing and sum to zero.
__device__ __forceinline__ double gram_entry_sum8(const UpdArgs& a, int nblocks, int e, int s) {
  const int T = a.R * (a.R + 1) / 2;
  constexpr int kB = 8;
  double acc = 0.0;
  for (int b0 = s; b0 < nblocks; b0 += 8 * kB) {
    double t[kB];
#pragma unroll
    for (int u = 0; u < kB; ++u) {
      const int b = b0 + 8 * u;
      t[u] = b < nblocks && e < T ? __ldcg(a.gram_part + static_cast<int64_t>(b) * T + e) : 0.0;
    }
#pragma unroll
    for (int w = kB / 2; w > 0; w >>= 1)
#pragma unroll
      for (int u = 0; u < w; ++u) t[u] += t[u + w];
    acc += t[0];
  }
  acc += __shfl_xor_sync(0xffffffffu, acc, 1);
  acc += __shfl_xor_sync(0xffffffffu, acc, 2);
  acc += __shfl_xor_sync(0xffffffffu, acc, 4);
  return acc;
}

__device__ __forceinline__ void store_gram_entry(const UpdArgs& a, int e, double v) {
  int r, c;
  tri_index(e, r, c);
  a.gram_out[r * a.R + c] = v;
  a.gram_out[c * a.R + r] = v;
}

// Scalar partial q combined over blocks by one warp (summed for q < kSumScal, else the
// maximum): lane l takes blocks l, l + 32, ... and the lanes are combined by a fixed
// butterfly.
__device__ __forceinline__ double scalar_sum(const UpdArgs& a, int nblocks, int q, int lane) {
  const bool sum = q < kSumScal;
  double s = 0.0;
  for (int b = lane; b < nblocks; b += 32) {
    const double v = __ldcg(a.scal_part + b * kScal + q);
    s = sum ? s + v : fmax(s, v);
  }
  for (int off = 16; off > 0; off >>= 1) {
    const double o = __shfl_xor_sync(0xffffffffu, s, off);
    s = sum ? s + o : fmax(s, o);
  }
  return s;
}

// The whole reduction in one CTA of 256 threads (8 warps: one per scalar).
__device__ void update_reduce_cta(const UpdArgs& a, int nblocks) {
  __shared__ double s_sum[kScal];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int T = a.R * (a.R + 1) / 2;
  for (int e = tid; e < T; e += blockDim.x) store_gram_entry(a, e, gram_entry_sum(a, nblocks, e));
  for (int q = warp; q < kScal; q += blockDim.x / 32) {
    const double v = scalar_sum(a, nblocks, q, lane);
    if (lane == 0) s_sum[q] = v;
  }
  __syncthreads();
  if (warp == 0) update_finalize(a, s_sum, lane);
}

// Separate reduction: CTAs 0..gridDim.x-2 sum kRedEntries packed Gram entries each (8 lanes
// per entry, fixed order), the last CTA the scalars.
__global__ void __launch_bounds__(256) k_update_reduce(UpdArgs a, int nblocks) {
  __shared__ double s_sum[kScal];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (a.ctrl->bad[a.mode]) return;
  const int T = a.R * (a.R + 1) / 2;
  if (blockIdx.x + 1 < gridDim.x) {
    const int e = blockIdx.x * kRedEntries + (tid >> 3);
    const double v = gram_entry_sum8(a, nblocks, e, tid & 7);
    if ((tid & 7) == 0 && e < T) store_gram_entry(a, e, v);
    return;
  }
  for (int q = warp; q < kScal; q += 8) {
    const double v = scalar_sum(a, nblocks, q, lane);
    if (lane == 0) s_sum[q] = v;
  }
  __syncthreads();
  if (warp == 0) update_finalize(a, s_sum, lane);
}

// The reduction of factor m's update (as k_update_reduce) followed, in the last of its CTAs
// to finish, by the coefficient system of factor m + 1 (as k_update_system, 256 threads):
// that system needs factor m's new Gram and nothing else of this sweep, so it runs without a
// separate launch.  `as` describes factor m + 1.
template <int S>
__global__ void __launch_bounds__(256) k_update_reduce_system(UpdArgs a, UpdArgs as,
                                                              int nblocks) {
  __shared__ double s_sum[kScal];
  __shared__ int s_last;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int T = a.R * (a.R + 1) / 2;
  // the run has stopped (stop changes only in this kernel's last CTA, after every CTA has
  // read it): nothing to do
  if (a.ctrl->stop) return;
  if (!a.ctrl->bad[a.mode]) {  // uniform
    if (blockIdx.x + 1 < gridDim.x) {
      const int e = blockIdx.x * kRedEntries + (tid >> 3);
      const double v = gram_entry_sum8(a, nblocks, e, tid & 7);
      if ((tid & 7) == 0 && e < T) store_gram_entry(a, e, v);
    } else {
      for (int q = warp; q < kScal; q += 8) {
        const double v = scalar_sum(a, nblocks, q, lane);
        if (lane == 0) s_sum[q] = v;
      }
      __syncthreads();
      if (warp == 0) update_finalize(a, s_sum, lane);
    }
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = atomicAdd(&a.ctrl->sys_count, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  system_any<S, 256>(as);
  if (tid == 0) {
    a.ctrl->sys_count = 0;
    // every CTA of this kernel has read stop by now
    if (a.snap && a.want_fit) a.ctrl->stop = a.ctrl->stop_next;
  }
}

}  // namespace

const float* update_sys_h32(const double* sys, int mode, int R) {
  return sys_view(const_cast<double*>(sys), mode, R).h32;
}
const float* update_sys_hinv32(const double* sys, int mode, int R) {
  return sys_view(const_cast<double*>(sys), mode, R).hinv32;
}
const double* update_sys_hinv64(const double* sys, int mode, int R) {
  return sys_view(const_cast<double*>(sys), mode, R).hinv64;
}

int update_blocks(int64_t I) { return static_cast<int>((I + kRowWarps - 1) / kRowWarps); }
int update_scalars() { return kScal; }
size_t update_sys_bytes(int N, int R) { return static_cast<size_t>(N) * R * R * 16; }

namespace {
UpdArgs make_args(const UpdateCall& u) {
  UpdArgs a{};
  a.grams = u.grams;
  a.sys = u.sys;
  a.M = u.M;
  a.A = u.A;
  a.At = u.At;
  a.Y = u.Y;
  a.ctrl = u.ctrl;
  a.gram_part = u.gram_part;
  a.scal_part = u.scal_part;
  a.gram_out = u.gram_out;
  a.snap = u.snap;
  a.wsplit = u.wsplit;
  a.ws_kpad = u.ws_kpad;
  a.ws_n = u.ws_n;
  a.ws_bf16 = u.ws_bf16 ? 1 : 0;
  a.I = u.I;
  a.N = u.N;
  a.mode = u.mode;
  a.R = u.R;
  a.inner = u.inner;
  a.rho_policy = u.rho_policy;
  a.kr_aux = u.kr_aux ? 1 : 0;
  a.want_fit = u.want_fit ? 1 : 0;
  a.fused = update_fused(u) ? 1 : 0;
  a.box_lo = u.box_lo;
  a.box_hi = u.box_hi;
  a.tail_only = u.tail_only ? 1 : 0;
  a.t_before = u.t_before;
  a.mu = u.mu;
  a.tau_incr = u.tau_incr;
  a.tau_decr = u.tau_decr;
  a.inv_r = 1.0 / u.R;
  return a;
}
}  // namespace

cudaError_t launch_update_system(const UpdateCall& u, cudaStream_t st) {
  const UpdArgs a = make_args(u);
  const int T = u.R * (u.R + 1) / 2;  // packed lower triangle, S entries per thread
#define NTF_SYS(s)                                    \
  {                                                   \
    prefer_shared_carveout<k_update_system<s>>();     \
    k_update_system<s><<<1, kSysThreads, 0, st>>>(a); \
  }
  if (T <= 1 * kSysThreads) NTF_SYS(1)
  else if (T <= 2 * kSysThreads) NTF_SYS(2)
  else if (T <= 4 * kSysThreads) NTF_SYS(4)
  else if (T <= 9 * kSysThreads) NTF_SYS(9)
  else return cudaErrorInvalidValue;
#undef NTF_SYS
  return cudaGetLastError();
}

cudaError_t launch_update_rows(const UpdateCall& u, cudaStream_t st) {
  const UpdArgs a = make_args(u);
  const size_t RR = static_cast<size_t>(u.R) * u.R;
  const int nb = update_blocks(u.I);
  const bool fp32 = u.rho_policy == NTF_RHO_TRACE;
  if (u.R <= 32) {
    switch ((u.R + 3) / 4) {
#define NTF_ROWS32(q)                                                       \
  case q:                                                                   \
    if (fp32) {                                                             \
      prefer_shared_carveout<k_update_rows32<float, 4 * q>>();              \
      k_update_rows32<float, 4 * q><<<nb, kRowThreads, 0, st>>>(a);         \
    } else {                                                                \
      prefer_shared_carveout<k_update_rows32<double, 4 * q>>();             \
      k_update_rows32<double, 4 * q><<<nb, kRowThreads, 0, st>>>(a);        \
    }                                                                       \
    break;
      NTF_ROWS32(1) NTF_ROWS32(2) NTF_ROWS32(3) NTF_ROWS32(4)
      NTF_ROWS32(5) NTF_ROWS32(6) NTF_ROWS32(7) NTF_ROWS32(8)
#undef NTF_ROWS32
      default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
  }
  const size_t real = fp32 ? 4 : 8;
  const size_t row_smem = ((RR * real + RR * 4 + 15) / 16) * 16 + kRowWarps * 64 * real +
                          kRowWarps * 64 * 4;
  cudaError_t e;
  if (fp32) {
    prefer_shared_carveout<k_update_rows<float>>();
    e = cudaFuncSetAttribute(k_update_rows<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(row_smem));
    if (e == cudaSuccess) k_update_rows<float><<<nb, kRowThreads, row_smem, st>>>(a);
  } else {
    prefer_shared_carveout<k_update_rows<double>>();
    e = cudaFuncSetAttribute(k_update_rows<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(row_smem));
    if (e == cudaSuccess) k_update_rows<double><<<nb, kRowThreads, row_smem, st>>>(a);
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_update_reduce_system(const UpdateCall& u, const UpdateCall& next,
                                        cudaStream_t st) {
  const UpdArgs a = make_args(u), as = make_args(next);
  const int gram_ctas = (u.R * (u.R + 1) / 2 + kRedEntries - 1) / kRedEntries;
  const int T = u.R * (u.R + 1) / 2, nb = update_blocks(u.I);
  const dim3 grid(gram_ctas + 1);
#define NTF_RSYS(s)                                              \
  {                                                              \
    prefer_shared_carveout<k_update_reduce_system<s>>();         \
    k_update_reduce_system<s><<<grid, 256, 0, st>>>(a, as, nb);  \
  }
  if (T <= 256) NTF_RSYS(1)
  else if (T <= 512) NTF_RSYS(2)
  else if (T <= 1024) NTF_RSYS(4)
  else if (T <= 2304) NTF_RSYS(9)
  else return cudaErrorInvalidValue;
#undef NTF_RSYS
  return cudaGetLastError();
}

bool update_fused(const UpdateCall& u) {
  return static_cast<int64_t>(update_blocks(u.I)) * u.R * (u.R + 1) / 2 <= kFusedReduceMax;
}

cudaError_t launch_update_reduce(const UpdateCall& u, cudaStream_t st) {
  if (update_fused(u)) return cudaSuccess;  // done by the rows kernel
  const UpdArgs a = make_args(u);
  const int gram_ctas = (u.R * (u.R + 1) / 2 + kRedEntries - 1) / kRedEntries;
  prefer_shared_carveout<k_update_reduce>();
  k_update_reduce<<<gram_ctas + 1, 256, 0, st>>>(a, update_blocks(u.I));
  return cudaGetLastError();
}

cudaError_t launch_update(const UpdateCall& u, cudaStream_t st) {
  cudaError_t e = launch_update_system(u, st);
  if (e == cudaSuccess) e = launch_update_rows(u, st);
  if (e == cudaSuccess) e = launch_update_reduce(u, st);
  return e;
}

}  // namespace ntf
