// One factor update of eq. (ADMM_NTF_ALS_C) followed by the projection and dual steps of
// eq. (ADMoM_NTF), repeated inner_iters times, as three launches:
//
//  k_update_system  one CTA: H = Hadamard_{m != n} Gram_m + rho I (FP64), its Cholesky factor
//                   L and H^{-1} = L^{-T} L^{-1} (FP64) -- the coefficient matrix common to all
//                   rows (App. B), factored once.  Stored as FP64 and as FP32 copies.
//  k_update_rows    one warp per row: x = H^{-1}(m + rho At - Y), At = (x + Y/rho)_+,
//                   Y += rho (x - At); per-CTA partial sums of the residual norms of
//                   Sec. III-C, of the new factor's Gram (FP64) and of the fit terms
//                   <M_i, f_i>, f_i^T G f_i.  The row arithmetic is FP32 under the trace
//                   penalty policy (then cond(H) <= R + 1) and FP64 otherwise.
//  k_update_reduce  fixed-order sums of the partials: the stored Gram of the factor, the
//                   residuals, the penalty rule (Sec. III-D) and, for the last factor of a
//                   sweep, the relative error ||X||^2 - 2<M, F> + sum_i f_i^T G f_i.
#include <cmath>

#include "ntf_internal.cuh"

namespace ntf {
namespace {

constexpr int kSysThreads = 256;
constexpr int kRowWarps = 8;  // rows per CTA
constexpr int kRowThreads = kRowWarps * 32;
constexpr int kScal = 8;      // scalar partials per CTA
constexpr int kRedEntries = 64;

// 1/sqrt(d) for d > 0: the single-precision estimate refined by one Newton-Raphson step for
// f(y) = y^-2 - d (y <- y (3 - d y^2) / 2), which squares its relative error (~1e-7 -> ~1e-14).
__device__ __forceinline__ double rsqrt_newton(double d) {
  const float df = static_cast<float>(d);
  if (!(df > 0.0f) || isinf(df) || df < 1e-30f) return rsqrt(d);
  const double y = static_cast<double>(rsqrtf(df));
  return y * fma(-0.5 * d * y, y, 1.5);
}

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
  double* gram_part;    // [blocks, R, R]
  double* scal_part;    // [blocks, kScal]
  double* gram_out;     // [R, R] stored Gram of this factor
  int64_t I;
  int N, mode, R, inner, rho_policy, kr_aux, want_fit;
  double mu, tau_incr, tau_decr;
};

__global__ void __launch_bounds__(kSysThreads) k_update_system(UpdArgs a) {
  extern __shared__ double sh[];
  const int R = a.R, RR = R * R;
  double* Hs = sh;          // Hadamard of the other Grams (no rho)
  double* Af = Hs + RR;     // H + rho I -> Cholesky factor -> H^{-1}
  double* Wm = Af + RR;     // L^{-1}
  double* invd = Wm + RR;   // [64] 1/L_kk
  __shared__ double s_rho, s_pinv;
  __shared__ int s_fail;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < RR; idx += kSysThreads) {
    double v = 1.0;
    for (int m = 0; m < a.N; ++m)
      if (m != a.mode) v *= a.grams[m * RR + idx];
    Hs[idx] = v;
    Af[idx] = v;
  }
  __syncthreads();
  if (tid == 0) {
    double rho;
    if (a.rho_policy == NTF_RHO_TRACE) {
      double tr = 0.0;
      for (int i = 0; i < R; ++i) tr += Hs[i * R + i];
      rho = tr / R;
    } else {
      rho = a.ctrl->rho[a.mode];
    }
    s_rho = rho;
    s_fail = !(rho > 0.0) || !isfinite(rho);
    for (int i = 0; i < R; ++i) Af[i * R + i] += rho;
  }
  __syncthreads();
  // Cholesky, right-looking, columns left unscaled (pivot d_k) and scaled by 1/L_kk after
  for (int k = 0; k < R && !s_fail; ++k) {
    if (tid == 0) {
      const double d = Af[k * R + k];
      if (!(d > 0.0) || !isfinite(d)) {
        s_fail = 1;
      } else {
        const double rs = rsqrt_newton(d);
        invd[k] = rs;
        Af[k * R + k] = d * rs;
        s_pinv = rs * rs;
      }
    }
    __syncthreads();
    if (s_fail) break;
    const double pinv = s_pinv;
    const int n = R - k - 1;
    for (int idx = tid; idx < n * n; idx += kSysThreads) {
      const int i = k + 1 + idx / n, j = k + 1 + idx % n;
      if (j <= i) Af[i * R + j] -= Af[i * R + k] * Af[j * R + k] * pinv;
    }
    __syncthreads();
  }
  if (s_fail) {
    if (tid == 0) {
      a.ctrl->bad[a.mode] = 1;
      atomicOr(&a.ctrl->status, kStNotSpd);
    }
    return;
  }
  for (int idx = tid; idx < RR; idx += kSysThreads) {
    const int i = idx / R, j = idx % R;
    if (j < i) Af[idx] *= invd[j];
    Wm[idx] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  // L^{-1}: column-oriented forward substitution on all columns at once; rows kept unscaled
  // (B) and scaled at the end: W[k][c] = B[k][c] / L_kk.
  for (int k = 0; k < R - 1; ++k) {
    const double rk = invd[k];
    const int n = R - k - 1, w = k + 1;
    for (int idx = tid; idx < n * w; idx += kSysThreads) {
      const int j = k + 1 + idx / w, c = idx % w;
      Wm[j * R + c] -= Af[j * R + k] * (Wm[k * R + c] * rk);
    }
    __syncthreads();
  }
  for (int idx = tid; idx < RR; idx += kSysThreads) {
    const int k = idx / R, c = idx % R;
    if (c <= k) Wm[idx] *= invd[k];
  }
  __syncthreads();
  const SysView sv = sys_view(a.sys, a.mode, R);
  for (int idx = tid; idx < RR; idx += kSysThreads) {
    const int i = idx / R, j = idx % R;
    double s = 0.0;
    for (int k = max(i, j); k < R; ++k) s = fma(Wm[k * R + i], Wm[k * R + j], s);
    sv.hinv64[idx] = s;
    sv.hinv32[idx] = static_cast<float>(s);
    sv.h32[idx] = static_cast<float>(Hs[idx]);
  }
  if (tid == 0) {
    a.ctrl->bad[a.mode] = 0;
    a.ctrl->stats[a.mode][5] = s_rho;
  }
}

// Rows.  Real = float (trace policy) or double.  One warp per row, lanes own elements lane
// and lane + 32; v and f are broadcast through a per-warp shared buffer.
template <typename Real>
__global__ void __launch_bounds__(kRowThreads) k_update_rows(UpdArgs a) {
  extern __shared__ double shd[];
  const int R = a.R, RR = R * R;
  Real* Hi = reinterpret_cast<Real*>(shd);                       // [RR] H^{-1}
  float* Hf = reinterpret_cast<float*>(Hi + RR);                 // [RR] H (fit only)
  Real* vbuf = reinterpret_cast<Real*>(shd + ((RR * sizeof(Real) + RR * 4 + 15) / 16) * 2);
  float* frow = reinterpret_cast<float*>(vbuf + kRowWarps * 64); // [kRowWarps][64]
  __shared__ double red[kRowWarps][kScal];
  if (a.ctrl->bad[a.mode]) return;  // uniform
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const SysView sv = sys_view(a.sys, a.mode, R);
  for (int idx = tid; idx < RR; idx += kRowThreads) {
    if constexpr (sizeof(Real) == 4) Hi[idx] = sv.hinv32[idx];
    else Hi[idx] = sv.hinv64[idx];
    if (a.want_fit) Hf[idx] = sv.h32[idx];
  }
  __syncthreads();
  const Real rho = static_cast<Real>(a.ctrl->stats[a.mode][5]);
  const Real rinv = Real(1) / rho;
  const int64_t row = static_cast<int64_t>(blockIdx.x) * kRowWarps + warp;
  float part[kScal] = {0, 0, 0, 0, 0, 0, 0, 0};
  const int j0 = lane, j1 = lane + 32;
  const bool h0 = j0 < R, h1 = j1 < R;
  Real* vb = vbuf + warp * 64;
  float* fr = frow + warp * 64;
  if (row < a.I) {
    const int64_t base = row * R;
    const Real m0 = h0 ? a.M[base + j0] : 0, m1 = h1 ? a.M[base + j1] : 0;
    Real t0 = h0 ? a.At[base + j0] : 0, t1 = h1 ? a.At[base + j1] : 0;
    Real y0 = h0 ? a.Y[base + j0] : 0, y1 = h1 ? a.Y[base + j1] : 0;
    const Real s0 = t0, s1 = t1;
    Real x0 = 0, x1 = 0;
    for (int it = 0; it < a.inner; ++it) {
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
      const Real n0 = fmax(Real(0), x0 + y0 * rinv), n1 = fmax(Real(0), x1 + y1 * rinv);
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
    if (a.want_fit) {
      part[5] = static_cast<float>(m0) * f0 + static_cast<float>(m1) * f1;
      __syncwarp();
      float g0 = 0.0f, g1 = 0.0f;
      for (int kk = 0; kk < R; ++kk) {
        const float fk = fr[kk];
        if (h0) g0 = fmaf(Hf[kk * R + j0], fk, g0);
        if (h1) g1 = fmaf(Hf[kk * R + j1], fk, g1);
      }
      part[6] = f0 * g0 + f1 * g1;
    }
  } else {
    if (h0) fr[j0] = 0.0f;
    if (h1) fr[j1] = 0.0f;
  }
#pragma unroll
  for (int q = 0; q < kScal; ++q)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) part[q] += __shfl_xor_sync(0xffffffffu, part[q], off);
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < kScal; ++q) red[warp][q] = part[q];
  __syncthreads();
  if (tid < kScal) {
    double s = 0.0;
    for (int w = 0; w < kRowWarps; ++w) s += red[w][tid];
    a.scal_part[blockIdx.x * kScal + tid] = s;
  }
  // this CTA's share of the new Gram: FP64 accumulation of products of the stored FP32
  // values (a product of two FP32 numbers is exact in FP64)
  double* gp = a.gram_part + static_cast<int64_t>(blockIdx.x) * RR;
  for (int idx = tid; idx < RR; idx += kRowThreads) {
    const int r = idx / R, s = idx % R;
    double g0 = 0.0, g1 = 0.0;
#pragma unroll
    for (int w = 0; w < kRowWarps; w += 2) {
      g0 = fma(static_cast<double>(frow[w * 64 + r]), static_cast<double>(frow[w * 64 + s]), g0);
      g1 = fma(static_cast<double>(frow[(w + 1) * 64 + r]),
               static_cast<double>(frow[(w + 1) * 64 + s]), g1);
    }
    gp[idx] = g0 + g1;
  }
}

// CTAs 0..gridDim.x-2: 64 Gram entries each, 4 threads per entry summing every 4th block,
// combined in a fixed order.  Last CTA: residuals, penalty rule, fit.
__global__ void __launch_bounds__(256) k_update_reduce(UpdArgs a, int nblocks) {
  __shared__ double sred[256][kScal];
  const int tid = threadIdx.x;
  if (a.ctrl->bad[a.mode]) return;
  const int RR = a.R * a.R;
  if (blockIdx.x + 1 < gridDim.x) {
    const int e = blockIdx.x * kRedEntries + tid / 4, part = tid % 4;
    double s0 = 0.0, s1 = 0.0;
    if (e < RR) {
      int b = part;
      for (; b + 4 < nblocks; b += 8) {
        s0 += a.gram_part[static_cast<int64_t>(b) * RR + e];
        s1 += a.gram_part[static_cast<int64_t>(b + 4) * RR + e];
      }
      if (b < nblocks) s0 += a.gram_part[static_cast<int64_t>(b) * RR + e];
    }
    sred[tid][0] = s0 + s1;
    __syncthreads();
    if (part == 0 && e < RR)
      a.gram_out[e] = ((sred[tid][0] + sred[tid + 1][0]) + sred[tid + 2][0]) + sred[tid + 3][0];
    return;
  }
  double s[kScal] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int b = tid; b < nblocks; b += 256)
#pragma unroll
    for (int q = 0; q < kScal; ++q) s[q] += a.scal_part[b * kScal + q];
#pragma unroll
  for (int q = 0; q < kScal; ++q) sred[tid][q] = s[q];
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (tid < w)
#pragma unroll
      for (int q = 0; q < kScal; ++q) sred[tid][q] += sred[tid + w][q];
    __syncthreads();
  }
  if (tid != 0) return;
  Ctrl* c = a.ctrl;
  const double rho = c->stats[a.mode][5];
  const double P = sqrt(sred[0][0]), D = rho * sqrt(sred[0][1]);
  c->stats[a.mode][0] = P;
  c->stats[a.mode][1] = D;
  c->stats[a.mode][2] = sqrt(sred[0][2]);
  c->stats[a.mode][3] = sqrt(sred[0][3]);
  c->stats[a.mode][4] = sqrt(sred[0][4]);
  bool finite = true;
  for (int q = 0; q < 5; ++q) finite = finite && isfinite(sred[0][q]);
  if (a.rho_policy == NTF_RHO_ADAPTIVE) {
    // eq. (varying_penalty_rule); the cases exclude each other because mu > 1
    double r = rho;
    if (P > a.mu * D) r = a.tau_incr * rho;
    else if (D > a.mu * P) r = rho / a.tau_decr;
    c->rho[a.mode] = r;
  } else if (a.rho_policy == NTF_RHO_TRACE) {
    c->rho[a.mode] = rho;
  }
  if (a.want_fit) {
    const double inner = sred[0][5], quad = sred[0][6];
    const double e2 = c->x_norm2 - 2.0 * inner + quad;
    c->fit_inner = inner;
    c->fit_gram = quad;
    c->rel_err = sqrt(fmax(e2, 0.0) / c->x_norm2);
    finite = finite && isfinite(e2);
  }
  if (!finite) atomicOr(&c->status, kStNonFinite);
}

}  // namespace

const float* update_sys_h32(const double* sys, int mode, int R) {
  return sys_view(const_cast<double*>(sys), mode, R).h32;
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
  a.I = u.I;
  a.N = u.N;
  a.mode = u.mode;
  a.R = u.R;
  a.inner = u.inner;
  a.rho_policy = u.rho_policy;
  a.kr_aux = u.kr_aux ? 1 : 0;
  a.want_fit = u.want_fit ? 1 : 0;
  a.mu = u.mu;
  a.tau_incr = u.tau_incr;
  a.tau_decr = u.tau_decr;
  return a;
}
}  // namespace

cudaError_t launch_update_system(const UpdateCall& u, cudaStream_t st) {
  const UpdArgs a = make_args(u);
  const size_t RR = static_cast<size_t>(u.R) * u.R;
  const size_t sys_smem = (3 * RR + 64) * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(k_update_system,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(sys_smem));
  if (e != cudaSuccess) return e;
  k_update_system<<<1, kSysThreads, sys_smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_update_rows(const UpdateCall& u, cudaStream_t st) {
  const UpdArgs a = make_args(u);
  const size_t RR = static_cast<size_t>(u.R) * u.R;
  const int nb = update_blocks(u.I);
  const bool fp32 = u.rho_policy == NTF_RHO_TRACE;
  const size_t real = fp32 ? 4 : 8;
  const size_t row_smem = ((RR * real + RR * 4 + 15) / 16) * 16 + kRowWarps * 64 * real +
                          kRowWarps * 64 * 4;
  cudaError_t e;
  if (fp32) {
    e = cudaFuncSetAttribute(k_update_rows<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(row_smem));
    if (e == cudaSuccess) k_update_rows<float><<<nb, kRowThreads, row_smem, st>>>(a);
  } else {
    e = cudaFuncSetAttribute(k_update_rows<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(row_smem));
    if (e == cudaSuccess) k_update_rows<double><<<nb, kRowThreads, row_smem, st>>>(a);
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_update_reduce(const UpdateCall& u, cudaStream_t st) {
  const UpdArgs a = make_args(u);
  const int gram_ctas = (u.R * u.R + kRedEntries - 1) / kRedEntries;
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
