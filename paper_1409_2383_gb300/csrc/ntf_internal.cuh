// Internal declarations of the GB300 NTF library: context, device control block, launch
// helpers.  Not part of the ABI (include/ntf.h is).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "ntf.h"

namespace ntf {

constexpr int kMaxOrder = 4;
constexpr int kMaxRank = 64;
constexpr int kNumSM = 152;  // used only to size grids; the real count is queried at create

// A group of consecutive modes whose factors are combined into Khatri-Rao rows.  Row q of
// the group's Khatri-Rao table decomposes with the LAST mode fastest, matching the
// row-major tensor layout: q = ((i_0 * dim_1) + i_1) * dim_2 + i_2.
struct Group {
  const float* F[3];
  int dim[3];
  int n;
};

// Deferred device-side error bits.
enum : int { kStNotSpd = 1, kStNonFinite = 2, kStTimeout = 4 };

// Small device-resident control block: penalties, residual norms and fit terms live here so
// that a whole sweep runs without host round trips.
struct Ctrl {
  double rho[kMaxOrder];          // penalty per factor (adaptive / fixed policies)
  double stats[kMaxOrder][8];     // primal, dual, |A|, |At|, |Y|, rho used, -, -
  double fit_inner;               // <M_N, F_N>
  double fit_gram;                // 1^T (Hadamard of all Grams) 1
  double rel_err;
  double x_norm2;
  int status;                     // kSt* bits
  int bad[kMaxOrder];             // 1 if the last system of factor n was not SPD
  int pad[3];
};

// ------------------------------------------------------------------ kernel launchers
// mttkrp.cu
struct GemmPlan {
  int splits;       // split-K factor
  int blocks;       // row blocks (GEMM-N) or column blocks (GEMM-T)
  int rows_per_blk; // GEMM-N rows per block
  bool vec16;       // 16-byte cp.async staging possible
};

GemmPlan plan_gemm_n(int64_t P, int64_t Q, int R, int dtype, const void* X, int num_sms);
GemmPlan plan_gemm_t(int64_t P, int64_t Q, int R, int dtype, const void* X, int num_sms);

// out (or partial[splits] if plan.splits > 1) [P, R] = X[P, Q] * KR(g)[Q, R]
cudaError_t launch_gemm_n(const void* X, int dtype, int64_t P, int64_t Q, int R, const Group& g,
                          const GemmPlan& plan, float* out_or_partial, cudaStream_t st);
// out (or partial) [Q, R] = X[P, Q]^T * KR(g)[P, R]
cudaError_t launch_gemm_t(const void* X, int dtype, int64_t P, int64_t Q, int R, const Group& g,
                          const GemmPlan& plan, float* out_or_partial, cudaStream_t st);
// out[n] = sum_s partial[s * n + i]
cudaError_t launch_sum_splits(const float* partial, int splits, int64_t n, float* out,
                              cudaStream_t st);
// T[Ia, Ib, R]:  fast: out[a, r] = sum_b T[a, b, r] F[b, r];  slow: out[b, r] = sum_a T F[a, r]
cudaError_t launch_post_fast(const float* T, int64_t Ia, int64_t Ib, int R, const float* F,
                             float* out, cudaStream_t st);
int post_slow_splits(int64_t Ia, int64_t Ib, int R, int num_sms);
cudaError_t launch_post_slow(const float* T, int64_t Ia, int64_t Ib, int R, const float* F,
                             int splits, float* partial, float* out, cudaStream_t st);
cudaError_t launch_norm2(const void* X, int dtype, int64_t n, double* partial, int blocks,
                         double* out, cudaStream_t st);
cudaError_t launch_to_bf16(const float* in, uint16_t* out, int64_t n, cudaStream_t st);

// admm.cu
cudaError_t launch_gram(const float* F, int64_t I, int R, double* G, cudaStream_t st);
cudaError_t launch_system(const double* grams, int N, int mode, int R, int rho_policy,
                          Ctrl* ctrl, double* H, double* L, cudaStream_t st);
int admm_row_blocks(int64_t I);
cudaError_t launch_admm_rows(const float* M, float* A, float* At, float* Y, const double* L,
                             int64_t I, int R, int inner, int mode, Ctrl* ctrl,
                             double* norm_part, cudaStream_t st);
cudaError_t launch_update_finalize(const double* norm_part, int nblocks, int mode,
                                   int rho_policy, double mu, double tau_incr,
                                   double tau_decr, Ctrl* ctrl, cudaStream_t st);
int fit_blocks(int64_t I, int R);
cudaError_t launch_fit(const float* M, const float* F, int64_t I, int R, const double* grams,
                       int N, double* partial, Ctrl* ctrl, cudaStream_t st);

}  // namespace ntf
