// Instantiation unit: GEMM-T MTTKRP contraction for bf16 tensor storage.
#include "mttkrp_kernels.cuh"

namespace ntf {
namespace detail {
template cudaError_t gemm_t_typed<__nv_bfloat16>(const __nv_bfloat16*, int64_t, int64_t, int, const float*,
                                         const GemmPlan&, float*, cudaStream_t);
}  // namespace detail
}  // namespace ntf
