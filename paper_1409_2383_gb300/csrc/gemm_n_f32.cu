// Instantiation unit: GEMM-N MTTKRP contraction for f32 tensor storage.
#include "mttkrp_kernels.cuh"

namespace ntf {
namespace detail {
template cudaError_t gemm_n_typed<float>(const float*, int64_t, int64_t, int, const float*,
                                         const GemmPlan&, float*, cudaStream_t);
}  // namespace detail
}  // namespace ntf
