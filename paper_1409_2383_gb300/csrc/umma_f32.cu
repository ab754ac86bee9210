// Tensor-core contractions for FP32 tensor storage (kernels in umma_kernels.cuh).
#include "umma_kernels.cuh"

namespace ntf {
namespace umma {
cudaError_t launch_f32(const UmmaPlan& p, const Args& a, cudaStream_t st) {
  return dispatch<true>(p, a, st);
}
}  // namespace umma
}  // namespace ntf
