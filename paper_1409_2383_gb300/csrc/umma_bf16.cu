// Tensor-core contractions for BF16 tensor storage (kernels in umma_kernels.cuh).
#include "umma_kernels.cuh"

namespace ntf {
namespace umma {
cudaError_t launch_bf16(const UmmaPlan& p, const Args& a, cudaStream_t st) {
  return dispatch<false>(p, a, st);
}
}  // namespace umma
}  // namespace ntf
