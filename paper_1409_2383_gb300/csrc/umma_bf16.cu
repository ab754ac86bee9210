// Tensor-core contractions for BF16 tensor storage (kernels in umma_kernels.cuh).
#include "umma_kernels.cuh"

namespace ntf {
namespace umma {
cudaError_t launch_bf16(const UmmaPlan& p, const Args& a, cudaStream_t st) {
  return dispatch<false>(p, a, st);
}

namespace {
// The contractions' bounded wait on an mbarrier that nothing completes: it gives up after
// limit_ns and reports the timeout the way the contractions do.
__global__ void k_wait_check(int* err, uint64_t limit_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x != 0) return;
  bar_init(&bar, 1);
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  if (!bar_wait(&bar, 0, nullptr, limit_ns)) atomicOr(err, kStTimeout);
}
}  // namespace

}  // namespace umma

cudaError_t launch_wait_check(int* err, uint64_t limit_ns, cudaStream_t st) {
  umma::k_wait_check<<<1, 32, 0, st>>>(err, limit_ns);
  return cudaGetLastError();
}
}  // namespace ntf
