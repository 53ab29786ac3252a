// Self-test of the bounded waits every pipeline kernel uses: one thread waits on an mbarrier
// that nothing arrives on, with the same wait helper and a short limit, and reports the
// expiry in the status word the host reads; the context stays usable.
#include <cuda_runtime.h>

#include "internal.h"
#include "tcgen05.cuh"

namespace rs {
namespace {

__global__ void wait_expiry_kernel(uint64_t limit_ns, uint32_t *status, uint32_t *waited_ms) {
  __shared__ __align__(8) uint64_t bar;
  const uint32_t a = smem_u32(&bar);
  if (threadIdx.x == 0) {
    mbar_init(a, 1);  // one arrival expected; none comes
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint64_t t0 = global_ns();
    if (!mbar_wait_for(a, 0, limit_ns)) atomicOr(status, kStatusWaitLimit);
    *waited_ms = static_cast<uint32_t>((global_ns() - t0) / 1000000ull);
  }
}

}  // namespace
}  // namespace rs

extern "C" SIM_API int sim_selftest_wait(int32_t limit_ms, int32_t *waited_ms, void *stream) {
  if (limit_ms < 1 || limit_ms > 1000 || !waited_ms) return SIM_E_INVALID;
  uint32_t *buf = nullptr;
  if (cudaMalloc(&buf, 8) != cudaSuccess) return SIM_E_NOMEM;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaMemsetAsync(buf, 0, 8, s);
  rs::wait_expiry_kernel<<<1, 32, 0, s>>>(static_cast<uint64_t>(limit_ms) * 1000000ull, buf, buf + 1);
  uint32_t h[2] = {0, 0};
  cudaMemcpyAsync(h, buf, 8, cudaMemcpyDeviceToHost, s);
  const cudaError_t e = cudaStreamSynchronize(s);
  cudaFree(buf);
  if (e != cudaSuccess) return SIM_E_CUDA;
  *waited_ms = static_cast<int32_t>(h[1]);
  return (h[0] & rs::kStatusWaitLimit) ? SIM_E_DEVICE : SIM_OK;
}
