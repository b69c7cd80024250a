// Self-test of the bounded waits the staging pipelines rely on (sllbm_selftest_bounded_wait).
//
// Every wait of the TMA-staged step kernels on an mbarrier has an iteration limit: if a stage
// never lands, the wait gives up, sets bit 2 of the context's flag (reported by sllbm_moments as
// SLLBM_ERR_CUDA) and the CTA stops, instead of hanging the GPU.  This kernel runs that wait on
// an mbarrier that nothing arrives on -- no copy involved, nothing in flight -- with a short limit,
// so that a test can check on the GPU that the wait runs out, reports it, and the kernel returns.
#include "../../include/sllbm.h"
#include "kernels.h"
#include "tma.cuh"

namespace sllbm {
namespace {

static __device__ int g_selftest_flag;

// One CTA: thread 0 initialises an mbarrier expecting one arrival that never comes; every thread
// waits for its first phase with the limited wait (4096 polls) and returns when it runs out.
__global__ void bounded_wait_selftest_kernel(int* flag) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  const bool landed = mbar_wait<4096>(&bar, 0u, flag);
  if (landed) atomicOr(flag, 8);   // a phase completed that nothing could complete: a failure
}

}  // namespace
}  // namespace sllbm

extern "C" sllbm_status sllbm_selftest_bounded_wait(void* cuda_stream) {
  using namespace sllbm;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  int* flag = nullptr;
  if (cudaGetSymbolAddress(reinterpret_cast<void**>(&flag), g_selftest_flag) != cudaSuccess) return SLLBM_ERR_CUDA;
  if (cudaMemsetAsync(flag, 0, sizeof(int), s) != cudaSuccess) return SLLBM_ERR_CUDA;
  bounded_wait_selftest_kernel<<<1, 64, 0, s>>>(flag);
  if (cudaGetLastError() != cudaSuccess) return SLLBM_ERR_CUDA;
  int host = 0;
  if (cudaMemcpyAsync(&host, flag, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return SLLBM_ERR_CUDA;
  // the wait must have run out (bit 2) and no phase may have completed (bit 3)
  return (host & 4) && !(host & 8) ? SLLBM_OK : SLLBM_ERR_CUDA;
}
