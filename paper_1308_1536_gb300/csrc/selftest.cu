// Failure detection self-test (the paper has no counterpart).  The kernels'
// hand-offs wait on mbarriers with a bounded number of polls and report
// MPDET_ETIMEOUT through their status word instead of hanging; this entry
// point runs one such bounded wait on a barrier that nothing completes (or,
// as a control, that the waiting block completes itself), so that a test
// can check the timeout path and that the context stays usable after it.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/mpdet.h"

namespace {

// One block of 32 threads: thread 0 initialises an mbarrier expecting one
// arrival; with arrive != 0 it arrives (phase 0 completes); every thread then
// polls phase 0 at most `limit` times, the form of the kernels' waits.
__global__ void k_wait_selftest(int* status, int limit, int arrive) {
  __shared__ __align__(8) uint64_t bar;
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(&bar);
  if (threadIdx.x == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(a));
  __syncthreads();
  if (arrive && threadIdx.x == 0) asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(a));
  uint32_t done = 0;
  for (int it = 0; it < limit && !done; ++it)
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done)
                 : "r"(a), "r"(0u));
  if (!done) atomicExch(status, MPDET_ETIMEOUT);
}

}  // namespace

extern "C" int mpdet_selftest_timeout(int32_t limit, int arrive, void* cuda_stream) {
  if (limit < 1) return MPDET_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int* d = nullptr;
  if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) return MPDET_ENOMEM;
  int h = -1;
  bool ok = cudaMemsetAsync(d, 0, sizeof(int), st) == cudaSuccess;
  if (ok) {
    k_wait_selftest<<<1, 32, 0, st>>>(d, limit, arrive);
    ok = cudaGetLastError() == cudaSuccess &&
         cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
         cudaStreamSynchronize(st) == cudaSuccess;
  }
  cudaFree(d);
  if (!ok) return MPDET_ECUDA;
  return h == MPDET_ETIMEOUT ? MPDET_ETIMEOUT : MPDET_OK;
}
