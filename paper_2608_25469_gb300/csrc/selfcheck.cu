// Self-check of the failure-detection path: the bounded mbarrier wait of the
// tensor-core kernels, run against a barrier that nothing arrives on.
#include <cuda_runtime.h>

#include "../../include/hsma.h"
#include "blocked.h"
#include "common.cuh"
#include "tma.cuh"
#include "trace.h"

namespace {
// One thread waits, with the library's bounded wait, on an mbarrier that
// expects one arrival that nothing makes: the wait runs out after limit_ns
// and raises HSMA_DEVERR_TIMEOUT in the device error word.
__global__ void wait_timeout_check_kernel(uint64_t limit_ns, unsigned int *err, int *returned) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  fence_mbar_init();
  const bool ok = mbar_wait_bounded(&bar, 0, limit_ns, err);
  *returned = ok ? 1 : 2;
}
}  // namespace

extern "C" HSMA_API hsma_status_t hsma_check_wait_timeout(uint64_t limit_ns, int *d_returned, void *stream) {
  if (d_returned == nullptr || limit_ns < 1000000ull || limit_ns > 2000000000ull) return HSMA_ERR_INVALID_ARG;
  unsigned int *err = hsma_dev_error_ptr();
  if (err == nullptr) return HSMA_ERR_CUDA;
  wait_timeout_check_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(limit_ns, err, d_returned);
  hsma_count_launches(1);
  return hsma_from_cuda(cudaGetLastError());
}
