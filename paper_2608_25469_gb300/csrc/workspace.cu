// Stream-ordered workspace allocation (see workspace.h).
#include <atomic>
#include <cstdlib>

#include "common.cuh"
#include "workspace.h"

namespace {
std::atomic<long> g_allocs{0};

long fault_after() {
  const char *e = std::getenv("HSMA_FAULT_ALLOC_AFTER");
  if (e == nullptr || *e == '\0') return -1;
  return std::atol(e);
}
}  // namespace

hsma_status_t hsma_ws_alloc(void **p, size_t bytes, cudaStream_t st) {
  *p = nullptr;
  const long lim = fault_after();
  const long k = g_allocs.fetch_add(1);
  if (lim >= 0 && k >= lim) return HSMA_ERR_NO_MEMORY;
  if (bytes == 0) return HSMA_OK;
  cudaError_t e = cudaMallocAsync(p, bytes, st);
  if (e != cudaSuccess) {
    *p = nullptr;
    (void)cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? HSMA_ERR_NO_MEMORY : HSMA_ERR_CUDA;
  }
  return HSMA_OK;
}

hsma_status_t hsma_ws_free(void *p, cudaStream_t st) {
  if (p == nullptr) return HSMA_OK;
  HSMA_CUDA_TRY(cudaFreeAsync(p, st));
  return HSMA_OK;
}
