// Stream-ordered workspace allocation (see workspace.h).
#include <atomic>
#include <cstdint>
#include <cstdlib>
#include <mutex>

#include "common.cuh"
#include "workspace.h"

namespace {
std::atomic<long> g_allocs{0};

// Freed workspace stays reserved in the library's pool up to this many bytes,
// so a call that follows a synchronisation does not map fresh physical memory
// for its workspace (the default pool of the device releases it at every
// synchronisation); memory above it goes back at synchronisation points.
constexpr uint64_t kPoolKeepBytes = 4ull << 30;
constexpr int kMaxDevices = 64;

// one stream-ordered memory pool per device, owned by the library (null when
// it could not be created: the device's default pool is used instead)
cudaMemPool_t library_pool(int dev) {
  static std::mutex mu;
  static cudaMemPool_t pools[kMaxDevices] = {};
  static bool tried[kMaxDevices] = {};
  if (dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  if (!tried[dev]) {
    tried[dev] = true;
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) == cudaSuccess) {
      uint64_t keep = kPoolKeepBytes;
      if (cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep) == cudaSuccess)
        pools[dev] = pool;
      else
        (void)cudaMemPoolDestroy(pool);
    }
    (void)cudaGetLastError();
  }
  return pools[dev];
}

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
  // under stream capture the allocation becomes a graph memory node from the
  // default pool, as before; otherwise it comes from the library's pool
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(st, &cap);
  if (e != cudaSuccess) return HSMA_ERR_CUDA;
  int dev = 0;
  cudaMemPool_t pool = nullptr;
  if (cap == cudaStreamCaptureStatusNone && cudaGetDevice(&dev) == cudaSuccess) pool = library_pool(dev);
  e = pool != nullptr ? cudaMallocFromPoolAsync(p, bytes, pool, st) : cudaMallocAsync(p, bytes, st);
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
