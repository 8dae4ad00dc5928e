// Internal workspace allocation: CUDA's stream-ordered allocator, from a
// per-device pool owned by the library that keeps up to 4 GiB of freed
// workspace reserved between calls (the device's default pool under stream
// capture), with a host-side fault injector for tests (HSMA_FAULT_ALLOC_AFTER=N makes every
// allocation after the first N fail with HSMA_ERR_NO_MEMORY).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "../../include/hsma.h"

hsma_status_t hsma_ws_alloc(void **p, size_t bytes, cudaStream_t st);
hsma_status_t hsma_ws_free(void *p, cudaStream_t st);
