// Internal interface of the device input generator (gen.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/hsma.h"

hsma_status_t hsma_gen_launch(int dtype, int kind, uint64_t seed, int64_t inst, int64_t m, int64_t cols, void *dst,
                              int64_t ld, cudaStream_t st);
