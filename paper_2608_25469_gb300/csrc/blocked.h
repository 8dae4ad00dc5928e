// Internal interface of the blocked large-case path (blocked.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/hsma.h"

// Blocked two-phase solve (Section 4.3) for HSMA_R64 / HSMA_C128 with
// diagonal block size nb.  Arguments already validated; alpha != 0.
hsma_status_t hsma_blocked_solve(int dtype, int nb, const void *A, int64_t lda, void *B, int64_t ldb, int64_t m,
                                 int64_t n, const double *alpha, int unit, cudaStream_t st);
