// Internal interface of the blocked large-case path (blocked.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/hsma.h"

// Configuration of the blocked path: diagonal block size, FP64 product tile
// shape (HSMA_TILE_*; 0 = by n), split K (HSMA_SPLITK_*) and the update
// direction (HSMA_LOOK_*), as the planner picks them.
struct HsmaBlockedCfg {
  int nb = 256;
  int tile = 0;
  int split_k = HSMA_SPLITK_AUTO;
  int looking = HSMA_LOOK_RIGHT;
};

// Blocked two-phase solve (Section 4.3) for HSMA_R64 / HSMA_C128.  Arguments
// already validated; alpha != 0.
hsma_status_t hsma_blocked_solve(int dtype, const HsmaBlockedCfg &cfg, const void *A, int64_t lda, void *B,
                                 int64_t ldb, int64_t m, int64_t n, const double *alpha, int unit, cudaStream_t st);

// Phase 1 alone: invert the N_B x N_B diagonal blocks of the lower triangle of
// A (dtype HSMA_R64, HSMA_C128 or HSMA_R32_BF16 for float data) into Dinv
// (ceil(m/nb) blocks of nb x nb, column-major, ld nb, zeros above the diagonal
// and outside a partial last block).  nb in {32, 64, 128, 256, 512}.
hsma_status_t hsma_diag_inverse(int dtype, int nb, const void *A, int64_t lda, int64_t m, int unit, void *Dinv,
                                cudaStream_t st);

// FP64 product used by the refinement residual: C = beta*C - L*X with L the
// lower triangle of A (unit diagonal if unit), all column-major fp64 (m x m,
// m x n).  If skip is non-NULL and *skip != 0 on the device, the launch does
// nothing.
hsma_status_t hsma_residual_f64(const double *A, int64_t lda, int unit, const double *X, int64_t ldx, double *C,
                                int64_t ldc, int64_t m, int64_t n, double beta, const int *skip, cudaStream_t st);

// Device address (current device) of the library's device error word, whose
// HSMA_DEVERR_* bits kernels raise; NULL on a CUDA error.
unsigned int *hsma_dev_error_ptr();

// SMs of the current device (cached per device); kHsmaDefaultSms (a GB300's
// 152) when no device can be queried, e.g. for host-only plan queries.
constexpr int kHsmaDefaultSms = 152;
int hsma_sm_count();
