// Internal interface of the reduced-precision modes (mixed.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/hsma.h"

// FP32-result solve with BF16 tensor-core trailing updates (FP32 accumulate).
hsma_status_t hsma_mixed_r32(int nb, int bf16_terms, const float *A, int64_t lda, float *B, int64_t ldb, int64_t m,
                             int64_t n, double alpha, int unit, cudaStream_t st);

// FP64-result solve: FP32-result solve plus FP64 iterative refinement.
hsma_status_t hsma_mixed_ir(int nb, const hsma_opts_t *opts, const double *A, int64_t lda, double *B, int64_t ldb,
                            int64_t m, int64_t n, double alpha, int unit, cudaStream_t st, hsma_info_t *info);

// Blocked FP64 / complex FP64 solve with the solve and trailing-update
// products emulated in FP64 on the BF16 tensor cores (exact integer slices);
// trailing updates are applied per panel of about panel_cols real columns.
hsma_status_t hsma_blocked_emulated(int dtype, int nb, int panel_cols, const void *A, int64_t lda, void *B,
                                    int64_t ldb, int64_t m, int64_t n, const double *alpha, int unit,
                                    cudaStream_t st);

// Device workspace hsma_blocked_emulated takes from the pool (bytes).
size_t hsma_blocked_emulated_ws_bytes(int dtype, int nb, int panel_cols, int64_t m, int64_t n);

// N_B and panel width of the emulated blocked path when neither the caller
// nor the table gives them.
constexpr int kHsmaEmulatedNb = 512;
constexpr int kEmuPanelColsDefault = 2048;

// Table key of the emulated-products configuration of dtype (R64 or C128).
constexpr int kEmulatedTableDtype(int dtype) { return dtype + 10; }

// complex64 blocked solve (m > 64): widened to complex128, solved with emulated
// FP64 products, rounded back into B.
hsma_status_t hsma_c64_blocked(int nb, int panel_cols, const void *A, int64_t lda, void *B, int64_t ldb, int64_t m,
                               int64_t n, const double *alpha, int unit, cudaStream_t st);

// The planner's choice for one solve with the given options (hsma_plan with
// opts; api.cu).
// FP32 inverses of the nb x nb diagonal blocks of L (m x m, lda) into Dinv
// (ceil(m / nb) blocks of nb x nb, ld nb, zeros above each diagonal and
// outside a partial block): 64 x 64 blocks by substitution, joined by doubling
// when nb is a power of two >= 128 (r32_inverse.cu), else substitution at nb.
hsma_status_t hsma_r32_diag_inverse(int nb, const float *A, int64_t lda, int64_t m, int unit, float *Dinv,
                                    cudaStream_t st);

hsma_status_t hsma_make_plan(int dtype, int64_t m, int64_t n, const hsma_opts_t *opts, hsma_plan_t *out);
