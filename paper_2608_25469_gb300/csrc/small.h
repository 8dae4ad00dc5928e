// Internal interface of the small-case kernels (small.cu).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/hsma.h"

// One solve with m <= 64 (g = 0: planner choice).  Arguments already validated.
// uplo / trans select the left-side variant (the kernel remaps indices; the
// default is the paper's left / lower / no-transpose case).
hsma_status_t hsma_small_single(int dtype, int g, const void *A, int64_t lda, void *B, int64_t ldb, int m, int n,
                                const double *alpha, int unit, cudaStream_t st, int uplo = HSMA_LOWER,
                                int trans = HSMA_NO_TRANS);

// Bytes of device scratch the varlen batch needs for `batch` instances.
size_t hsma_vbatched_scratch_bytes(int32_t batch);

// Varlen batch (schedule pre-pass + persistent solve).  `scratch` holds
// hsma_vbatched_scratch_bytes(batch) bytes of device memory.  skip_large:
// instances with m > 64 are skipped without a status bit (the caller solves
// them on the blocked path); otherwise they are flagged HSMA_DEVERR_BAD_SIZE.
hsma_status_t hsma_small_vbatched(int dtype, int32_t batch, const int32_t *dm, const int32_t *dn,
                                  const double *alpha, const void *const *dA, const int32_t *dlda,
                                  void *const *dB, const int32_t *dldb, int unit, uint32_t *status,
                                  int32_t *scratch, cudaStream_t st, int uplo = HSMA_LOWER,
                                  int trans = HSMA_NO_TRANS, int skip_large = 0);

// Varlen batch of factor solves in one launch (schedule pre-pass + fused
// kernel): chol = 0, X = U^{-1} L^{-1} P^T (alpha B) from packed LU factors
// (dipiv may be NULL); chol = 1, X = L^{-H} L^{-1} (alpha B) from a lower
// Cholesky factor (dipiv ignored).
hsma_status_t hsma_small_getrs_vbatched(int dtype, int32_t batch, const int32_t *dm, const int32_t *dn,
                                        const double *alpha, const void *const *dLU, const int32_t *dlda,
                                        const int32_t *const *dipiv, void *const *dB, const int32_t *dldb,
                                        uint32_t *status, int32_t *scratch, cudaStream_t st, int chol = 0,
                                        int skip_large = 0);

// Row interchanges of a varlen batch of LU-factor solves (LAPACK ipiv, one
// pointer per instance, dipiv may be NULL) applied to B ahead of two separate
// triangular-solve launches, and the sizes those launches take: m_eff[b] is
// m_b, or 0 when a pivot of instance b is out of range (flagged
// HSMA_DEVERR_BAD_PIVOT, B untouched).  m_eff: batch int32 of device memory.
hsma_status_t hsma_small_lu_pivots(int dtype, int32_t batch, const int32_t *dm, const int32_t *dn,
                                   const int32_t *dlda, const int32_t *dldb, const void *const *dA,
                                   void *const *dB, const int32_t *const *dipiv, int32_t *m_eff, uint32_t *status,
                                   cudaStream_t st);

// Column-packed varlen batch for the left / lower / no-transpose solve in
// HSMA_C128 (packed.cu): schedule, prep and solve passes (a_packed: every A_i
// is in LAPACK's packed lower storage, column c holding rows c .. m_i - 1, and
// dlda is only validated, as for a square layout; uplo / trans select the
// left-side variant through the per-instance kernel's index map, identity
// only with a_packed);
// `scratch` holds hsma_vbatched_packed_scratch_bytes(dtype, batch, max_m)
// bytes (max_m: a bound on every m_i, 0 = 64; above 64, instances with
// m > 64 are skipped without a status bit, as skip_large below).  Results
// equal hsma_small_vbatched's bit for bit.
size_t hsma_vbatched_packed_scratch_bytes(int dtype, int32_t batch, int32_t max_m);
// dtypes whose varlen batch runs the column-packed kernels (measured faster
// than the per-instance kernel: complex128; real FP64 keeps the per-instance
// kernel, whose G choice already fills its lanes at 4x less work per element,
// and so does complex64, where the packed form ran at 2890 against 4800
// GFLOP/s: FP32 arithmetic is cheap, and the triangle reads through the
// caches cost more than the per-instance kernel's shared-memory staging)
inline bool hsma_vbatched_packed_dtype(int dtype) { return dtype == HSMA_C128; }
hsma_status_t hsma_small_vbatched_packed(int dtype, int32_t batch, int32_t max_m, const int32_t *dm,
                                         const int32_t *dn, const double *alpha, const void *const *dA,
                                         const int32_t *dlda, void *const *dB, const int32_t *dldb, int unit,
                                         uint32_t *status, void *scratch, cudaStream_t st, int a_packed = 0,
                                         int uplo = HSMA_LOWER, int trans = HSMA_NO_TRANS);

// dtypes the small kernels and the varlen batch handle
inline bool hsma_small_dtype(int dtype) {
  return dtype == HSMA_R64 || dtype == HSMA_C128 || dtype == HSMA_R32 || dtype == HSMA_C64;
}

// element size in bytes of a small-path dtype
inline int hsma_small_esize(int dtype) { return (dtype == HSMA_C128) ? 16 : (dtype == HSMA_R32 ? 4 : 8); }
