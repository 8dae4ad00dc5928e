// The other BLAS triangular-solve variants (side, uplo, trans) by index
// remapping onto the left / lower / no-transpose solve (the paper's case).
//
// Let T be the triangular matrix the solve applies: T = op(A) for the left
// side (op(A) X = alpha B), T = op(A)^T for the right side (X op(A) = alpha B
// is op(A)^T X^T = alpha B^T).  With r the identity when T is lower triangular
// and the row reversal i -> mE-1-i when it is upper, L(i,k) = T(r(i), r(k)) is
// lower triangular, and L Y = alpha B' with B'(i,j) = B(r(i), j) (left) or
// B(j, r(i)) (right) gives X by the inverse map.  L and B' are gathered into
// workspace (only the referenced triangle of A is read), the left / lower /
// no-transpose solve runs on them, and X is scattered back into B.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "../../include/hsma.h"
#include "common.cuh"
#include "small.h"
#include "trace.h"
#include "workspace.h"

namespace {

template <class T>
__device__ __forceinline__ T conj_of(T v) {
  if constexpr (Elem<T>::kComplex) v.im = -v.im;
  return v;
}

// L (mE x mE, ld mE): L(i,k) = T(r(i), r(k)) below and on the diagonal, 0 above.
// T(p,q) = A(p,q) or, with tsrc, A(q,p); conjugated with cj.
template <class T>
__global__ void remap_a_kernel(const T *__restrict__ A, int64_t lda, int64_t mE, int rev, int tsrc, int cj, T *L) {
  HSMA_FOR_RC(i, k, mE, mE) {
    const int64_t e = i + k * mE;
    if (i < k) {
      L[e] = Elem<T>::zero();
      continue;
    }
    const int64_t p = rev ? mE - 1 - i : i, q = rev ? mE - 1 - k : k;
    T v = tsrc ? A[q + p * lda] : A[p + q * lda];
    L[e] = cj ? conj_of(v) : v;
  }
}

// B' (mE x nE, ld mE) and B: B'(i,j) = B(r(i), j) (left) or B(j, r(i)) (right);
// scatter writes B from B'.
template <class T>
__global__ void remap_b_kernel(T *B, int64_t ldb, T *Bp, int64_t mE, int64_t nE, int rev, int right, int scatter) {
  HSMA_FOR_RC(i, j, mE, nE) {
    const int64_t e = i + j * mE;
    const int64_t p = rev ? mE - 1 - i : i;
    T *b = right ? B + j + p * ldb : B + p + j * ldb;
    if (scatter)
      *b = Bp[e];
    else
      Bp[e] = *b;
  }
}

template <class T>
hsma_status_t variant_impl(int dtype, int side, int uplo, int trans, int diag, int64_t m, int64_t n,
                           const void *alpha, const T *A, int64_t lda, T *B, int64_t ldb, cudaStream_t st,
                           const hsma_opts_t *opts, hsma_info_t *info) {
  const bool right = side == HSMA_RIGHT;
  const int64_t mE = right ? n : m, nE = right ? m : n;
  const bool op_lower = (uplo == HSMA_LOWER) != (trans != HSMA_NO_TRANS);
  const bool t_lower = right ? !op_lower : op_lower;  // right: T = op(A)^T
  const int rev = t_lower ? 0 : 1;
  // T(p,q) from A: left T = op(A): transposed source when op transposes;
  // right T = op(A)^T: transposed source when op does not transpose
  const int tsrc = right ? (trans == HSMA_NO_TRANS) : (trans != HSMA_NO_TRANS);
  const int cj = trans == HSMA_CONJ_TRANS && Elem<T>::kComplex;
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  const size_t l_b = al(sizeof(T) * (size_t)mE * mE), b_b = al(sizeof(T) * (size_t)mE * nE);
  void *ws = nullptr;
  hsma_status_t s = hsma_ws_alloc(&ws, l_b + b_b, st);
  if (s != HSMA_OK) return s;
  T *L = static_cast<T *>(ws);
  T *Bp = reinterpret_cast<T *>(static_cast<unsigned char *>(ws) + l_b);
  {
    HsmaTraceScope ts("remap", st, 2);
    remap_a_kernel<T><<<hsma_grid_rc(mE, mE), 256, 0, st>>>(A, lda, mE, rev, tsrc, cj, L);
    remap_b_kernel<T><<<hsma_grid_rc(mE, nE), 256, 0, st>>>(B, ldb, Bp, mE, nE, rev, right ? 1 : 0, 0);
    s = hsma_from_cuda(cudaGetLastError());
  }
  if (s == HSMA_OK) s = hsma_trsm_llnn_ex(dtype, diag, mE, nE, alpha, L, mE, Bp, mE, st, opts, info);
  if (s == HSMA_OK) {
    HsmaTraceScope ts("remap", st);
    remap_b_kernel<T><<<hsma_grid_rc(mE, nE), 256, 0, st>>>(B, ldb, Bp, mE, nE, rev, right ? 1 : 0, 1);
    s = hsma_from_cuda(cudaGetLastError());
  }
  hsma_status_t f = hsma_ws_free(ws, st);
  return s != HSMA_OK ? s : f;
}

}  // namespace

extern "C" HSMA_API hsma_status_t hsma_trsm(int dtype, int side, int uplo, int trans, int diag, int64_t m, int64_t n,
                                            const void *alpha, const void *A, int64_t lda, void *B, int64_t ldb,
                                            void *stream, const hsma_opts_t *opts, hsma_info_t *info) {
  if (dtype < HSMA_R64 || dtype > HSMA_C64) return HSMA_ERR_INVALID_ARG;
  if ((side != HSMA_LEFT && side != HSMA_RIGHT) || (uplo != HSMA_LOWER && uplo != HSMA_UPPER) ||
      trans < HSMA_NO_TRANS || trans > HSMA_CONJ_TRANS || (diag != HSMA_NON_UNIT && diag != HSMA_UNIT))
    return HSMA_ERR_INVALID_ARG;
  const int64_t na = side == HSMA_LEFT ? m : n;
  if (m < 0 || n < 0 || lda < std::max<int64_t>(1, na) || ldb < std::max<int64_t>(1, m)) return HSMA_ERR_INVALID_ARG;
  if (side == HSMA_LEFT && uplo == HSMA_LOWER && trans == HSMA_NO_TRANS)
    return hsma_trsm_llnn_ex(dtype, diag, m, n, alpha, A, lda, B, ldb, stream, opts, info);
  if (m == 0 || n == 0) return HSMA_OK;
  if (alpha == nullptr || A == nullptr || B == nullptr) return HSMA_ERR_INVALID_ARG;
  const double *a = static_cast<const double *>(alpha);
  const bool cx = dtype == HSMA_C128 || dtype == HSMA_C64;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (a[0] == 0.0 && (!cx || a[1] == 0.0)) {  // B := 0, A not referenced
    const size_t eb = dtype == HSMA_C128 ? 16 : ((dtype == HSMA_R32 || dtype == HSMA_R32_BF16) ? 4 : 8);
    HSMA_CUDA_TRY(cudaMemset2DAsync(B, (size_t)ldb * eb, 0, (size_t)m * eb, (size_t)n, st));
    return HSMA_OK;
  }
  // left side, m <= 64: the small kernels remap indices themselves (no copies)
  const bool small_path = side == HSMA_LEFT && m <= 64 && hsma_small_dtype(dtype) &&
                          (opts == nullptr || opts->path != HSMA_PATH_BLOCKED);
  if (small_path) {
    if (info) {
      std::memset(info, 0, sizeof(*info));
      info->plan.path = HSMA_PATH_SMALL;
    }
    return hsma_small_single(dtype, 0, A, lda, B, ldb, (int)m, (int)n, a, diag == HSMA_UNIT, st, uplo, trans);
  }
  switch (dtype) {
    case HSMA_C128:
      return variant_impl<cplx>(dtype, side, uplo, trans, diag, m, n, alpha, static_cast<const cplx *>(A), lda,
                                static_cast<cplx *>(B), ldb, st, opts, info);
    case HSMA_C64:
      return variant_impl<cplxf>(dtype, side, uplo, trans, diag, m, n, alpha, static_cast<const cplxf *>(A), lda,
                                 static_cast<cplxf *>(B), ldb, st, opts, info);
    case HSMA_R32:
    case HSMA_R32_BF16:
      return variant_impl<float>(dtype, side, uplo, trans, diag, m, n, alpha, static_cast<const float *>(A), lda,
                                 static_cast<float *>(B), ldb, st, opts, info);
    default:
      return variant_impl<double>(dtype, side, uplo, trans, diag, m, n, alpha, static_cast<const double *>(A), lda,
                                  static_cast<double *>(B), ldb, st, opts, info);
  }
}
