// Solves with LU and Cholesky factors for one system of any size: the row
// interchanges (LU), then the two triangular solves through hsma_trsm, which
// picks the small kernel (index-mapped) or the blocked path per solve.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/hsma.h"
#include "blocked.h"
#include "common.cuh"
#include "trace.h"
#include "workspace.h"

namespace {

// Largest m whose pivots and permutation fit the shared memory of one CTA.
constexpr int64_t kPermSmemMax = 28000;

// perm[r] = the row of B that row r of P^T B takes, from LAPACK's sequential
// interchanges (row k with row ipiv[k]-1, k = 0..m-1).  One CTA: the pivots
// are loaded cooperatively, one thread applies the interchanges in order.  A
// pivot outside [k, m) raises HSMA_DEVERR_BAD_PIVOT and leaves perm as the
// identity.
__global__ void build_perm_kernel(const int32_t *__restrict__ ipiv, int64_t m, int32_t *perm, unsigned int *err) {
  extern __shared__ int32_t sh[];
  const bool in_smem = m <= kPermSmemMax;
  int32_t *piv = in_smem ? sh : nullptr;
  int32_t *p = in_smem ? sh + m : perm;
  for (int64_t k = threadIdx.x; k < m; k += blockDim.x) {
    if (in_smem) piv[k] = ipiv[k] - 1;
    p[k] = (int32_t)k;
  }
  __syncthreads();
  __shared__ int bad;
  if (threadIdx.x == 0) {
    bad = 0;
    for (int64_t k = 0; k < m; ++k) {
      const int64_t q = in_smem ? piv[k] : (int64_t)ipiv[k] - 1;
      if (q < k || q >= m) {
        bad = 1;
        break;
      }
      const int32_t t = p[k];
      p[k] = p[q];
      p[q] = t;
    }
    if (bad && err != nullptr) atomicOr(err, HSMA_DEVERR_BAD_PIVOT);
  }
  __syncthreads();
  for (int64_t k = threadIdx.x; k < m; k += blockDim.x) {
    if (bad)
      perm[k] = (int32_t)k;
    else if (in_smem)
      perm[k] = p[k];
  }
}

// W(r, j) = B(perm[r], j)
template <class T>
__global__ void gather_rows_kernel(const T *__restrict__ B, int64_t ldb, const int32_t *__restrict__ perm, int64_t m,
                                   int64_t n, T *W) {
  HSMA_FOR_RC(r, j, m, n) W[r + j * m] = B[perm[r] + j * ldb];
}

template <class T>
hsma_status_t permute_rows(const int32_t *ipiv, int64_t m, int64_t n, T *B, int64_t ldb, cudaStream_t st) {
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  const size_t perm_b = al(sizeof(int32_t) * (size_t)m), w_b = al(sizeof(T) * (size_t)m * n);
  void *ws = nullptr;
  hsma_status_t s = hsma_ws_alloc(&ws, perm_b + w_b, st);
  if (s != HSMA_OK) return s;
  int32_t *perm = static_cast<int32_t *>(ws);
  T *W = reinterpret_cast<T *>(static_cast<unsigned char *>(ws) + perm_b);
  {
    HsmaTraceScope ts("interchange", st, 2);
    const size_t smem = m <= kPermSmemMax ? sizeof(int32_t) * 2 * (size_t)m : 0;
    static DeviceFlags attr;
    if (!attr.test()) {
      cudaError_t e = cudaFuncSetAttribute(build_perm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)(sizeof(int32_t) * 2 * kPermSmemMax));
      if (e != cudaSuccess) s = hsma_from_cuda(e);
      attr.set();
    }
    if (s == HSMA_OK) {
      build_perm_kernel<<<1, 1024, smem, st>>>(ipiv, m, perm, hsma_dev_error_ptr());
      gather_rows_kernel<T><<<hsma_grid_rc(m, n), 256, 0, st>>>(B, ldb, perm, m, n, W);
      s = hsma_from_cuda(cudaGetLastError());
    }
    if (s == HSMA_OK)
      s = hsma_from_cuda(cudaMemcpy2DAsync(B, sizeof(T) * ldb, W, sizeof(T) * m, sizeof(T) * m, n,
                                           cudaMemcpyDeviceToDevice, st));
  }
  hsma_status_t f = hsma_ws_free(ws, st);
  return s != HSMA_OK ? s : f;
}

hsma_status_t check_common(int dtype, int64_t m, int64_t n, int64_t lda, int64_t ldb) {
  if (dtype < HSMA_R64 || dtype > HSMA_C64) return HSMA_ERR_INVALID_ARG;
  if (m < 0 || n < 0 || lda < std::max<int64_t>(1, m) || ldb < std::max<int64_t>(1, m)) return HSMA_ERR_INVALID_ARG;
  return HSMA_OK;
}

}  // namespace

extern "C" HSMA_API hsma_status_t hsma_getrs(int dtype, int64_t m, int64_t n, const void *alpha, const void *LU,
                                             int64_t lda, const int32_t *ipiv, void *B, int64_t ldb, void *stream,
                                             const hsma_opts_t *opts) {
  hsma_status_t s = check_common(dtype, m, n, lda, ldb);
  if (s != HSMA_OK) return s;
  if (m == 0 || n == 0) return HSMA_OK;
  if (alpha == nullptr || LU == nullptr || B == nullptr) return HSMA_ERR_INVALID_ARG;
  if (m > INT32_MAX) return HSMA_ERR_UNSUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (ipiv != nullptr) {
    switch (dtype) {
      case HSMA_C128: s = permute_rows<cplx>(ipiv, m, n, static_cast<cplx *>(B), ldb, st); break;
      case HSMA_C64: s = permute_rows<cplxf>(ipiv, m, n, static_cast<cplxf *>(B), ldb, st); break;
      case HSMA_R32:
      case HSMA_R32_BF16: s = permute_rows<float>(ipiv, m, n, static_cast<float *>(B), ldb, st); break;
      default: s = permute_rows<double>(ipiv, m, n, static_cast<double *>(B), ldb, st); break;
    }
    if (s != HSMA_OK) return s;
  }
  const double one[2] = {1.0, 0.0};
  s = hsma_trsm(dtype, HSMA_LEFT, HSMA_LOWER, HSMA_NO_TRANS, HSMA_UNIT, m, n, alpha, LU, lda, B, ldb, stream, opts,
                nullptr);
  if (s != HSMA_OK) return s;
  return hsma_trsm(dtype, HSMA_LEFT, HSMA_UPPER, HSMA_NO_TRANS, HSMA_NON_UNIT, m, n, one, LU, lda, B, ldb, stream,
                   opts, nullptr);
}

extern "C" HSMA_API hsma_status_t hsma_potrs(int dtype, int64_t m, int64_t n, const void *alpha, const void *L,
                                             int64_t lda, void *B, int64_t ldb, void *stream,
                                             const hsma_opts_t *opts) {
  hsma_status_t s = check_common(dtype, m, n, lda, ldb);
  if (s != HSMA_OK) return s;
  if (m == 0 || n == 0) return HSMA_OK;
  if (alpha == nullptr || L == nullptr || B == nullptr) return HSMA_ERR_INVALID_ARG;
  const bool cx = dtype == HSMA_C128 || dtype == HSMA_C64;
  const double one[2] = {1.0, 0.0};
  s = hsma_trsm(dtype, HSMA_LEFT, HSMA_LOWER, HSMA_NO_TRANS, HSMA_NON_UNIT, m, n, alpha, L, lda, B, ldb, stream, opts,
                nullptr);
  if (s != HSMA_OK) return s;
  return hsma_trsm(dtype, HSMA_LEFT, HSMA_LOWER, cx ? HSMA_CONJ_TRANS : HSMA_TRANS, HSMA_NON_UNIT, m, n, one, L, lda,
                   B, ldb, stream, opts, nullptr);
}
