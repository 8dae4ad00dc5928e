// Reduced-precision modes of the blocked solve (the paper lists mixed
// precision as future work, Section 6; the blocked algorithm is Section 4.3),
// and FP64 products emulated on the BF16 tensor cores.
//
// FP32-result mode (HSMA_R32_BF16): phase 1 inverts the diagonal blocks in
// FP32; phase 2 forms X_r = D_r^{-1} B_r and applies the trailing update
// B_{r+1:} -= A_{r+1:,r} X_r on the 5th-generation tensor cores: operands in
// BF16, products accumulated in FP32 in tensor memory (tcgen05.mma kind::f16,
// 128 x 256 tiles, TMA loads with 128-byte swizzle).  The solve product cuts
// both operands into three BF16 slices (24 significant bits, exact for FP32)
// and sums the six slice pairs with p + q <= 2 in one accumulator (the
// refinement's correction solves use FP32 FMAs instead).  With three
// terms per update the operands are split, a = hi(a) + lo(a), and the products
// hi*hi + hi*lo + lo*hi are accumulated in one pass by concatenating along K:
// [A_hi A_hi A_lo] [X_hi; X_lo; X_hi].
//
// FP64-result mode (HSMA_R64_IR): X_0 from the FP32-result solve of the
// rounded data, then iterative refinement: R = alpha B - L X in FP64 (emulated
// on the tensor cores, below, or FP64 tensor products), C from the FP32-result
// solve of L C = R, X += C in FP64, until
// ||R||_F / (||L||_F ||X||_F + |alpha| ||B||_F) <= tol.  Every refinement
// kernel checks a device-side "converged" flag first, so the host enqueues the
// maximum number of steps without waiting on the device.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <type_traits>

#include "blocked.h"
#include "common.cuh"
#include "mixed.h"
#include "tma.cuh"
#include "trace.h"
#include "workspace.h"

#include "tc_gemm.cuh"

namespace {

// ---------------------------------------------------------------------------
// FP32 products on the CUDA cores: C = beta*(A*B), A optionally lower
// triangular (row tile i0 reads k < i0 + 128 only).  128 x 128 tiles, 8 x 8
// outputs per thread, K slices of 8 staged in shared memory double-buffered
// (the next slice is read from global memory into registers while the
// current one is used).
// ---------------------------------------------------------------------------
constexpr int SG_BM = 128, SG_BN = 128, SG_BK = 8;

__global__ void __launch_bounds__(256) sgemm_scale_kernel(const float *__restrict__ A, int64_t lda,
                                                          const float *__restrict__ Bm, int64_t ldb, float *C,
                                                          int64_t ldc, int M, int N, int K, float beta, int tri,
                                                          const int *skip) {
  if (skip != nullptr && *(volatile const int *)skip) return;
  __shared__ __align__(16) float sA[2][SG_BK][SG_BM];
  __shared__ __align__(16) float sB[2][SG_BK][SG_BN];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int m0 = blockIdx.x * SG_BM, n0 = blockIdx.y * SG_BN;
  const int kend = tri ? min(K, m0 + SG_BM) : K;
  // loader mapping: A slice 8 x 128 (k, m): thread -> (k = tid / 32, m = 4 * (tid % 32) .. +3)
  //                 B slice 8 x 128 (k, n): thread -> (n = tid / 2, k = 4 * (tid % 2) .. +3)
  const int ak = tid / 32, am = 4 * (tid % 32);
  const int bn = tid / 2, bk = 4 * (tid % 2);
  float ra[4], rb[4];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int row = m0 + am + u, col = k0 + ak;
      ra[u] = (row < M && col < kend) ? __ldg(A + row + (int64_t)col * lda) : 0.0f;
      const int kr = k0 + bk + u, cn = n0 + bn;
      rb[u] = (kr < kend && cn < N) ? __ldg(Bm + kr + (int64_t)cn * ldb) : 0.0f;
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      sA[buf][ak][am + u] = ra[u];
      sB[buf][bk + u][bn] = rb[u];
    }
  };
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
  const int nk = (kend + SG_BK - 1) / SG_BK;
  if (nk > 0) {
    fetch(0);
    store(0);
  }
  __syncthreads();
  for (int kt = 0; kt < nk; ++kt) {
    const int cur = kt & 1;
    if (kt + 1 < nk) fetch((kt + 1) * SG_BK);
#pragma unroll
    for (int kk = 0; kk < SG_BK; ++kk) {
      float a[8], b[8];
      const float4 a0 = *reinterpret_cast<const float4 *>(&sA[cur][kk][tx * 4]);
      const float4 a1 = *reinterpret_cast<const float4 *>(&sA[cur][kk][64 + tx * 4]);
      const float4 b0 = *reinterpret_cast<const float4 *>(&sB[cur][kk][ty * 4]);
      const float4 b1 = *reinterpret_cast<const float4 *>(&sB[cur][kk][64 + ty * 4]);
      a[0] = a0.x; a[1] = a0.y; a[2] = a0.z; a[3] = a0.w; a[4] = a1.x; a[5] = a1.y; a[6] = a1.z; a[7] = a1.w;
      b[0] = b0.x; b[1] = b0.y; b[2] = b0.z; b[3] = b0.w; b[4] = b1.x; b[5] = b1.y; b[6] = b1.z; b[7] = b1.w;
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (kt + 1 < nk) store(cur ^ 1);
    __syncthreads();
  }
  // thread rows: tx*4 .. +3 and 64 + tx*4 .. +3; columns: ty*4 .. +3 and 64 + ty*4 .. +3
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int col = n0 + (j < 4 ? ty * 4 + j : 64 + ty * 4 + (j - 4));
    if (col >= N) continue;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int row = m0 + (i < 4 ? tx * 4 + i : 64 + tx * 4 + (i - 4));
      if (row < M) C[row + (int64_t)col * ldc] = beta * acc[i][j];
    }
  }
}

// ---------------------------------------------------------------------------
// Conversions to the tensor-core operand layouts (split_bf16 / split3_bf16
// come from tc_gemm.cuh, whose FP32-result epilogue writes the same splits).
// ---------------------------------------------------------------------------
// A panel (rows x nb, column-major fp32, lda) -> A' rows x Kp row-major BF16:
// terms 1: [hi], terms 3: [hi | hi | lo]; columns past terms*nb are zero.
// One 32 x 32 tile (rows i0.., columns k0..) per CTA of 256 threads.
// A tile of 32 rows x kPanelTileK columns of the panel: read as 32 columns
// of 32 consecutive rows (128-byte loads), written as BF16 pairs of
// consecutive K (128-byte stores; nb is even).
constexpr int kPanelTileK = 64;
__device__ __forceinline__ void convert_panel_tile(const float *__restrict__ A, int64_t lda, int rows, int nb,
                                                   int terms, int Kp, __nv_bfloat16 *out, int i0, int k0) {
  __shared__ float tile[kPanelTileK][33];
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
  for (int kk = ty; kk < kPanelTileK; kk += 8) {
    const int i = i0 + tx, k = k0 + kk;
    tile[kk][tx] = (i < rows && k < nb) ? A[i + (int64_t)k * lda] : 0.0f;
  }
  __syncthreads();
  const int k = k0 + 2 * tx;  // this lane's pair of K values
  for (int ii = ty; ii < 32; ii += 8) {
    const int i = i0 + ii;
    if (i >= rows) continue;
    __nv_bfloat16 *o = out + (int64_t)i * Kp;
    if (k < nb) {
      __nv_bfloat16 h0, l0, h1, l1;
      split_bf16(tile[2 * tx][ii], h0, l0);
      split_bf16(tile[2 * tx + 1][ii], h1, l1);
      const __nv_bfloat162 hi = __halves2bfloat162(h0, h1), lo = __halves2bfloat162(l0, l1);
      *reinterpret_cast<__nv_bfloat162 *>(o + k) = hi;
      if (terms == 3) {
        *reinterpret_cast<__nv_bfloat162 *>(o + nb + k) = hi;
        *reinterpret_cast<__nv_bfloat162 *>(o + 2 * nb + k) = lo;
      }
    }
    // zero padding columns [terms*nb, Kp)
    for (int kp = terms * nb + 2 * tx; kp < Kp && k0 == 0; kp += 64)
      *reinterpret_cast<__nv_bfloat162 *>(o + kp) = __floats2bfloat162_rn(0.0f, 0.0f);
  }
}

__global__ void __launch_bounds__(256) convert_panel_kernel(const float *__restrict__ A, int64_t lda, int rows,
                                                            int nb, int terms, int Kp, __nv_bfloat16 *out) {
  convert_panel_tile(A, lda, rows, nb, terms, Kp, out, blockIdx.x * 32, blockIdx.y * kPanelTileK);
}

// Every step's panel in one launch (blockIdx.z = step r < nblk - 1, whose
// diagonal block is full): rows m - (r+1) nb below the block, stored at
// element offset (r m - nb r (r+1) / 2) Kp, the sum of the earlier panels.
__global__ void __launch_bounds__(256) convert_panels_kernel(const float *__restrict__ A, int64_t lda, int64_t m,
                                                             int nb, int terms, int Kp, __nv_bfloat16 *panels) {
  const int64_t r = blockIdx.z, r0 = r * nb;
  const int rows = (int)(m - r0 - nb);
  const int i0 = blockIdx.x * 32;
  if (i0 >= rows) return;  // uniform over the CTA
  const int64_t off = (r * m - (int64_t)nb * r * (r + 1) / 2) * Kp;
  convert_panel_tile(A + (r0 + nb) + r0 * lda, lda, rows, nb, terms, Kp, panels + off, i0,
                     blockIdx.y * kPanelTileK);
}

// X_r (nb x n, column-major fp32, ldx) -> X' n x Kp row-major BF16:
// terms 1: [hi], terms 3: [hi | lo | hi]; zero padding to Kp.
__global__ void __launch_bounds__(256) convert_x_kernel(const float *__restrict__ X, int64_t ldx, int nb, int n,
                                                        int terms, int Kp, __nv_bfloat16 *out, const int *skip) {
  if (skip != nullptr && *(volatile const int *)skip) return;
  // rows: k within one part (plus the zero tail), columns: j
  HSMA_FOR_RC(k, j, nb, n) {
    const float x = X[k + j * ldx];
    __nv_bfloat16 hi, lo;
    split_bf16(x, hi, lo);
    __nv_bfloat16 *o = out + j * Kp + k;
    o[0] = hi;
    if (terms == 3) {
      o[nb] = lo;
      o[2 * nb] = hi;
    }
  }
  const int tail0 = terms * nb;
  HSMA_FOR_RC(k, j, Kp - tail0, n) out[j * Kp + tail0 + k] = __float2bfloat16_rn(0.0f);
}

int g_launch_grid(int64_t total) {
  int64_t b = (total + 255) / 256;
  return (int)std::min<int64_t>(std::max<int64_t>(b, 1), (int64_t)hsma_sm_count() * 32);
}

hsma_status_t bf16_update(const __nv_bfloat16 *Ap, const __nv_bfloat16 *Bp, int M, int N, int Kp, float beta, float *C,
                          int64_t ldc, cudaStream_t st) {
  TcArgs a{};
  a.C32 = C;
  a.ldc = ldc;
  a.beta = beta;
  a.M = M;
  a.N = N;
  a.K = Kp;
  return tc_gemm<TC_F32>(Ap, 1, Bp, 1, a, "update_bf16", st);
}

hsma_status_t sgemm_scale(const float *A, int64_t lda, const float *Bm, int64_t ldb, float *C, int64_t ldc, int M,
                          int N, int K, float beta, int tri, const int *skip, cudaStream_t st) {
  if (M <= 0 || N <= 0) return HSMA_OK;
  dim3 grid((M + SG_BM - 1) / SG_BM, (N + SG_BN - 1) / SG_BN);
  if (grid.y > 65535) return HSMA_ERR_UNSUPPORTED;
  HsmaTraceScope ts("solve_sgemm", st);
  sgemm_scale_kernel<<<grid, 256, 0, st>>>(A, lda, Bm, ldb, C, ldc, M, N, K, beta, tri, skip);
  HSMA_CUDA_TRY(cudaGetLastError());
  return HSMA_OK;
}

int round_up(int a, int b) { return (a + b - 1) / b * b; }

// Pieces of the FP32-result solve that depend on A only: the FP32 inverses of
// the diagonal blocks and (when kept) the BF16 operand panels of every
// trailing update.  The refinement reuses them for all its corrections.
struct R32Plan {
  int nb = 0, terms = 0, Kp = 0;
  int64_t m = 0;
  const float *A = nullptr;
  int64_t lda = 0;
  int unit = 0;
  float *Dinv = nullptr;
  __nv_bfloat16 *panels = nullptr;  // step r's panel at panel_off(r), rows x Kp; null: converted per step
  // solve products on the tensor cores (the negated inverses cut into three
  // BF16 slices, [block][slice][nb][Kd], row-major, Kd = nb rounded up to 64),
  // else FP32 FMAs on the CUDA cores.  The tensor-core form is faster; its FP32
  // accumulation inside the MMA is less accurate (about ten times the FP32
  // rounding error here), which costs the refinement an extra step, so the
  // FP64-result mode keeps the FP32 FMAs.
  bool tc_solve = false;
  __nv_bfloat16 *dslices = nullptr;
};


int r32_kd(int nb) { return round_up(nb, TC_BK); }

size_t r32_dslices_elems(int nb, int64_t m) { return (size_t)((m + nb - 1) / nb) * 3 * nb * r32_kd(nb); }

// negated three-way slices of every diagonal-block inverse (column-major nb x nb
// blocks, zeros outside the computed part) as out[blk][s][i][k]
__global__ void r32_dslice_kernel(const float *__restrict__ Dinv, int nb, int64_t nblk, int Kd,
                                  __nv_bfloat16 *out) {
  const int64_t per = (int64_t)nb * Kd;
  HSMA_FOR_RC(k, c, Kd, nblk * nb) {
    const int64_t b = c / nb, i = c - b * nb;  // one division per column
    const float v = k < nb ? -Dinv[b * nb * nb + i + k * nb] : 0.0f;
    __nv_bfloat16 x0, x1, x2;
    split3_bf16(v, x0, x1, x2);
    __nv_bfloat16 *o = out + b * 3 * per + i * Kd + k;
    o[0] = x0;
    o[per] = x1;
    o[2 * per] = x2;
  }
}

// three-way slices of scale * W (sr x n, column-major, ld ldw) as
// out[s][j][k] (row-major n x Kd per slice, zero beyond sr)
__global__ void r32_xslice_kernel(const float *__restrict__ W, int64_t ldw, int sr, int64_t n, int Kd, float scale,
                                  __nv_bfloat16 *out, const int *skip) {
  if (skip != nullptr && *(volatile const int *)skip) return;
  const int64_t per = n * Kd;
  HSMA_FOR_RC(k, j, Kd, n) {
    const int64_t e = j * Kd + k;
    const float v = k < sr ? scale * W[k + j * ldw] : 0.0f;
    __nv_bfloat16 x0, x1, x2;
    split3_bf16(v, x0, x1, x2);
    out[e] = x0;
    out[per + e] = x1;
    out[2 * per + e] = x2;
  }
}

int64_t panel_rows(const R32Plan &P, int64_t r) {
  const int64_t r0 = r * P.nb, sr = std::min<int64_t>(P.nb, P.m - r0);
  return std::max<int64_t>(P.m - r0 - sr, 0);
}

size_t panel_off(const R32Plan &P, int64_t r) {
  size_t off = 0;
  for (int64_t q = 0; q < r; ++q) off += (size_t)panel_rows(P, q) * P.Kp;
  return off;
}

size_t r32_panels_elems(int nb, int terms, int64_t m) {
  R32Plan P;
  P.nb = nb;
  P.m = m;
  P.Kp = round_up(terms * nb, TC_BK);
  return panel_off(P, (m + nb - 1) / nb);
}

// copy rows x cols (column-major) unless *skip is set
__global__ void copy_f32_kernel(const float *__restrict__ src, int64_t lds, float *dst, int64_t ldd, int rows,
                                int64_t cols, const int *skip) {
  if (skip != nullptr && *(volatile const int *)skip) return;
  HSMA_FOR_RC(i, j, rows, cols) dst[i + j * ldd] = src[i + j * lds];
}

// Phase 1 of the FP32-result solve: the diagonal-block inverses, their
// slices for the tensor-core solve products, and every update panel converted
// to split BF16 in one launch.
hsma_status_t r32_prepare(R32Plan &P, bool keep_panels, cudaStream_t st) {
  hsma_status_t s = hsma_r32_diag_inverse(P.nb, P.A, P.lda, P.m, P.unit, P.Dinv, st);
  if (s != HSMA_OK) return s;
  const int64_t nblk = (P.m + P.nb - 1) / P.nb;
  HsmaTraceScope ts("convert", st, (P.tc_solve ? 1 : 0) + (keep_panels && nblk >= 2 ? 1 : 0));
  if (P.tc_solve) {
    r32_dslice_kernel<<<hsma_grid_rc(r32_kd(P.nb), nblk * P.nb), 256, 0, st>>>(P.Dinv, P.nb, nblk, r32_kd(P.nb),
                                                                                 P.dslices);
    HSMA_CUDA_TRY(cudaGetLastError());
  }
  if (!keep_panels || nblk < 2) return HSMA_OK;
  if (nblk - 1 > 65535) return HSMA_ERR_UNSUPPORTED;
  const dim3 g((unsigned)((P.m - P.nb + 31) / 32), (unsigned)((P.nb + kPanelTileK - 1) / kPanelTileK),
               (unsigned)(nblk - 1));
  convert_panels_kernel<<<g, 256, 0, st>>>(P.A, P.lda, P.m, P.nb, P.terms, P.Kp, P.panels);
  HSMA_CUDA_TRY(cudaGetLastError());
  return HSMA_OK;
}

// Phase 2 of the FP32-result solve, in place on B (fp32).  Every launch is
// skipped once *skip is set on the device (null: never).
hsma_status_t r32_apply(const R32Plan &P, float *B, int64_t ldb, int64_t n, float alpha, const int *skip,
                        cudaStream_t st) {
  const int nb = P.nb, Kp = P.Kp;
  const int64_t m = P.m, nblk = (m + nb - 1) / nb;
  const int64_t rows_max = std::max<int64_t>(m - nb, 1);
  const size_t w_b = P.tc_solve ? 0 : sizeof(float) * (size_t)nb * n;
  const size_t a_b = P.panels ? 0 : sizeof(__nv_bfloat16) * (size_t)rows_max * Kp;
  // Paired updates (every panel converted up front): after an even block only
  // the next block row takes X_r; after an odd block one product applies
  // X_{r-1} and X_r to every row below (two slice pairs in one accumulator),
  // so the trailing rows of B are read and written once per two blocks.  The
  // two splits live in two buffers.
  const bool pair = P.panels != nullptr;
  const size_t x1_b = sizeof(__nv_bfloat16) * (size_t)n * Kp;
  const size_t x_b = (pair ? 2 : 1) * x1_b;
  const int Kd = r32_kd(nb);
  const size_t x3_b = P.tc_solve ? sizeof(__nv_bfloat16) * 3 * (size_t)n * Kd : 0;
  auto al = [](size_t v) { return (v + 1023) & ~(size_t)1023; };
  void *ws = nullptr;
  hsma_status_t s = hsma_ws_alloc(&ws, al(w_b) + al(a_b) + al(x_b) + al(x3_b), st);
  if (s != HSMA_OK) return s;
  unsigned char *base = static_cast<unsigned char *>(ws);
  float *W = reinterpret_cast<float *>(base);
  __nv_bfloat16 *Ap = reinterpret_cast<__nv_bfloat16 *>(base + al(w_b));
  __nv_bfloat16 *Xp = reinterpret_cast<__nv_bfloat16 *>(base + al(w_b) + al(a_b));
  __nv_bfloat16 *X3 = reinterpret_cast<__nv_bfloat16 *>(base + al(w_b) + al(a_b) + al(x_b));
  // X_r = D_r^{-1} (scale W): slice pairs (p, q) with p + q <= 2 of the three
  // BF16 slices of each operand, summed in one FP32 accumulator
  TcArgs sa{};
  {
    const uint8_t ps[6][2] = {{0, 0}, {0, 1}, {1, 0}, {0, 2}, {1, 1}, {2, 0}};
    sa.nunits = 1;
    sa.ubeg[0] = 0;
    sa.ubeg[1] = 6;
    for (int q = 0; q < 6; ++q) {
      sa.pa[q] = ps[q][0];
      sa.pb[q] = ps[q][1];
    }
  }
  // With the tensor-core solve products, the split of X_r that the update
  // multiplies comes out of the solve product's epilogue, and the slices of
  // the next block row out of the update's (the same values the separate
  // conversion kernels give); the zero tails of both operands are set once.
  if (P.tc_solve) {
    cudaError_t e = cudaMemsetAsync(Xp, 0, x_b, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(X3, 0, x3_b, st);
    if (e != cudaSuccess) s = hsma_from_cuda(e);
  }
  bool x3_ready = false;
  for (int64_t r = 0; r < nblk && s == HSMA_OK; ++r) {
    const int64_t r0 = r * nb;
    const int sr = (int)std::min<int64_t>(nb, m - r0);
    const bool last = r0 + sr >= m;
    if (!P.tc_solve) {
      HsmaTraceScope ts("copy", st);
      copy_f32_kernel<<<hsma_grid_rc(sr, n), 256, 0, st>>>(B + r0, ldb, W, nb, sr, n, skip);
    }
    if (P.tc_solve) {
      // the product reads only the slices, so they are cut from B_r itself
      // (r = 0, or after a partial next block) and X_r is written straight
      // back into B_r
      if (!x3_ready) {
        HsmaTraceScope ts("convert", st);
        r32_xslice_kernel<<<hsma_grid_rc(Kd, n), 256, 0, st>>>(B + r0, ldb, sr, n, Kd, r == 0 ? alpha : 1.0f, X3,
                                                                skip);
        if ((s = hsma_from_cuda(cudaGetLastError())) != HSMA_OK) break;
      }
      sa.xs2 = last ? nullptr : Xp + (pair ? (r & 1) * (int64_t)n * Kp : 0);
      sa.ld2 = Kp;
      sa.nb2 = nb;
      sa.terms2 = P.terms;
      sa.rows2 = sr;
      sa.C32 = B + r0;
      sa.ldc = ldb;
      sa.beta = 0.0f;
      sa.M = sr;
      sa.N = (int)n;
      sa.K = Kd;
      sa.tri = 1;
      sa.skip = skip;
      SliceLayout dl;
      dl.rows = nb;  // the inverse's slices are stored nb rows high
      s = tc_gemm<TC_F32>(P.dslices + (size_t)r * 3 * nb * Kd, 3, X3, 3, sa, "solve_bf16", st, dl);
    } else {
      s = sgemm_scale(P.Dinv + (size_t)r * nb * nb, nb, W, nb, B + r0, ldb, sr, (int)n, sr, r == 0 ? alpha : 1.0f, 1,
                      skip, st);
    }
    if (s != HSMA_OK || last) break;
    const int rows = (int)(m - r0 - sr);
    const __nv_bfloat16 *panel = P.panels ? P.panels + panel_off(P, r) : Ap;
    if (!P.panels || !P.tc_solve) {
      HsmaTraceScope ts("convert", st, (P.panels ? 0 : 1) + (P.tc_solve ? 0 : 1));
      if (!P.panels) {
        dim3 g1((rows + 31) / 32, (nb + kPanelTileK - 1) / kPanelTileK);
        convert_panel_kernel<<<g1, 256, 0, st>>>(P.A + (r0 + sr) + r0 * P.lda, P.lda, rows, nb, P.terms, Kp, Ap);
      }
      if (!P.tc_solve)
        convert_x_kernel<<<hsma_grid_rc(nb, n), 256, 0, st>>>(B + r0, ldb, nb, (int)n, P.terms, Kp,
                                                              Xp + (pair ? (r & 1) * (int64_t)n * Kp : 0), skip);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) {
        s = hsma_from_cuda(e);
        break;
      }
    }
    TcArgs a{};
    // paired: an even block updates its next block row only (the first rows
    // of its panel), an odd one every row below with both blocks' products
    const int upd_rows = pair && (r & 1) == 0 ? (int)std::min<int64_t>(nb, rows) : rows;
    // the next block row's slices for its solve product, when it is a full block
    x3_ready = P.tc_solve && upd_rows >= nb;
    if (x3_ready) {
      a.xs3 = X3;
      a.per3 = n * (int64_t)Kd;
      a.ld3 = Kd;
      a.r3 = 0;
      a.rows3 = nb;
    }
    a.C32 = B + r0 + sr;
    a.ldc = ldb;
    // alpha scales a row block at its first update: block 1 at r = 0, and
    // (paired) the rows below block 1 at r = 1
    a.beta = (r == 0 || (pair && r == 1)) ? alpha : 1.0f;
    a.M = upd_rows;
    a.N = (int)n;
    a.K = Kp;
    a.skip = skip;
    if (pair && (r & 1) == 1) {
      // panel r-1 from its row nb on and panel r cover the same rows, one
      // uniform stride apart; X_{r-1} and X_r sit in the two split buffers
      a.nunits = 1;
      a.ubeg[0] = 0;
      a.ubeg[1] = 2;
      a.pa[0] = 0;
      a.pb[0] = 0;
      a.pa[1] = 1;
      a.pb[1] = 1;
      SliceLayout la, lb;
      la.rows = rows;
      la.kext = Kp;
      la.ld = Kp;
      la.sst = (int64_t)rows * Kp;
      lb.rows = n;
      lb.kext = Kp;
      lb.ld = Kp;
      lb.sst = n * (int64_t)Kp;
      s = tc_gemm<TC_F32>(P.panels + panel_off(P, r - 1) + (size_t)nb * Kp, 2, Xp, 2, a, "update_bf16", st, la,
                          lb);
    } else {
      s = tc_gemm<TC_F32>(panel, 1, Xp + (pair ? (r & 1) * (int64_t)n * Kp : 0), 1, a, "update_bf16", st);
    }
  }
  hsma_status_t f = hsma_ws_free(ws, st);
  return s != HSMA_OK ? s : f;
}

// FP32-result blocked solve in place on B (fp32).  Workspace from the pool.
hsma_status_t r32_solve(int nb, int terms, const float *A, int64_t lda, float *B, int64_t ldb, int64_t m, int64_t n,
                        float alpha, int unit, cudaStream_t st) {
  if (nb < 32) nb = 32;
  R32Plan P;
  P.nb = nb;
  P.terms = terms;
  P.Kp = round_up(terms * nb, TC_BK);
  P.m = m;
  P.A = A;
  P.lda = lda;
  P.unit = unit;
  const int64_t nblk = (m + nb - 1) / nb;
  auto al = [](size_t v) { return (v + 1023) & ~(size_t)1023; };
  const size_t dinv_b = al(sizeof(float) * (size_t)nblk * nb * nb);
  const size_t ds_b = al(sizeof(__nv_bfloat16) * r32_dslices_elems(nb, m));
  // every step's A panel is converted up front, in one launch
  const size_t pan_b = al(sizeof(__nv_bfloat16) * r32_panels_elems(nb, terms, m));
  void *ws = nullptr;
  hsma_status_t s = hsma_ws_alloc(&ws, dinv_b + ds_b + pan_b, st);
  if (s != HSMA_OK) return s;
  P.Dinv = static_cast<float *>(ws);
  P.tc_solve = true;
  P.dslices = reinterpret_cast<__nv_bfloat16 *>(static_cast<unsigned char *>(ws) + dinv_b);
  P.panels = reinterpret_cast<__nv_bfloat16 *>(static_cast<unsigned char *>(ws) + dinv_b + ds_b);
  s = r32_prepare(P, true, st);
  if (s == HSMA_OK) s = r32_apply(P, B, ldb, n, alpha, nullptr, st);
  hsma_status_t f = hsma_ws_free(ws, st);
  return s != HSMA_OK ? s : f;
}

// ---------------------------------------------------------------------------
// Refinement helpers (each returns at once when *flag is set)
// ---------------------------------------------------------------------------
__global__ void f64_to_f32_kernel(const double *__restrict__ src, int64_t lds, float *dst, int64_t ldd, int64_t rows,
                                  int64_t cols, int lower, const int *flag) {
  if (flag != nullptr && *(volatile const int *)flag) return;
  HSMA_FOR_RC(i, j, rows, cols) {
    if (lower && i < j) continue;
    dst[i + j * ldd] = (float)src[i + j * lds];
  }
}

// dst = alpha * src (m x n, both ld m)
__global__ void scale_copy_kernel(const double *__restrict__ src, double *dst, int64_t total, double alpha,
                                  const int *flag) {
  if (flag != nullptr && *(volatile const int *)flag) return;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = alpha * src[e];
}

// X += (double) C   (or X = (double) C when assign)
__global__ void accumulate_kernel(double *X, int64_t ldx, const float *__restrict__ Cc, int64_t ldc, int64_t rows,
                                  int64_t cols, int assign, const int *flag) {
  if (flag != nullptr && *(volatile const int *)flag) return;
  HSMA_FOR_RC(i, j, rows, cols) {
    const double c = (double)Cc[i + j * ldc];
    X[i + j * ldx] = assign ? c : X[i + j * ldx] + c;
  }
}

// sums[slot] += sum of squares (lower triangle only when lower; unit diagonal counts 1)
__global__ void sumsq_kernel(const double *__restrict__ M_, int64_t ld, int64_t rows, int64_t cols, int lower,
                             int unit, double *sums, int slot, const int *flag) {
  if (flag != nullptr && *(volatile const int *)flag) return;
  double acc = 0.0;
  HSMA_FOR_RC(i, j, rows, cols) {
    if (lower && i < j) continue;
    const double v = (lower && unit && i == j) ? 1.0 : M_[i + j * ld];
    acc = fma(v, v, acc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(&sums[slot], acc);
}

// sums: [0] ||L||^2, [1] ||B||^2, [2] ||R||^2, [3] ||X||^2; state: [0] converged, [1] steps, [2..3] eta (double).
// At the last allowed check (last != 0) a refinement that has not reached the
// tolerance raises HSMA_DEVERR_NOT_CONVERGED in the device error word, so the
// failure is visible to callers that do not ask for the info block.
__global__ void check_kernel(double *sums, int *state, double alpha_abs, double tol, int step, int last,
                             unsigned int *err) {
  if (state[0]) return;
  const double nr = sqrt(sums[2]), den = sqrt(sums[0]) * sqrt(sums[3]) + alpha_abs * sqrt(sums[1]);
  const double eta = den > 0.0 ? nr / den : nr;
  *reinterpret_cast<double *>(state + 2) = eta;
  state[1] = step;
  if (eta <= tol) state[0] = 1;
  else if (last && err != nullptr) atomicOr(err, HSMA_DEVERR_NOT_CONVERGED);
  sums[2] = 0.0;
  sums[3] = 0.0;
}

// ---------------------------------------------------------------------------
// FP64 products emulated on the BF16 tensor cores (Ozaki-style exact slices).
//
// Row i of the left operand is scaled by 2^-e_i and column j of the right
// operand by 2^-f_j (powers of two with |entry| < 2^e), so every scaled entry
// lies in (-1, 1).  It is rounded to the fixed-point integer I = a 2^(59 - e)
// (bits below 2^-59 of the row or column scale are dropped) and cut from the
// top into kOzS signed base-64 digits, I = sum_p d_p 2^(59 - b_p) with
// b_p = 5 + 6(p-1) and d_p in [-32, 32], using integer operations only.  A
// digit is exact in BF16 and a product of two digits is at most 2^10, so a sum
// of g slice-pair products over K terms is an integer below 2^24 whenever
// g K <= 2^14: the FP32 tensor-memory accumulation is exact.  Pairs with the
// same p + q share the weight 2^-(b_p + b_q); they are grouped into
// accumulation units of at most 2^14 / K pairs, and each unit is folded into
// the FP64 result once, with weight 2^(e_i + f_j - b_p - b_q).  Pairs with
// p + q > kOzS + 1 are dropped; they and the fixed-point rounding contribute
// below 2^-59 of |row scale| |column scale| per product term.
// ---------------------------------------------------------------------------
constexpr int kOzFrac = 59;
constexpr int kOzMaxK = 1 << 14;
constexpr int kOzExpEmpty = -1100;  // exponent of an all-zero row

__host__ __device__ constexpr int oz_bits(int p) { return 5 + 6 * (p - 1); }
static_assert(oz_bits(kOzS) == kOzFrac, "the last digit has weight 2^-kOzFrac");

// e with |x| < 2^e, from the bits of |x| (x != 0)
__device__ __forceinline__ int oz_exponent(uint64_t absbits) {
  const int ea = (int)(absbits >> 52);
  return ea != 0 ? ea - 1022 : 64 - __clzll((long long)absbits) - 1074;
}

// round(a 2^(kOzFrac - e)) for |a| < 2^e (ties away from zero)
__device__ __forceinline__ int64_t oz_fixed(double a, int e) {
  const uint64_t bits = (uint64_t)__double_as_longlong(a);
  const int ea = (int)((bits >> 52) & 0x7ff);
  uint64_t mant = bits & 0xfffffffffffffull;
  if (ea == 0 && mant == 0) return 0;
  int ex = -1074;
  if (ea != 0) {
    mant |= 1ull << 52;
    ex = ea - 1075;
  }
  const int sh = ex - e + kOzFrac;  // a 2^(kOzFrac - e) = mant 2^sh
  int64_t I = 0;
  if (sh >= 0)
    I = (int64_t)(mant << sh);
  else if (sh > -64)
    I = (int64_t)((mant + (1ull << (-sh - 1))) >> (-sh));
  return (bits >> 63) ? -I : I;
}

// the kOzS digits of I, slice p at out[(p-1) stride]
__device__ __forceinline__ void oz_put_digits(int64_t I, __nv_bfloat16 *out, size_t stride) {
#pragma unroll
  for (int p = 1; p <= kOzS; ++p) {
    const int sh = kOzFrac - oz_bits(p);
    int64_t d = I;
    if (sh > 0) {
      d = (I + (1ll << (sh - 1))) >> sh;
      I -= d << sh;
    }
    out[(size_t)(p - 1) * stride] = __float2bfloat16_rn((float)(int)d);
  }
}

__device__ __forceinline__ uint64_t oz_absbits(double x) {
  return (uint64_t)__double_as_longlong(x) & 0x7fffffffffffffffull;
}

// Entry (r, k) of the rows x K block of a column-major matrix (T = double, or
// complex double as (re, im)) under a mode: 0 = the whole block; 1 = lower
// triangle (k <= r); 2 = lower triangle with a unit diagonal.
template <bool CPLX>
__device__ __forceinline__ void oz_entry(const double *__restrict__ A, int64_t lda, int rows, int K, int mode, int r,
                                         int k, double &re, double &im) {
  constexpr int W = CPLX ? 2 : 1;
  re = 0.0;
  im = 0.0;
  if (r >= rows || k >= K || (mode != 0 && k > r)) return;
  if (mode == 2 && k == r) {
    re = 1.0;
    return;
  }
  re = A[W * (r + (int64_t)k * lda)];
  if (CPLX) im = A[W * (r + (int64_t)k * lda) + 1];
}

// K-balancing exponents: g_k with max_r |A_rk| < 2^g_k over the block (complex:
// one g per complex column, stored for both real columns 2k and 2k+1).  The
// left operand is sliced as A_rk 2^-g_k and the right one as X_kj 2^g_k, which
// leaves the product unchanged and makes the row and column scales of badly
// scaled operands (D_r L D_c) meaningful.  A column without nonzeros keeps
// kOzExpEmpty and the right operand's row k is then ignored.  A CTA covers 32
// columns x 256 rows (a warp per column, lanes down the rows) and folds its
// maxima in with atomicMax over the kOzExpEmpty fill.
__global__ void oz_fill_kernel(int *p, int n, int v) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) p[k] = v;
}

template <bool CPLX>
__global__ void __launch_bounds__(256) oz_kexp_kernel(const double *__restrict__ A, int64_t lda, int rows, int K,
                                                      int mode, int *kexp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r0 = blockIdx.y * 256;
  for (int k = blockIdx.x * 32 + warp; k < min(K, blockIdx.x * 32 + 32); k += 8) {
    uint64_t mx = 0;
    for (int r = r0 + lane; r < min(rows, r0 + 256); r += 32) {
      double re, im;
      oz_entry<CPLX>(A, lda, rows, K, mode, r, k, re, im);
      mx = max(mx, max(oz_absbits(re), oz_absbits(im)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, (uint64_t)__shfl_down_sync(0xffffffffu, mx, o));
    if (lane == 0 && mx != 0) {
      const int e = oz_exponent(mx);
      atomicMax(&kexp[(CPLX ? 2 : 1) * k], e);
      if (CPLX) atomicMax(&kexp[2 * k + 1], e);
    }
  }
}

// Slices of a left operand: the rows x K block (mode as in oz_entry; complex
// expanded to the real 2 rows x 2 K form with [re -im; im re] per entry),
// balanced by 2^-g_k, as out[p][row][k], rows' x Kp row-major per slice (zero
// beyond K'), plus the row exponents.  One CTA per 32 rows: a pass for the
// exponents, a pass for the digits.
template <bool CPLX>
__global__ void __launch_bounds__(256) oz_slice_a_kernel(const double *__restrict__ A, int64_t lda, int rows, int K,
                                                         int Kp, int mode, const int *__restrict__ kexp, int *rexp,
                                                         __nv_bfloat16 *out, size_t sstride) {
  constexpr int W = CPLX ? 2 : 1;
  constexpr int KT = 32 / W;  // source columns per tile
  __shared__ double sre[KT][33], sim[CPLX ? KT : 1][33];
  __shared__ int sg[KT];
  __shared__ int red[8][32];
  __shared__ int se[32];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int i0 = blockIdx.x * 32;
  const int i = i0 + tx;
  int ex = INT_MIN;
  const int kend = mode != 0 ? min(K, i + 1) : K;
  for (int k = ty; k < kend && i < rows; k += 8) {
    double re, im;
    oz_entry<CPLX>(A, lda, rows, K, mode, i, k, re, im);
    const uint64_t ab = max(oz_absbits(re), oz_absbits(im));
    if (ab != 0) ex = max(ex, oz_exponent(ab) - kexp[W * k]);
  }
  red[ty][tx] = ex;
  __syncthreads();
  if (ty == 0) {
    for (int w = 1; w < 8; ++w) ex = max(ex, red[w][tx]);
    const int e = ex == INT_MIN ? kOzExpEmpty : ex;
    se[tx] = e;
    if (i < rows) {
      rexp[W * i] = e;
      if (CPLX) rexp[W * i + 1] = e;
    }
  }
  __syncthreads();
  for (int k0 = 0; k0 < Kp; k0 += 32) {
    const int kc0 = k0 / W;
    for (int kk = ty; kk < KT; kk += 8) {
      double re, im;
      oz_entry<CPLX>(A, lda, rows, K, mode, i, kc0 + kk, re, im);
      sre[kk][tx] = re;
      if (CPLX) sim[kk][tx] = im;
    }
    if (threadIdx.x < KT) sg[threadIdx.x] = kc0 + (int)threadIdx.x < K ? kexp[W * (kc0 + threadIdx.x)] : 0;
    __syncthreads();
    const int g = sg[tx / W];
    for (int ii = ty; ii < 32; ii += 8) {
      const int r = i0 + ii;
      if (r >= rows) break;
      const int e = se[ii];
      const bool zero = e == kOzExpEmpty;
      if (CPLX) {
        const double re = sre[tx >> 1][ii], im = sim[tx >> 1][ii];
        const bool first = (tx & 1) == 0;
        oz_put_digits(zero ? 0 : oz_fixed(first ? re : -im, e + g), out + (size_t)(2 * r) * Kp + k0 + tx, sstride);
        oz_put_digits(zero ? 0 : oz_fixed(first ? im : re, e + g), out + (size_t)(2 * r + 1) * Kp + k0 + tx,
                      sstride);
      } else {
        oz_put_digits(zero ? 0 : oz_fixed(sre[tx][ii], e + g), out + (size_t)r * Kp + k0 + tx, sstride);
      }
    }
    __syncthreads();
  }
}

// Slices of a right operand: K x N column-major (complex: its real view with
// 2K rows), balanced by 2^g_k (rows with g_k = kOzExpEmpty are ignored), as
// out[q][j][k], N x Kp row-major per slice (zero beyond K), plus the column
// exponents.  One warp per column; a lane handles two consecutive k, so each
// slice is written 128 bytes per warp step.
__global__ void __launch_bounds__(256) oz_slice_x_kernel(const double *__restrict__ X, int64_t ldx, int K, int N,
                                                         int Kp, const int *__restrict__ kexp, int *cexp,
                                                         __nv_bfloat16 *out, size_t sstride, const int *skip) {
  if (skip != nullptr && *(volatile const int *)skip) return;
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t j = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; j < N; j += nwarps) {
    const double *x = X + j * ldx;
    int ex = INT_MIN;
    for (int k = lane; k < K; k += 32) {
      const uint64_t ab = oz_absbits(x[k]);
      const int g = kexp[k];
      if (ab != 0 && g != kOzExpEmpty) ex = max(ex, oz_exponent(ab) + g);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ex = max(ex, __shfl_xor_sync(0xffffffffu, ex, o));
    const int e = ex == INT_MIN ? 0 : ex;
    if (lane == 0) cexp[j] = e;
    __nv_bfloat162 *o2 = reinterpret_cast<__nv_bfloat162 *>(out + (size_t)j * Kp);
    for (int k = 2 * lane; k < Kp; k += 64) {
      int64_t I[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int g = k + h < K ? kexp[k + h] : kOzExpEmpty;
        I[h] = g != kOzExpEmpty ? oz_fixed(x[k + h], e - g) : 0;
      }
#pragma unroll
      for (int p = 1; p <= kOzS; ++p) {
        const int sh = kOzFrac - oz_bits(p);
        float d[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          int64_t v = I[h];
          if (sh > 0) {
            v = (I[h] + (1ll << (sh - 1))) >> sh;
            I[h] -= v << sh;
          }
          d[h] = (float)(int)v;
        }
        o2[(size_t)(p - 1) * (sstride / 2) + k / 2] = __floats2bfloat162_rn(d[0], d[1]);
      }
    }
  }
}

// One sliced operand: kOzS slices of rows x Kp BF16 digits, an exponent per
// row, and (left operands) the K-balancing exponents.
struct OzOperand {
  __nv_bfloat16 *slices = nullptr;
  int *exps = nullptr;
  int *kexp = nullptr;
  int rows = 0, Kp = 0;
};

int oz_kp(int64_t K) { return (int)((K + TC_BK - 1) / TC_BK) * TC_BK; }

size_t oz_slices_bytes(int64_t rows, int Kp) {
  return (kOzS * (size_t)rows * Kp * sizeof(__nv_bfloat16) + 1023) & ~(size_t)1023;
}

size_t oz_operand_bytes(int64_t rows, int Kp) {
  return oz_slices_bytes(rows, Kp) + ((sizeof(int) * (size_t)rows + 1023) & ~(size_t)1023) +
         ((sizeof(int) * (size_t)Kp + 1023) & ~(size_t)1023);
}

OzOperand oz_operand(void *ws, int64_t rows, int Kp) {
  OzOperand o;
  unsigned char *b = static_cast<unsigned char *>(ws);
  o.slices = reinterpret_cast<__nv_bfloat16 *>(b);
  o.exps = reinterpret_cast<int *>(b + oz_slices_bytes(rows, Kp));
  o.kexp = reinterpret_cast<int *>(b + oz_slices_bytes(rows, Kp) + ((sizeof(int) * (size_t)rows + 1023) & ~(size_t)1023));
  o.rows = (int)rows;
  o.Kp = Kp;
  return o;
}

// Slice the rows x K block of A (lda in elements of the dtype) into o (o.rows =
// W rows), with its K-balancing exponents in o.kexp.
hsma_status_t oz_slice_a(bool cplx, const double *A, int64_t lda, int rows, int K, int mode, OzOperand &o,
                         cudaStream_t st) {
  if (rows <= 0 || K <= 0) return HSMA_OK;
  const size_t ss = (size_t)o.rows * o.Kp;
  const dim3 kg((unsigned)((K + 31) / 32), (unsigned)((rows + 255) / 256));
  if (kg.y > 65535) return HSMA_ERR_UNSUPPORTED;
  const int kw = (cplx ? 2 : 1) * K;
  oz_fill_kernel<<<(kw + 255) / 256, 256, 0, st>>>(o.kexp, kw, kOzExpEmpty);
  if (cplx) {
    oz_kexp_kernel<true><<<kg, 256, 0, st>>>(A, lda, rows, K, mode, o.kexp);
    oz_slice_a_kernel<true><<<(rows + 31) / 32, 256, 0, st>>>(A, lda, rows, K, o.Kp, mode, o.kexp, o.exps, o.slices,
                                                               ss);
  } else {
    oz_kexp_kernel<false><<<kg, 256, 0, st>>>(A, lda, rows, K, mode, o.kexp);
    oz_slice_a_kernel<false><<<(rows + 31) / 32, 256, 0, st>>>(A, lda, rows, K, o.Kp, mode, o.kexp, o.exps,
                                                                o.slices, ss);
  }
  HSMA_CUDA_TRY(cudaGetLastError());
  return HSMA_OK;
}

// Slice the K x N real matrix X (complex: its real view) into o (o.rows = N),
// balanced by the K-balancing exponents of the left operand it multiplies.
hsma_status_t oz_slice_x(const double *X, int64_t ldx, int K, const int *kexp, OzOperand &o, const int *skip,
                         cudaStream_t st) {
  if (o.rows <= 0) return HSMA_OK;
  const int grid = std::min((o.rows + 7) / 8, hsma_sm_count() * 16);
  oz_slice_x_kernel<<<grid, 256, 0, st>>>(X, ldx, K, o.rows, o.Kp, kexp, o.exps, o.slices, (size_t)o.rows * o.Kp,
                                          skip);
  HSMA_CUDA_TRY(cudaGetLastError());
  return HSMA_OK;
}

// Unit table: pairs of equal p + q, smallest weights first, at most
// 2^14 / Kp pairs per unit (exact FP32 sums).
void oz_units(int Kp, TcArgs &a) {
  const int gmax = std::max(1, kOzMaxK / Kp);
  int np = 0, nu = 0;
  for (int s = kOzS + 1; s >= 2; --s) {
    int in_unit = 0;
    for (int p = std::max(1, s - kOzS); p <= std::min(kOzS, s - 1); ++p) {
      if (in_unit == 0) {
        a.ubeg[nu] = (uint8_t)np;
        a.uexp[nu] = (int8_t)(-(oz_bits(p) + oz_bits(s - p)));
        ++nu;
      }
      a.pa[np] = (uint8_t)(p - 1);
      a.pb[np] = (uint8_t)(s - p - 1);
      ++np;
      if (++in_unit == gmax) in_unit = 0;
    }
  }
  a.ubeg[nu] = (uint8_t)np;
  a.nunits = nu;
}

// C (M x N, column-major FP64) = (beta0 ? C : 0) -/+ L X in emulated FP64,
// L and X given by their slices; tri: L is lower triangular.
hsma_status_t oz_product(const OzOperand &L, const OzOperand &X, double *C, int64_t ldc, int beta0, int negate,
                         int tri, const int *skip, const char *phase, cudaStream_t st) {
  if (L.Kp != X.Kp || L.Kp > kOzMaxK) return HSMA_ERR_INVALID_ARG;
  TcArgs a{};
  a.C64 = C;
  a.ldc = ldc;
  a.beta0 = beta0;
  a.negate = negate;
  a.rexp = L.exps;
  a.cexp = X.exps;
  a.M = L.rows;
  a.N = X.rows;
  a.K = L.Kp;
  a.tri = tri;
  a.skip = skip;
  oz_units(L.Kp, a);
  return tc_gemm<TC_OZ>(L.slices, kOzS, X.slices, kOzS, a, phase, st);
}

// R -= L X in emulated FP64 (R holds alpha B on entry); skip: device flag.
// K runs in chunks of kOzResidualChunk columns of L: chunk c touches only rows
// below its start (L is lower triangular) and each launch re-reads a chunk's
// slices, which stay in L2, for all its slice pairs; one launch over the whole
// K would stream every row tile's full slices from memory once per pair.
constexpr int kOzResidualChunk = 1024;

hsma_status_t oz_residual(const OzOperand &L, const double *X, int64_t ldx, double *R, int64_t ldr, OzOperand &Xo,
                          const int *skip, cudaStream_t st) {
  {
    HsmaTraceScope ts("residual_slices", st);
    hsma_status_t s = oz_slice_x(X, ldx, L.rows, L.kexp, Xo, skip, st);
    if (s != HSMA_OK) return s;
  }
  const int64_t m = L.rows, Kp = L.Kp;
  for (int64_t c0 = 0; c0 < m; c0 += kOzResidualChunk) {
    const int kc = (int)std::min<int64_t>(kOzResidualChunk, m - c0);
    TcArgs a{};
    a.C64 = R + c0;
    a.ldc = ldr;
    a.beta0 = 1;
    a.negate = 0;
    a.rexp = L.exps + c0;
    a.cexp = Xo.exps;
    a.M = (int)(m - c0);
    a.N = Xo.rows;
    a.K = oz_kp(kc);
    a.tri = 1;  // rows c0 + i need chunk columns <= i only
    a.skip = skip;
    oz_units(a.K, a);
    SliceLayout la, lb;  // views into the full slice stacks at row / K offset c0
    la.rows = m - c0;
    la.kext = Kp - c0;
    la.ld = Kp;
    la.sst = m * Kp;
    lb.rows = Xo.rows;
    lb.kext = Kp - c0;
    lb.ld = Kp;
    lb.sst = (int64_t)Xo.rows * Kp;
    hsma_status_t s = tc_gemm<TC_OZ>(L.slices + c0 * Kp + c0, kOzS, Xo.slices + c0, kOzS, a, "residual", st, la, lb);
    if (s != HSMA_OK) return s;
  }
  return HSMA_OK;
}

__global__ void scale_kernel(double *B, int64_t ldb, int64_t rows, int64_t n, double ar, double ai, int cplx) {
  HSMA_FOR_RC(i, j, rows, n) {
    if (cplx) {
      double *p = B + 2 * (i + j * ldb);
      const double re = p[0], im = p[1];
      p[0] = ar * re - ai * im;
      p[1] = ar * im + ai * re;
    } else {
      B[i + j * ldb] *= ar;
    }
  }
}


// Blocked solve (Section 4.3) with both products of every block step, the
// solve X_r = D_r^{-1} B_r and the trailing update B_{r+1:} -= A_{r+1:,r} X_r,
// emulated in FP64 on the BF16 tensor cores.  The diagonal blocks are
// inverted in FP64 (Algorithm 2).  Complex operands run as real products of
// the expanded forms (rows [re -im; im re] on the left, the interleaved real
// view on the right and in B), so a complex product is four real ones.
//
// Each emulated product adds every accumulation unit into B once in FP64, so
// its cost per element of B grows with the number of units, not with K.  The
// updates are therefore applied per panel of h diagonal blocks (about 2048
// real columns): inside a panel, each solved block updates only the panel's
// remaining rows; below the panel, one update with K = h N_B covers all h
// blocks.  The result is the same product sum, grouped differently.
// The panel width (real columns; the panel's trailing update runs with K =
// that many real columns) comes from the planner: the autotuned table, else
// kEmuPanelColsDefault.  Measured on GB300 for m = 16384 FP64 / 8192
// complex128: 1024 columns 217 / 112 ms, 2048 columns 208 / 105 ms, 3072 and
// 4096 columns slower again.

// Workspace of blocked_emulated: the inverses, one block row of B, and the
// slices of an update panel, of one inverse and of the right operand.
struct EmuLayout {
  int W = 1, h = 1, Kpb = 0, Kpp = 0;
  int64_t P = 0;
  size_t dinv_b = 0, w_b = 0, pa_b = 0, pd_b = 0, px_b = 0;
  size_t total() const { return dinv_b + w_b + pa_b + pd_b + px_b; }
};

EmuLayout emu_layout(bool cplx, int nb, int panel_cols, int64_t m, int64_t n) {
  EmuLayout L;
  L.W = cplx ? 2 : 1;
  const int64_t nblk = (m + nb - 1) / nb;
  L.h = std::max(1, (panel_cols > 0 ? panel_cols : kEmuPanelColsDefault) / (L.W * nb));
  L.P = (int64_t)L.h * nb;  // panel width (source columns)
  L.Kpb = oz_kp((int64_t)L.W * nb);
  L.Kpp = oz_kp(L.W * L.P);
  auto al = [](size_t v) { return (v + 1023) & ~(size_t)1023; };
  const size_t eb = sizeof(double) * L.W;
  L.dinv_b = al(eb * (size_t)nblk * nb * nb);
  L.w_b = al(eb * (size_t)nb * n);
  L.pa_b = al(oz_operand_bytes((int64_t)L.W * m, L.Kpp));
  L.pd_b = al(oz_operand_bytes((int64_t)L.W * nb, L.Kpb));
  L.px_b = al(oz_operand_bytes(n, L.Kpp));
  return L;
}

hsma_status_t blocked_emulated(bool cplx, int nb, int panel_cols, const double *A, int64_t lda, double *B,
                               int64_t ldb, int64_t m,
                               int64_t n, const double *alpha, int unit, cudaStream_t st) {
  const EmuLayout E = emu_layout(cplx, nb, panel_cols, m, n);
  const int W = E.W;
  const int64_t P = E.P;
  const int Kpb = E.Kpb, Kpp = E.Kpp;
  if (Kpp > kOzMaxK || (int64_t)W * m > INT32_MAX || n > INT32_MAX) return HSMA_ERR_UNSUPPORTED;
  const size_t eb = sizeof(double) * W;
  const size_t dinv_b = E.dinv_b, w_b = E.w_b, pa_b = E.pa_b;
  void *ws = nullptr;
  hsma_status_t s = hsma_ws_alloc(&ws, E.total(), st);
  if (s != HSMA_OK) return s;
  unsigned char *base = static_cast<unsigned char *>(ws);
  double *Dinv = reinterpret_cast<double *>(base);
  double *Wb = reinterpret_cast<double *>(base + dinv_b);
  unsigned char *pa_mem = base + dinv_b + w_b, *px_mem = base + dinv_b + w_b + pa_b + E.pd_b;
  // views of the operand buffers for a given K (the buffers hold the widest)
  auto view = [](unsigned char *mem, int64_t rows_cap, int Kp, int64_t rows) {
    OzOperand o = oz_operand(mem, rows_cap, Kp);
    o.rows = (int)rows;
    return o;
  };
  OzOperand Pd = oz_operand(base + dinv_b + w_b + pa_b, (int64_t)W * nb, Kpb);
  // B rows [rb, rb + rows) -= A[rb : rb + rows, c0 : c0 + k] X[c0 : c0 + k]
  auto update = [&](int64_t rb, int64_t rows, int64_t c0, int k, const char *phase) -> hsma_status_t {
    const int Kp = oz_kp((int64_t)W * k);
    OzOperand Pa = view(pa_mem, (int64_t)W * m, Kp, (int64_t)W * rows);
    OzOperand Px = view(px_mem, n, Kp, n);
    {
      HsmaTraceScope ts("slices", st, 4);  // oz_slice_a: 3 kernels, oz_slice_x: 1
      hsma_status_t e = oz_slice_a(cplx, A + W * (rb + c0 * lda), lda, (int)rows, k, 0, Pa, st);
      if (e == HSMA_OK) e = oz_slice_x(B + W * c0, (int64_t)W * ldb, W * k, Pa.kexp, Px, nullptr, st);
      if (e != HSMA_OK) return e;
    }
    return oz_product(Pa, Px, B + W * rb, (int64_t)W * ldb, 1, 0, 0, nullptr, phase, st);
  };
  do {
    if ((s = hsma_diag_inverse(cplx ? HSMA_C128 : HSMA_R64, nb, A, lda, m, unit, Dinv, st)) != HSMA_OK) break;
    if (alpha[0] != 1.0 || (cplx && alpha[1] != 0.0)) {
      HsmaTraceScope ts("copy", st);
      scale_kernel<<<hsma_grid_rc(m, n), 256, 0, st>>>(B, ldb, m, n, alpha[0], cplx ? alpha[1] : 0.0, cplx);
      if ((s = hsma_from_cuda(cudaGetLastError())) != HSMA_OK) break;
    }
    for (int64_t R0 = 0; R0 < m && s == HSMA_OK; R0 += P) {
      const int64_t PR = std::min<int64_t>(P, m - R0);
      for (int64_t r0 = R0; r0 < R0 + PR && s == HSMA_OK; r0 += nb) {
        const int64_t r = r0 / nb;
        const int sr = (int)std::min<int64_t>(nb, m - r0);
        {
          HsmaTraceScope ts("copy", st, 0);
          cudaError_t e =
              cudaMemcpy2DAsync(Wb, eb * nb, B + W * r0, eb * ldb, eb * sr, n, cudaMemcpyDeviceToDevice, st);
          if ((s = hsma_from_cuda(e)) != HSMA_OK) break;
        }
        // X_r = D_r^{-1} B_r
        Pd.rows = W * sr;
        OzOperand Px = view(px_mem, n, Kpb, n);
        {
          HsmaTraceScope ts("slices", st, 4);
          if ((s = oz_slice_a(cplx, Dinv + (size_t)W * r * nb * nb, nb, sr, sr, 1, Pd, st)) != HSMA_OK) break;
          if ((s = oz_slice_x(Wb, (int64_t)W * nb, W * sr, Pd.kexp, Px, nullptr, st)) != HSMA_OK) break;
        }
        if ((s = oz_product(Pd, Px, B + W * r0, (int64_t)W * ldb, 0, 1, 1, nullptr, "solve_gemm", st)) != HSMA_OK)
          break;
        // the panel's remaining rows
        const int64_t rin = R0 + PR - (r0 + sr);
        if (rin > 0) s = update(r0 + sr, rin, r0, sr, "update_gemm");
      }
      // every row below the panel, K = the panel's width
      const int64_t rout = m - (R0 + PR);
      if (s == HSMA_OK && rout > 0) s = update(R0 + PR, rout, R0, (int)PR, "update_gemm");
    }
  } while (0);
  hsma_status_t f = hsma_ws_free(ws, st);
  return s != HSMA_OK ? s : f;
}

}  // namespace

hsma_status_t hsma_mixed_r32(int nb, int bf16_terms, const float *A, int64_t lda, float *B, int64_t ldb, int64_t m,
                             int64_t n, double alpha, int unit, cudaStream_t st) {
  const int terms = bf16_terms == 0 ? 3 : bf16_terms;
  if (terms != 1 && terms != 3) return HSMA_ERR_INVALID_ARG;
  if (m > INT32_MAX || n > INT32_MAX) return HSMA_ERR_UNSUPPORTED;
  return r32_solve(nb, terms, A, lda, B, ldb, m, n, (float)alpha, unit, st);
}

hsma_status_t hsma_mixed_ir(int nb, const hsma_opts_t *opts, const double *A, int64_t lda, double *B, int64_t ldb,
                            int64_t m, int64_t n, double alpha, int unit, cudaStream_t st, hsma_info_t *info) {
  const int terms = (opts && opts->bf16_terms) ? opts->bf16_terms : 3;
  const int itmax = (opts && opts->ir_max_iter > 0) ? opts->ir_max_iter : 10;
  const double tol = (opts && opts->ir_tol > 0.0) ? opts->ir_tol : 1e-15;
  const int res_mode = opts ? opts->ir_residual : 0;
  if (terms != 1 && terms != 3) return HSMA_ERR_INVALID_ARG;
  if (res_mode != 0 && res_mode != 1) return HSMA_ERR_INVALID_ARG;
  if (m > INT32_MAX || n > INT32_MAX) return HSMA_ERR_UNSUPPORTED;
  // residual products: emulated FP64 on the BF16 tensor cores unless asked
  // otherwise or K is beyond the exactness bound of the slice sums
  const bool emulated = res_mode == 0 && m <= kOzMaxK;
  auto al = [](size_t v) { return (v + 1023) & ~(size_t)1023; };
  const size_t a32_b = sizeof(float) * (size_t)m * m;
  const size_t r32_b = sizeof(float) * (size_t)m * n;
  const size_t b0_b = sizeof(double) * (size_t)m * n;
  const size_t r64_b = b0_b;
  const size_t st_b = 1024;
  const int ozkp = oz_kp(m);
  const size_t ozl_b = emulated ? al(oz_operand_bytes(m, ozkp)) : 0;
  const size_t ozx_b = emulated ? al(oz_operand_bytes(n, ozkp)) : 0;
  // the FP32 inverses and BF16 panels of L, shared by the first solve and every correction
  R32Plan P;
  P.nb = nb < 32 ? 32 : nb;
  P.terms = terms;
  P.Kp = round_up(terms * P.nb, TC_BK);
  P.m = m;
  P.lda = m;
  P.unit = unit;
  const size_t dinv_b = al(sizeof(float) * (size_t)((m + P.nb - 1) / P.nb) * P.nb * P.nb);
  const size_t pan_b = al(sizeof(__nv_bfloat16) * r32_panels_elems(P.nb, terms, m));
  void *ws = nullptr;
  hsma_status_t s = hsma_ws_alloc(
      &ws, al(a32_b) + al(r32_b) + al(b0_b) + al(r64_b) + st_b + ozl_b + ozx_b + dinv_b + pan_b, st);
  if (s != HSMA_OK) return s;
  unsigned char *base = static_cast<unsigned char *>(ws);
  float *A32 = reinterpret_cast<float *>(base);
  float *R32 = reinterpret_cast<float *>(base + al(a32_b));
  double *B0 = reinterpret_cast<double *>(base + al(a32_b) + al(r32_b));
  double *R64 = reinterpret_cast<double *>(base + al(a32_b) + al(r32_b) + al(b0_b));
  double *sums = reinterpret_cast<double *>(base + al(a32_b) + al(r32_b) + al(b0_b) + al(r64_b));
  int *state = reinterpret_cast<int *>(sums + 8);
  void *ozl_ws = base + al(a32_b) + al(r32_b) + al(b0_b) + al(r64_b) + st_b;
  void *ozx_ws = static_cast<unsigned char *>(ozl_ws) + ozl_b;
  OzOperand Lsl = oz_operand(ozl_ws, m, ozkp), Xsl = oz_operand(ozx_ws, n, ozkp);
  P.A = A32;
  P.Dinv = reinterpret_cast<float *>(static_cast<unsigned char *>(ozx_ws) + ozx_b);
  P.panels = reinterpret_cast<__nv_bfloat16 *>(reinterpret_cast<unsigned char *>(P.Dinv) + dinv_b);
  const dim3 grid = hsma_grid_rc(m, n);
  auto fail = [&](cudaError_t e) { return e == cudaSuccess ? HSMA_OK : hsma_from_cuda(e); };
  do {
    if ((s = fail(cudaMemsetAsync(sums, 0, st_b, st))) != HSMA_OK) break;
    if ((s = fail(cudaMemcpy2DAsync(B0, sizeof(double) * m, B, sizeof(double) * ldb, sizeof(double) * m, n,
                                    cudaMemcpyDeviceToDevice, st))) != HSMA_OK)
      break;
    {
      HsmaTraceScope ts("convert", st, 4);
      f64_to_f32_kernel<<<hsma_grid_rc(m, m), 256, 0, st>>>(A, lda, A32, m, m, m, 1, nullptr);
      f64_to_f32_kernel<<<grid, 256, 0, st>>>(B, ldb, R32, m, m, n, 0, nullptr);
      sumsq_kernel<<<hsma_grid_rc(m, m), 256, 0, st>>>(A, lda, m, m, 1, unit, sums, 0, nullptr);
      sumsq_kernel<<<grid, 256, 0, st>>>(B0, m, m, n, 0, 0, sums, 1, nullptr);
      if ((s = fail(cudaGetLastError())) != HSMA_OK) break;
    }
    if (emulated) {
      HsmaTraceScope ts("residual_slices", st, 3);
      if ((s = oz_slice_a(false, A, lda, (int)m, (int)m, unit ? 2 : 1, Lsl, st)) != HSMA_OK) break;
    }
    // X_0 from the FP32-result solve of the rounded data
    if ((s = r32_prepare(P, true, st)) != HSMA_OK) break;
    if ((s = r32_apply(P, R32, m, n, (float)alpha, nullptr, st)) != HSMA_OK) break;
    {
      HsmaTraceScope ts("refine", st);
      accumulate_kernel<<<grid, 256, 0, st>>>(B, ldb, R32, m, m, n, 1, nullptr);
    }
    // Outside stream capture the host reads the stopping test after every
    // step and launches nothing more once it holds; under capture every step
    // is recorded and the device skips the ones after convergence.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if ((s = fail(cudaStreamIsCapturing(st, &cap))) != HSMA_OK) break;
    const bool host_test = cap == cudaStreamCaptureStatusNone;
    for (int it = 0; it <= itmax && s == HSMA_OK; ++it) {
      // R = alpha B - L X in FP64, then the stopping test
      if (emulated) {
        {
          HsmaTraceScope ts("refine", st);
          scale_copy_kernel<<<g_launch_grid(m * n), 256, 0, st>>>(B0, R64, m * n, alpha, state);
        }
        if ((s = oz_residual(Lsl, B, ldb, R64, m, Xsl, state, st)) != HSMA_OK) break;
      } else {
        if ((s = fail(cudaMemcpy2DAsync(R64, sizeof(double) * m, B0, sizeof(double) * m, sizeof(double) * m, n,
                                        cudaMemcpyDeviceToDevice, st))) != HSMA_OK)
          break;
        if ((s = hsma_residual_f64(A, lda, unit, B, ldb, R64, m, m, n, alpha, state, st)) != HSMA_OK) break;
      }
      {
        HsmaTraceScope ts("refine", st, 3);
        sumsq_kernel<<<grid, 256, 0, st>>>(R64, m, m, n, 0, 0, sums, 2, state);
        sumsq_kernel<<<grid, 256, 0, st>>>(B, ldb, m, n, 0, 0, sums, 3, state);
        check_kernel<<<1, 1, 0, st>>>(sums, state, std::fabs(alpha), tol, it, it == itmax ? 1 : 0,
                                      hsma_dev_error_ptr());
        if (it == itmax) break;
        if (host_test) {
          int conv = 0;
          if ((s = fail(cudaMemcpyAsync(&conv, state, sizeof conv, cudaMemcpyDeviceToHost, st))) != HSMA_OK) break;
          if ((s = fail(cudaStreamSynchronize(st))) != HSMA_OK) break;
          if (conv) break;
        }
        f64_to_f32_kernel<<<grid, 256, 0, st>>>(R64, m, R32, m, m, n, 0, state);
        hsma_count_launches(1);
        if ((s = fail(cudaGetLastError())) != HSMA_OK) break;
      }
      // correction C from the FP32-result solve of L C = R (alpha = 1), X += C
      if ((s = r32_apply(P, R32, m, n, 1.0f, state, st)) != HSMA_OK) break;
      {
        HsmaTraceScope ts("refine", st);
        accumulate_kernel<<<grid, 256, 0, st>>>(B, ldb, R32, m, m, n, 0, state);
      }
      if ((s = fail(cudaGetLastError())) != HSMA_OK) break;
    }
    if (s == HSMA_OK && info != nullptr) {
      int h[4] = {0, 0, 0, 0};
      if ((s = fail(cudaMemcpyAsync(h, state, sizeof h, cudaMemcpyDeviceToHost, st))) != HSMA_OK) break;
      if ((s = fail(cudaStreamSynchronize(st))) != HSMA_OK) break;
      info->converged = h[0];
      info->ir_iters = h[1];
      std::memcpy(&info->ir_residual, h + 2, sizeof(double));
    }
  } while (0);
  hsma_status_t f = hsma_ws_free(ws, st);
  if (s == HSMA_OK && info != nullptr && !info->converged) s = HSMA_ERR_NOT_CONVERGED;
  return s != HSMA_OK ? s : f;
}

extern "C" HSMA_API hsma_status_t hsma_gemm_bf16_update(int64_t M, int64_t N, int64_t K, const void *A,
                                                        const void *Bt, float beta, float *C, int64_t ldc,
                                                        void *stream) {
  if (M < 0 || N < 0 || K < 0 || ldc < std::max<int64_t>(1, M)) return HSMA_ERR_INVALID_ARG;
  if (M == 0 || N == 0) return HSMA_OK;
  if (A == nullptr || Bt == nullptr || C == nullptr || K == 0 || K % 64 != 0) return HSMA_ERR_INVALID_ARG;
  if (M > INT32_MAX || N > INT32_MAX || K > INT32_MAX) return HSMA_ERR_UNSUPPORTED;
  return bf16_update(static_cast<const __nv_bfloat16 *>(A), static_cast<const __nv_bfloat16 *>(Bt), (int)M, (int)N,
                     (int)K, beta, C, ldc, static_cast<cudaStream_t>(stream));
}

hsma_status_t hsma_blocked_emulated(int dtype, int nb, int panel_cols, const void *A, int64_t lda, void *B,
                                    int64_t ldb, int64_t m, int64_t n, const double *alpha, int unit,
                                    cudaStream_t st) {
  if (dtype != HSMA_R64 && dtype != HSMA_C128) return HSMA_ERR_INVALID_ARG;
  return blocked_emulated(dtype == HSMA_C128, nb, panel_cols, static_cast<const double *>(A), lda,
                          static_cast<double *>(B), ldb, m, n, alpha, unit, st);
}

size_t hsma_blocked_emulated_ws_bytes(int dtype, int nb, int panel_cols, int64_t m, int64_t n) {
  return emu_layout(dtype == HSMA_C128, nb, panel_cols, m, n).total();
}

extern "C" HSMA_API hsma_status_t hsma_gemm_f64_emulated(int64_t M, int64_t N, int64_t K, const double *A,
                                                         int64_t lda, const double *X, int64_t ldx, double *C,
                                                         int64_t ldc, void *stream) {
  if (M < 0 || N < 0 || K < 0 || lda < std::max<int64_t>(1, M) || ldx < std::max<int64_t>(1, K) ||
      ldc < std::max<int64_t>(1, M))
    return HSMA_ERR_INVALID_ARG;
  if (M == 0 || N == 0 || K == 0) return HSMA_OK;
  if (A == nullptr || X == nullptr || C == nullptr) return HSMA_ERR_INVALID_ARG;
  if (K > kOzMaxK || M > INT32_MAX || N > INT32_MAX) return HSMA_ERR_UNSUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int Kp = oz_kp(K);
  const size_t a_b = oz_operand_bytes(M, Kp), x_b = oz_operand_bytes(N, Kp);
  void *ws = nullptr;
  hsma_status_t s = hsma_ws_alloc(&ws, a_b + x_b, st);
  if (s != HSMA_OK) return s;
  OzOperand Ao = oz_operand(ws, M, Kp), Xo = oz_operand(static_cast<unsigned char *>(ws) + a_b, N, Kp);
  s = oz_slice_a(false, A, lda, (int)M, (int)K, 0, Ao, st);
  if (s == HSMA_OK) s = oz_slice_x(X, ldx, (int)K, Ao.kexp, Xo, nullptr, st);
  if (s == HSMA_OK) s = oz_product(Ao, Xo, C, ldc, 1, 0, 0, nullptr, "emulated_gemm", st);
  hsma_status_t f = hsma_ws_free(ws, st);
  return s != HSMA_OK ? s : f;
}

namespace {

// complex64 lower triangle (zeros above) or block -> complex128, column-major
__global__ void c64_to_c128_kernel(const cplxf *__restrict__ src, int64_t lds, cplx *dst, int64_t ldd, int64_t rows,
                                   int64_t cols, int lower) {
  HSMA_FOR_RC(i, j, rows, cols) {
    cplx v{0.0, 0.0};
    if (!lower || i >= j) {
      const cplxf x = src[i + j * lds];
      v = cplx{(double)x.re, (double)x.im};
    }
    dst[i + j * ldd] = v;
  }
}

__global__ void c128_to_c64_kernel(const cplx *__restrict__ src, int64_t lds, cplxf *dst, int64_t ldd, int64_t rows,
                                   int64_t cols) {
  HSMA_FOR_RC(i, j, rows, cols) {
    const cplx v = src[i + j * lds];
    dst[i + j * ldd] = cplxf{(float)v.re, (float)v.im};
  }
}

}  // namespace

hsma_status_t hsma_c64_blocked(int nb, int panel_cols, const void *A, int64_t lda, void *B, int64_t ldb, int64_t m,
                               int64_t n, const double *alpha, int unit, cudaStream_t st) {
  auto al = [](size_t v) { return (v + 1023) & ~(size_t)1023; };
  const size_t a_b = al(sizeof(cplx) * (size_t)m * m), b_b = al(sizeof(cplx) * (size_t)m * n);
  void *ws = nullptr;
  hsma_status_t s = hsma_ws_alloc(&ws, a_b + b_b, st);
  if (s != HSMA_OK) return s;
  cplx *A2 = static_cast<cplx *>(ws);
  cplx *B2 = reinterpret_cast<cplx *>(static_cast<unsigned char *>(ws) + a_b);
  {
    HsmaTraceScope ts("copy", st, 2);
    c64_to_c128_kernel<<<hsma_grid_rc(m, m), 256, 0, st>>>(static_cast<const cplxf *>(A), lda, A2, m, m, m, 1);
    c64_to_c128_kernel<<<hsma_grid_rc(m, n), 256, 0, st>>>(static_cast<const cplxf *>(B), ldb, B2, m, m, n, 0);
    s = hsma_from_cuda(cudaGetLastError());
  }
  if (s == HSMA_OK) s = blocked_emulated(true, nb, panel_cols, reinterpret_cast<const double *>(A2), m,
                                         reinterpret_cast<double *>(B2), m, m, n, alpha, unit, st);
  if (s == HSMA_OK) {
    HsmaTraceScope ts("copy", st);
    c128_to_c64_kernel<<<hsma_grid_rc(m, n), 256, 0, st>>>(B2, m, static_cast<cplxf *>(B), ldb, m, n);
    s = hsma_from_cuda(cudaGetLastError());
  }
  hsma_status_t f = hsma_ws_free(ws, st);
  return s != HSMA_OK ? s : f;
}
