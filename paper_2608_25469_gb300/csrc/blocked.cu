// Large-case blocked solve (Section 4.3), fp64 and complex128.
//
// Phase 1 (Section 4.3, "parallel diagonal block inversion"): the N_B x N_B
// diagonal blocks D_t are inverted independently, all in one launch.  Each CTA
// produces a group of columns of D_t^{-1} by forward substitution against the
// identity (Section 4.3.1): the columns of D_t are streamed through a two-slot
// shared-memory buffer (Algorithm 2's double buffering: column k+1 is staged
// while column k is used), so shared memory is O(N_B).  The columns of the
// inverse live in registers: lane group g of a warp holds rows g, g+G, ...,
// and the register window slides down by one slot every G steps.
//
// Phase 2 (Section 4.3, "sequential GEMM update and solve"), for r = 0..k:
//   X_r = D_r^{-1} B_r                       (solve product, triangular)
//   B_{r+1:} = beta B_{r+1:} - A_{r+1:,r} X_r (trailing update)
// This is the right-looking order of the same arithmetic; the paper's
// left-looking update B_r -= A_{r,0:r} X_{0:r} accumulates the same products.
// alpha is folded in once: X_0 = alpha D_0^{-1} B_0 and beta = alpha at r = 0.
//
// Both products run on the FP64 tensor path (mma.sync m8n8k4 .f64, "DMMA"),
// complex as four real products, with operand tiles brought into shared memory
// by TMA (cp.async.bulk.tensor) behind mbarriers, or by plain loads when a
// leading dimension rules TMA out (an odd fp64 leading dimension).
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "blocked.h"
#include "common.cuh"
#include "tma.cuh"
#include "trace.h"
#include "workspace.h"

__device__ unsigned int g_hsma_dev_error = 0;

namespace {

// ---------------------------------------------------------------------------
// Phase 1: diagonal-block inversion
// ---------------------------------------------------------------------------
constexpr int kInvSlots = 32;  // register slots per lane: N_B = 32 * G

template <class T, int G>
__global__ void __launch_bounds__(256) diag_inverse_kernel(const T *__restrict__ A, int64_t lda, int64_t m, int unit,
                                                            T *__restrict__ Dinv) {
  using E = Elem<T>;
  constexpr int R = kInvSlots, NB = 32 * G, C = 32 / G;
  __shared__ T sRinv[NB];
  __shared__ T sCol[2][NB];
  const int nthr = blockDim.x, tid = threadIdx.x;
  const int CT = (nthr / 32) * C;
  const int64_t r0 = (int64_t)blockIdx.x * NB;
  const int s = (int)((m - r0) < NB ? (m - r0) : NB);
  const int j0 = blockIdx.y * CT;
  T *Y = Dinv + (int64_t)blockIdx.x * NB * NB;
  const T *D = A + r0 + r0 * lda;

  for (int r = tid; r < NB; r += nthr) sRinv[r] = (r < s) ? (unit ? E::one() : E::recip(E::ld(D + r + (int64_t)r * lda))) : E::zero();
  // zeros outside the computed region: whole columns >= s, rows < j0 and rows >= s
  for (int e = tid; e < CT * NB; e += nthr) {
    const int col = j0 + e / NB, row = e % NB;
    if (col < NB && (col >= s || row < j0 || row >= s)) Y[row + (int64_t)col * NB] = E::zero();
  }
  __syncthreads();
  if (j0 >= s) return;

  const int warp = tid >> 5, lane = tid & 31;
  const int g = lane % G, c = lane / G;
  const int j = j0 + warp * C + c;
  const bool colok = j < s;
  const int q0 = j0 / G;

  T x[R];
#pragma unroll
  for (int t = 0; t < R; ++t) x[t] = (colok && g + G * (t + q0) == j) ? sRinv[j] : E::zero();

  // loader role: rows tid, tid + nthr (N_B <= 2 * nthr)
  auto fetch = [&](int k, T *pf) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = tid + h * nthr;
      pf[h] = (r > k && r < s && k < s) ? E::ld(D + r + (int64_t)k * lda) : E::zero();
    }
  };
  auto put = [&](int k, const T *pf) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = tid + h * nthr;
      if (r < NB) sCol[k & 1][r] = E::mul(sRinv[r < s ? r : 0], pf[h]);
    }
  };
  T pf[2];
  fetch(j0, pf);
  put(j0, pf);
  fetch(j0 + 1, pf);
  __syncthreads();

  for (int q = q0; q * G < s; ++q) {
#pragma unroll
    for (int u = 0; u < G; ++u) {
      const int k = q * G + u;
      if (k >= s) break;
      if (k + 1 < s) put(k + 1, pf);
      if (k + 2 < s) fetch(k + 2, pf);
      const T *dc = sCol[k & 1];
      const T xk = (G == 1) ? x[0] : E::shfl(x[0], c * G + u);
      if (u < G - 1) {
        const T nv = E::fms(dc[g + G * q], xk, x[0]);
        if (g > u) x[0] = nv;
      }
#pragma unroll
      for (int t = 1; t < R; ++t) {
        if ((q + t) * G >= s) break;
        x[t] = E::fms(dc[g + G * (q + t)], xk, x[t]);
      }
      __syncthreads();
    }
    const int row = g + G * q;
    if (colok && row < s) Y[row + (int64_t)j * NB] = x[0];
#pragma unroll
    for (int t = 0; t < R - 1; ++t) x[t] = x[t + 1];
    x[R - 1] = E::zero();
  }
}

// ---------------------------------------------------------------------------
// Phase 2 products on the FP64 tensor path
// ---------------------------------------------------------------------------
constexpr int GEMM_THREADS = 128;

template <class T>
struct GemmK;
template <>
struct GemmK<double> {
  static constexpr int BK = 32;
};
template <>
struct GemmK<cplx> {
  static constexpr int BK = 16;
};

// CTA tile: WARPS_M x WARPS_N warps, each owning WM x WN blocks of 8 x 8.
// Narrow tiles keep the tensor lanes busy when n is small.
template <int WARPS_M_, int WARPS_N_, int WM_, int WN_>
struct Tile {
  static constexpr int WARPS_M = WARPS_M_, WARPS_N = WARPS_N_, WM = WM_, WN = WN_;
  static constexpr int BM = WARPS_M * WM * 8, BN = WARPS_N * WN * 8;
};
using TileWide = Tile<2, 2, 4, 4>;  // 64 x 64
using TileN16 = Tile<4, 1, 4, 2>;   // 128 x 16
using TileN8 = Tile<4, 1, 4, 1>;    // 128 x 8

// UPDATE: C = beta*C - A*B;  SCALE: C = beta*(A*B);  PARTIAL: P[z] = A*B over
// this launch's z-th K chunk (a later fixed-order sum finishes the product)
enum { MODE_UPDATE = 0, MODE_SCALE = 1, MODE_PARTIAL = 2 };

template <class T>
struct GemmArgs {
  const T *A;  // M x K (column-major, lda)
  int64_t lda;
  const T *Bm;  // K x N (column-major, ldb)
  int64_t ldb;
  T *C;  // M x N (column-major, ldc)
  int64_t ldc;
  int M, N, K;
  int mode;
  T beta;
  int tri;     // A is lower triangular: row tile i0 needs k < i0 + BM only
  int mask;    // read only A's lower triangle (zeros above; ones on the diagonal if unit); plain loads
  int unit;
  int kchunk;  // K per z-slice (a multiple of BK); K when not split
  T *P;        // PARTIAL: slices of M x N (ld M)
  T *C2;       // rows < split_rows are written to C2 (ld ldc2) instead of C; old values still come from C
  int64_t ldc2;
  int split_rows;
  const int *skip;  // device flag: when set, the launch does nothing
  unsigned int *err;
  uint64_t limit_ns;
};

template <class T, class TL>
constexpr int stage_bytes() {
  return (GemmK<T>::BK * TL::BM + TL::BN * GemmK<T>::BK) * (int)sizeof(T);
}
constexpr int kStages = 3;

__device__ __forceinline__ void dmma884(double &d0, double &d1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(d0), "+d"(d1)
               : "d"(a), "d"(b));
}

template <class T, class TL>
struct Acc;
template <class TL>
struct Acc<double, TL> {
  double v[TL::WM][TL::WN][2];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < TL::WM; ++i)
#pragma unroll
      for (int j = 0; j < TL::WN; ++j) v[i][j][0] = v[i][j][1] = 0.0;
  }
  __device__ __forceinline__ double get(int i, int j, int q) const { return v[i][j][q]; }
};
template <class TL>
struct Acc<cplx, TL> {
  double re[TL::WM][TL::WN][2];
  double im[TL::WM][TL::WN][2];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < TL::WM; ++i)
#pragma unroll
      for (int j = 0; j < TL::WN; ++j) re[i][j][0] = re[i][j][1] = im[i][j][0] = im[i][j][1] = 0.0;
  }
  __device__ __forceinline__ cplx get(int i, int j, int q) const { return cplx{re[i][j][q], im[i][j][q]}; }
};

// one BK-deep slice from shared memory: sA[k][BM], sB[BN][k]
template <class TL>
__device__ __forceinline__ void mma_slice(Acc<double, TL> &acc, const double *sA, const double *sB, int wm, int wn,
                                          int g, int t) {
  constexpr int BK = GemmK<double>::BK;
#pragma unroll
  for (int kk = 0; kk < BK; kk += 4) {
    double a[TL::WM], b[TL::WN];
#pragma unroll
    for (int i = 0; i < TL::WM; ++i) a[i] = sA[(kk + t) * TL::BM + wm * TL::WM * 8 + i * 8 + g];
#pragma unroll
    for (int jn = 0; jn < TL::WN; ++jn) b[jn] = sB[(wn * TL::WN * 8 + jn * 8 + g) * BK + kk + t];
#pragma unroll
    for (int i = 0; i < TL::WM; ++i)
#pragma unroll
      for (int jn = 0; jn < TL::WN; ++jn) dmma884(acc.v[i][jn][0], acc.v[i][jn][1], a[i], b[jn]);
  }
}

template <class TL>
__device__ __forceinline__ void mma_slice(Acc<cplx, TL> &acc, const cplx *sA, const cplx *sB, int wm, int wn, int g,
                                          int t) {
  constexpr int BK = GemmK<cplx>::BK;
#pragma unroll
  for (int kk = 0; kk < BK; kk += 4) {
    cplx a[TL::WM], b[TL::WN];
#pragma unroll
    for (int i = 0; i < TL::WM; ++i) a[i] = sA[(kk + t) * TL::BM + wm * TL::WM * 8 + i * 8 + g];
#pragma unroll
    for (int jn = 0; jn < TL::WN; ++jn) b[jn] = sB[(wn * TL::WN * 8 + jn * 8 + g) * BK + kk + t];
#pragma unroll
    for (int i = 0; i < TL::WM; ++i)
#pragma unroll
      for (int jn = 0; jn < TL::WN; ++jn) {
        dmma884(acc.re[i][jn][0], acc.re[i][jn][1], a[i].re, b[jn].re);
        dmma884(acc.re[i][jn][0], acc.re[i][jn][1], -a[i].im, b[jn].im);
        dmma884(acc.im[i][jn][0], acc.im[i][jn][1], a[i].re, b[jn].im);
        dmma884(acc.im[i][jn][0], acc.im[i][jn][1], a[i].im, b[jn].re);
      }
  }
}

__device__ __forceinline__ double sub(double a, double b) { return a - b; }
__device__ __forceinline__ cplx sub(cplx a, cplx b) { return cplx{a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ double add(double a, double b) { return a + b; }
__device__ __forceinline__ cplx add(cplx a, cplx b) { return cplx{a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ bool is_one(double a) { return a == 1.0; }
__device__ __forceinline__ bool is_one(cplx a) { return a.re == 1.0 && a.im == 0.0; }

// out = beta*C - v (UPDATE) or beta*v (SCALE)
template <class T>
__device__ __forceinline__ void finish_elem(int mode, T beta, bool b1, T *cp, T v) {
  using E = Elem<T>;
  if (mode == MODE_UPDATE) {
    const T old = *cp;
    *cp = sub(b1 ? old : E::mul(beta, old), v);
  } else {
    *cp = b1 ? v : E::mul(beta, v);
  }
}

template <class T, class TL>
__device__ __forceinline__ void epilogue(const GemmArgs<T> &p, const Acc<T, TL> &acc, int m0, int n0, int wm, int wn,
                                         int g, int t) {
  using E = Elem<T>;
  const bool b1 = is_one(p.beta);
  T *P = p.P + (size_t)blockIdx.z * p.M * p.N;
#pragma unroll
  for (int i = 0; i < TL::WM; ++i) {
    const int row = m0 + wm * TL::WM * 8 + i * 8 + g;
    if (row >= p.M) continue;
    if (p.mode == MODE_PARTIAL) {
#pragma unroll
      for (int jn = 0; jn < TL::WN; ++jn)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int col = n0 + wn * TL::WN * 8 + jn * 8 + 2 * t + q;
          if (col < p.N) P[row + (size_t)col * p.M] = acc.get(i, jn, q);
        }
      continue;
    }
    // this row's old values of C first, then the results (loads do not wait behind stores)
    T old[TL::WN][2];
    if (p.mode == MODE_UPDATE) {
#pragma unroll
      for (int jn = 0; jn < TL::WN; ++jn)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int col = n0 + wn * TL::WN * 8 + jn * 8 + 2 * t + q;
          old[jn][q] = col < p.N ? p.C[row + (int64_t)col * p.ldc] : E::zero();
        }
    }
    const bool redirect = row < p.split_rows;
#pragma unroll
    for (int jn = 0; jn < TL::WN; ++jn)
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int col = n0 + wn * TL::WN * 8 + jn * 8 + 2 * t + q;
        if (col >= p.N) continue;
        const T v = acc.get(i, jn, q);
        T *cp = redirect ? p.C2 + row + (int64_t)col * p.ldc2 : p.C + row + (int64_t)col * p.ldc;
        if (p.mode == MODE_UPDATE)
          *cp = sub(b1 ? old[jn][q] : E::mul(p.beta, old[jn][q]), v);
        else
          *cp = b1 ? v : E::mul(p.beta, v);
      }
  }
}

// words per element for the 8-byte TMA view of T
template <class T>
constexpr int words() {
  return (int)(sizeof(T) / 8);
}

template <class T, class TL, bool kTma>
__global__ void __launch_bounds__(GEMM_THREADS) gemm_kernel(const GemmArgs<T> p,
                                                            const __grid_constant__ CUtensorMap mapA,
                                                            const __grid_constant__ CUtensorMap mapB) {
  constexpr int BK = GemmK<T>::BK, BM = TL::BM, BN = TL::BN;
  constexpr int SB = stage_bytes<T, TL>();
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[kStages];
  if (p.skip != nullptr && *(volatile const int *)p.skip != 0) return;
  unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
  auto sA = [&](int s) { return reinterpret_cast<T *>(smem + s * SB); };
  auto sB = [&](int s) { return reinterpret_cast<T *>(smem + s * SB + BK * BM * sizeof(T)); };

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wm = warp % TL::WARPS_M, wn = warp / TL::WARPS_M, g = lane >> 2, t = lane & 3;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int kall = p.tri ? min(p.K, m0 + BM) : p.K;
  const int kbeg = blockIdx.z * p.kchunk;
  const int kend = min(kall, kbeg + p.kchunk);
  const int nk = kend > kbeg ? (kend - kbeg + BK - 1) / BK : 0;

  Acc<T, TL> acc;
  acc.zero();

  if constexpr (kTma) {
    if (tid == 0) {
      for (int s = 0; s < kStages; ++s) mbar_init(&full[s], 1);
      fence_mbar_init();
    }
    __syncthreads();
    auto issue = [&](int kt, int s) {
      mbar_arrive_expect_tx(&full[s], SB);
      tma_load_2d(sA(s), &mapA, &full[s], m0 * words<T>(), kbeg + kt * BK);
      tma_load_2d(sB(s), &mapB, &full[s], (kbeg + kt * BK) * words<T>(), n0);
    };
    if (tid == 0)
      for (int s = 0; s < kStages && s < nk; ++s) issue(s, s);
    int kt = 0;
    for (; kt < nk; ++kt) {
      const int s = kt % kStages;
      const bool ok = mbar_wait_bounded(&full[s], (kt / kStages) & 1, p.limit_ns, p.err);
      if (__syncthreads_or(!ok)) break;
      mma_slice(acc, sA(s), sB(s), wm, wn, g, t);
      __syncthreads();
      if (tid == 0 && kt + kStages < nk) issue(kt + kStages, s);
    }
    if (kt < nk) {
      // timed out: let the copies this CTA issued land (bounded) before leaving
      if (tid == 0)
        for (int k2 = kt; k2 < nk && k2 < kt + kStages; ++k2)
          mbar_wait_bounded(&full[k2 % kStages], (k2 / kStages) & 1, p.limit_ns, p.err);
      return;
    }
  } else {
    using E = Elem<T>;
    for (int kt = 0; kt < nk; ++kt) {
      T *a = sA(0), *b = sB(0);
      const int k0 = kbeg + kt * BK;
      for (int e = tid; e < BK * BM; e += GEMM_THREADS) {
        const int kk = e / BM, mm = e % BM;
        const int row = m0 + mm, col = k0 + kk;
        T v = (row < p.M && col < p.K && !(p.mask && col > row)) ? E::ld(p.A + row + (int64_t)col * p.lda)
                                                                   : E::zero();
        if (p.mask && p.unit && col == row && row < p.M) v = E::one();
        a[e] = v;
      }
      for (int e = tid; e < BN * BK; e += GEMM_THREADS) {
        const int nn = e / BK, kk = e % BK;
        const int row = k0 + kk, col = n0 + nn;
        b[e] = (row < p.K && col < p.N) ? E::ld(p.Bm + row + (int64_t)col * p.ldb) : E::zero();
      }
      __syncthreads();
      mma_slice(acc, a, b, wm, wn, g, t);
      __syncthreads();
    }
  }
  epilogue(p, acc, m0, n0, wm, wn, g, t);
}

// C = mode(beta C, sum_z P[z]) over the M x N region, z in increasing order
template <class T>
__global__ void __launch_bounds__(256) reduce_partials_kernel(const T *__restrict__ P, int S, int M, int N, T *C,
                                                              int64_t ldc, T *C2, int64_t ldc2, int split_rows,
                                                              int mode, T beta) {
  using E = Elem<T>;
  const int64_t total = (int64_t)M * N;
  const bool b1 = is_one(beta);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    T v = P[e];
    for (int z = 1; z < S; ++z) v = add(v, P[e + (int64_t)z * total]);
    const int row = (int)(e % M), col = (int)(e / M);
    const T *src = C + row + (int64_t)col * ldc;
    T *dst = row < split_rows ? C2 + row + (int64_t)col * ldc2 : C + row + (int64_t)col * ldc;
    if (mode == MODE_UPDATE)
      *dst = sub(b1 ? *src : E::mul(beta, *src), v);
    else
      *dst = b1 ? v : E::mul(beta, v);
  }
}

template <class T, class TL>
size_t gemm_smem_bytes(bool tma) {
  return (size_t)(tma ? kStages : 1) * stage_bytes<T, TL>() + 128;
}

template <class T, class TL>
hsma_status_t gemm_attrs() {
  static DeviceFlags done;
  if (done.test()) return HSMA_OK;
  HSMA_CUDA_TRY(cudaFuncSetAttribute(gemm_kernel<T, TL, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)gemm_smem_bytes<T, TL>(true)));
  HSMA_CUDA_TRY(cudaFuncSetAttribute(gemm_kernel<T, TL, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)gemm_smem_bytes<T, TL>(false)));
  done.set();
  return HSMA_OK;
}

template <class T>
bool tma_ok(const void *p, int64_t ld) {
  return ((uintptr_t)p % 16 == 0) && ((ld * (int64_t)sizeof(T)) % 16 == 0);
}

int sm_count() { return hsma_sm_count(); }

// Elements of partial-product workspace the split products of one solve may
// need: a product is split only while its tiles number fewer than two per SM,
// so S x M x N stays below 2 x SMs x (one tile) for either tile shape.
size_t partial_elems_max() {
  const size_t sms = (size_t)sm_count();
  return 2 * sms * 64 * 64 + 2 * sms * 128 * 16;
}

template <class T, class TL>
hsma_status_t gemm_tiled(const GemmArgs<T> &p0, const char *phase, cudaStream_t st, T *P, size_t P_elems) {
  hsma_status_t s = gemm_attrs<T, TL>();
  if (s != HSMA_OK) return s;
  constexpr int BK = GemmK<T>::BK;
  GemmArgs<T> p = p0;
  p.err = hsma_dev_error_ptr();
  if (p.err == nullptr) return HSMA_ERR_CUDA;
  if (p.limit_ns == 0) p.limit_ns = 4000000000ull;  // 4 s of wall time per barrier wait
  const int tiles_m = (p.M + TL::BM - 1) / TL::BM, tiles_n = (p.N + TL::BN - 1) / TL::BN;
  // split K while the tiles alone leave the GPU short of two CTAs per SM
  int S = 1;
  const int target = 2 * sm_count();
  if (P != nullptr && (int64_t)tiles_m * tiles_n < target) {
    S = target / (tiles_m * tiles_n);
    S = std::min(S, std::max(1, p.K / (2 * BK)));
    S = std::min(S, 16);
    while (S > 1 && (size_t)S * p.M * p.N > P_elems) --S;
  }
  p.kchunk = S > 1 ? ((p.K + S - 1) / S + BK - 1) / BK * BK : p.K;
  if (S > 1) S = (p.K + p.kchunk - 1) / p.kchunk;
  const int final_mode = p.mode;
  if (S > 1) {
    p.mode = MODE_PARTIAL;
    p.P = P;
  }
  const bool use_tma = !p.mask && tma_ok<T>(p.A, p.lda) && tma_ok<T>(p.Bm, p.ldb);
  CUtensorMap ma, mb;
  std::memset(&ma, 0, sizeof ma);
  std::memset(&mb, 0, sizeof mb);
  if (use_tma) {
    constexpr int w = words<T>();
    if (!hsma_make_map_2d(&ma, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 8, p.A, (uint64_t)p.M * w, (uint64_t)p.K,
                          (uint64_t)p.lda * w, TL::BM * w, BK) ||
        !hsma_make_map_2d(&mb, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 8, p.Bm, (uint64_t)p.K * w, (uint64_t)p.N,
                          (uint64_t)p.ldb * w, BK * w, TL::BN))
      return HSMA_ERR_CUDA;
  }
  dim3 grid(tiles_m, tiles_n, S);
  if (grid.y > 65535) return HSMA_ERR_UNSUPPORTED;
  {
    HsmaTraceScope ts(phase, st);
    if (use_tma)
      gemm_kernel<T, TL, true><<<grid, GEMM_THREADS, gemm_smem_bytes<T, TL>(true), st>>>(p, ma, mb);
    else
      gemm_kernel<T, TL, false><<<grid, GEMM_THREADS, gemm_smem_bytes<T, TL>(false), st>>>(p, ma, mb);
  }
  HSMA_CUDA_TRY(cudaGetLastError());
  if (S > 1) {
    const int64_t total = (int64_t)p.M * p.N;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 4 * sm_count());
    HsmaTraceScope ts("reduce", st);
    reduce_partials_kernel<T><<<blocks, 256, 0, st>>>(P, S, p.M, p.N, p.C, p.ldc, p.C2, p.ldc2, p.split_rows,
                                                      final_mode, p.beta);
    HSMA_CUDA_TRY(cudaGetLastError());
  }
  return HSMA_OK;
}

// Launch one product.  Tile shape: `tile` (HSMA_TILE_*), or by n when 0
// (128 x 8 for n <= 8, 128 x 16 for n <= 48, else 64 x 64).  K is split across
// CTAs when the output alone has too few tiles and a partial-product
// workspace P is given (P = nullptr: never).  `phase` names it for the tracer.
template <class T>
hsma_status_t gemm(const GemmArgs<T> &p, const char *phase, cudaStream_t st, T *P = nullptr, size_t P_elems = 0,
                   int tile = 0) {
  if (p.M <= 0 || p.N <= 0) return HSMA_OK;
  if (tile == 0) tile = p.N <= 8 ? HSMA_TILE_128x8 : p.N <= 48 ? HSMA_TILE_128x16 : HSMA_TILE_64x64;
  if (tile == HSMA_TILE_128x8) return gemm_tiled<T, TileN8>(p, phase, st, P, P_elems);
  if (tile == HSMA_TILE_128x16) return gemm_tiled<T, TileN16>(p, phase, st, P, P_elems);
  return gemm_tiled<T, TileWide>(p, phase, st, P, P_elems);
}

template <class T, int G>
hsma_status_t launch_inverse_g(const T *A, int64_t lda, int64_t m, int unit, T *Dinv, cudaStream_t st) {
  constexpr int NB = 32 * G, C = 32 / G;
  const int warps = std::min(8, NB / C);
  const int CT = warps * C;
  dim3 grid((unsigned)((m + NB - 1) / NB), (unsigned)(NB / CT));
  HsmaTraceScope ts("diag_inverse", st);
  diag_inverse_kernel<T, G><<<grid, warps * 32, 0, st>>>(A, lda, m, unit, Dinv);
  HSMA_CUDA_TRY(cudaGetLastError());
  return HSMA_OK;
}

template <class T>
hsma_status_t launch_inverse(int nb, const T *A, int64_t lda, int64_t m, int unit, T *Dinv, cudaStream_t st) {
  switch (nb) {
    case 32: return launch_inverse_g<T, 1>(A, lda, m, unit, Dinv, st);
    case 64: return launch_inverse_g<T, 2>(A, lda, m, unit, Dinv, st);
    case 128: return launch_inverse_g<T, 4>(A, lda, m, unit, Dinv, st);
    case 256: return launch_inverse_g<T, 8>(A, lda, m, unit, Dinv, st);
    case 512: return launch_inverse_g<T, 16>(A, lda, m, unit, Dinv, st);
    default: return HSMA_ERR_UNSUPPORTED;
  }
}

template <class T>
T make_scalar(const double *a);
template <>
double make_scalar<double>(const double *a) {
  return a[0];
}
template <>
cplx make_scalar<cplx>(const double *a) {
  return cplx{a[0], a[1]};
}

// Blocked two-phase solve (Section 4.3).  Phase 1 inverts every diagonal
// block; phase 2 walks the block rows r: X_r = D_r^{-1} W, where W holds the
// block row's right-hand side after the updates, and the updates are either
//   right-looking: after X_r, B_{r+1:} -= A_{r+1:, r} X_r (one product with
//                  M = m - r0 - s_r rows, K = s_r; the next block row goes to W);
//   left-looking:  before X_r, W = alpha B_r - A_{r, 0:r} X_{0:r} (one product
//                  with M = s_r rows, K = r0, the paper's form of the update).
// alpha is applied once, to each block row's first use.
template <class T>
hsma_status_t blocked_impl(const HsmaBlockedCfg &cfg, const T *A, int64_t lda, T *B, int64_t ldb, int64_t m,
                           int64_t n, const double *alpha, int unit, cudaStream_t st) {
  const int nb = cfg.nb;
  const bool left = cfg.looking == HSMA_LOOK_LEFT;
  const int64_t nblk = (m + nb - 1) / nb;
  const T al = make_scalar<T>(alpha);
  const T one = make_scalar<T>((const double[2]){1.0, 0.0});
  void *ws = nullptr;
  const size_t dinv_bytes = sizeof(T) * (size_t)nblk * nb * nb;
  const size_t w_bytes = sizeof(T) * (size_t)nb * n;
  // partial products of split-K launches (only when n is small, unless split K is off)
  const size_t p_elems =
      cfg.split_k != HSMA_SPLITK_OFF && (size_t)n * 64 < (size_t)2 * sm_count() * 64 * 64 ? partial_elems_max() : 0;
  hsma_status_t s = hsma_ws_alloc(&ws, dinv_bytes + w_bytes + sizeof(T) * p_elems, st);
  if (s != HSMA_OK) return s;
  T *Dinv = static_cast<T *>(ws);
  T *W = reinterpret_cast<T *>(static_cast<unsigned char *>(ws) + dinv_bytes);
  T *Pw = p_elems ? reinterpret_cast<T *>(static_cast<unsigned char *>(ws) + dinv_bytes + w_bytes) : nullptr;
  s = launch_inverse<T>(nb, A, lda, m, unit, Dinv, st);
  // W holds the current block row's right-hand side: copied from B for the
  // first block, written by the previous trailing update for the others, so
  // the solve product can write X_r straight into B_r.
  if (s == HSMA_OK) {
    HsmaTraceScope ts("copy", st, 0);
    const int s0 = (int)std::min<int64_t>(nb, m);
    cudaError_t e = cudaMemcpy2DAsync(W, sizeof(T) * nb, B, sizeof(T) * ldb, sizeof(T) * s0, n,
                                      cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) s = hsma_from_cuda(e);
  }
  for (int64_t r = 0; r < nblk && s == HSMA_OK; ++r) {
    const int64_t r0 = r * nb;
    const int sr = (int)std::min<int64_t>(nb, m - r0);
    if (left && r > 0) {
      // W = alpha B_r - A_{r, 0:r} X_{0:r}
      GemmArgs<T> pl{};
      pl.A = A + r0;
      pl.lda = lda;
      pl.Bm = B;
      pl.ldb = ldb;
      pl.C = B + r0;
      pl.ldc = ldb;
      pl.C2 = W;
      pl.ldc2 = nb;
      pl.split_rows = sr;
      pl.M = sr;
      pl.N = (int)n;
      pl.K = (int)r0;
      pl.mode = MODE_UPDATE;
      pl.beta = al;
      pl.tri = 0;
      s = gemm<T>(pl, "update_gemm", st, Pw, p_elems, cfg.tile);
      if (s != HSMA_OK) break;
    }
    // X_r = D_r^{-1} (scale * W)
    GemmArgs<T> ps{};
    ps.A = Dinv + (size_t)r * nb * nb;
    ps.lda = nb;
    ps.Bm = W;
    ps.ldb = nb;
    ps.C = B + r0;
    ps.ldc = ldb;
    ps.M = sr;
    ps.N = (int)n;
    ps.K = sr;
    ps.mode = MODE_SCALE;
    ps.beta = r == 0 ? al : one;
    ps.tri = 1;
    s = gemm<T>(ps, "solve_gemm", st, Pw, p_elems, cfg.tile);
    if (s != HSMA_OK || r0 + sr >= m) break;
    if (left) continue;
    // B_{r+1:} = beta B_{r+1:} - A_{r+1:, r} X_r; the next block row goes to W
    GemmArgs<T> pu{};
    pu.A = A + (r0 + sr) + r0 * lda;
    pu.lda = lda;
    pu.Bm = B + r0;
    pu.ldb = ldb;
    pu.C = B + r0 + sr;
    pu.ldc = ldb;
    pu.C2 = W;
    pu.ldc2 = nb;
    pu.split_rows = (int)std::min<int64_t>(nb, m - r0 - sr);
    pu.M = (int)(m - r0 - sr);
    pu.N = (int)n;
    pu.K = sr;
    pu.mode = MODE_UPDATE;
    pu.beta = r == 0 ? al : one;
    pu.tri = 0;
    s = gemm<T>(pu, "update_gemm", st, Pw, p_elems, cfg.tile);
  }
  hsma_status_t f = hsma_ws_free(ws, st);
  return s != HSMA_OK ? s : f;
}

}  // namespace

int hsma_sm_count() {
  static int n[64] = {0};
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= 64) return kHsmaDefaultSms;
  if (n[d] == 0) cudaDeviceGetAttribute(&n[d], cudaDevAttrMultiProcessorCount, d);
  return n[d] > 0 ? n[d] : kHsmaDefaultSms;
}

unsigned int *hsma_dev_error_ptr() {
  static unsigned int *ptr[64] = {nullptr};
  static std::mutex mu;
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  if (ptr[d] == nullptr && cudaGetSymbolAddress((void **)&ptr[d], g_hsma_dev_error) != cudaSuccess) ptr[d] = nullptr;
  return ptr[d];
}

hsma_status_t hsma_diag_inverse(int dtype, int nb, const void *A, int64_t lda, int64_t m, int unit, void *Dinv,
                                cudaStream_t st) {
  switch (dtype) {
    case HSMA_C128:
      return launch_inverse<cplx>(nb, static_cast<const cplx *>(A), lda, m, unit, static_cast<cplx *>(Dinv), st);
    case HSMA_R32_BF16:
      return launch_inverse<float>(nb, static_cast<const float *>(A), lda, m, unit, static_cast<float *>(Dinv), st);
    default:
      return launch_inverse<double>(nb, static_cast<const double *>(A), lda, m, unit, static_cast<double *>(Dinv),
                                    st);
  }
}

hsma_status_t hsma_residual_f64(const double *A, int64_t lda, int unit, const double *X, int64_t ldx, double *C,
                                int64_t ldc, int64_t m, int64_t n, double beta, const int *skip, cudaStream_t st) {
  if (m > INT32_MAX || n > INT32_MAX) return HSMA_ERR_UNSUPPORTED;
  GemmArgs<double> p{};
  p.A = A;
  p.lda = lda;
  p.Bm = X;
  p.ldb = ldx;
  p.C = C;
  p.ldc = ldc;
  p.M = (int)m;
  p.N = (int)n;
  p.K = (int)m;
  p.mode = MODE_UPDATE;
  p.beta = beta;
  p.tri = 1;
  p.mask = 1;
  p.unit = unit;
  p.skip = skip;
  return gemm<double>(p, "residual", st);
}

// ---------------------------------------------------------------------------
PFN_encodeTiled hsma_encode_fn() {
  static PFN_encodeTiled fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_encodeTiled>(p);
  });
  return fn;
}

bool hsma_make_map_2d(CUtensorMap *map, CUtensorMapDataType dt, int elem_bytes, const void *base, uint64_t rows,
                      uint64_t cols, uint64_t ld_elems, uint32_t box_rows, uint32_t box_cols, CUtensorMapSwizzle swz) {
  PFN_encodeTiled enc = hsma_encode_fn();
  if (enc == nullptr) return false;
  if ((uintptr_t)base % 16 != 0 || (ld_elems * elem_bytes) % 16 != 0) return false;
  const cuuint64_t dims[2] = {rows, cols};
  const cuuint64_t strides[1] = {ld_elems * (uint64_t)elem_bytes};
  const cuuint32_t box[2] = {box_rows, box_cols};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, dt, 2, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

hsma_status_t hsma_blocked_solve(int dtype, const HsmaBlockedCfg &cfg, const void *A, int64_t lda, void *B,
                                 int64_t ldb, int64_t m, int64_t n, const double *alpha, int unit, cudaStream_t st) {
  if (n > INT32_MAX || m > INT32_MAX) return HSMA_ERR_UNSUPPORTED;
  if (dtype == HSMA_C128)
    return blocked_impl<cplx>(cfg, static_cast<const cplx *>(A), lda, static_cast<cplx *>(B), ldb, m, n, alpha,
                              unit, st);
  return blocked_impl<double>(cfg, static_cast<const double *>(A), lda, static_cast<double *>(B), ldb, m, n, alpha,
                              unit, st);
}

extern "C" HSMA_API hsma_status_t hsma_device_status(unsigned int *out) {
  if (out == nullptr) return HSMA_ERR_INVALID_ARG;
  unsigned int v = 0, z = 0;
  HSMA_CUDA_TRY(cudaDeviceSynchronize());
  HSMA_CUDA_TRY(cudaMemcpyFromSymbol(&v, g_hsma_dev_error, sizeof v));
  HSMA_CUDA_TRY(cudaMemcpyToSymbol(g_hsma_dev_error, &z, sizeof z));
  *out = v;
  return HSMA_OK;
}
