// Small-case direct solve (m <= 64), single and varlen-batched.
//
// Section 4.2.1: the triangle of A stays in shared memory, the columns of B
// (becoming X) stay in registers, and rows are solved in order; each solved
// row x_i updates the rows below it with column i of A.  On this GPU the FP64
// pipe, not memory, bounds the work (a warp-wide FP64 instruction occupies a
// sub-partition for 64 cycles and masked lanes still pay), so the layout is
// chosen to keep FP64 lanes busy:
//
//  * a warp owns C = 32/G columns; the rows of each column are spread over G
//    lanes (row r in lane group r % G, register slot r / G).  G is chosen per
//    instance by a cost model counting warp-wide FP64 instructions;
//  * the diagonal is folded in while staging: row r of the strict lower
//    triangle is stored pre-multiplied by 1/a_rr and B's row r by alpha/a_rr,
//    so a solved value needs no further arithmetic before it is broadcast
//    (warp shuffle when G > 1);
//  * the substitution is fully unrolled so X stays in registers; steps past
//    m and slots past ceil(m/G) are skipped with warp-uniform branches.
//
// The per-instance arithmetic is independent of the batch it sits in.  The
// kernels can read A and B through an index map (row reversal, transposed or
// conjugated reads), which gives the other left-side variants without copies;
// the paper's case runs a kernel without the map.
#include <cuda_runtime.h>

#include <mutex>
#include <type_traits>

#include "common.cuh"
#include "small.h"
#include "trace.h"

namespace {

// Warps per CTA of the single-solve kernel and of the batched kernel, the
// batched kernel's minimum resident CTAs per SM (register cap; 0 = none) and
// its set of row-group variants (bit log2(G)).  Defaults chosen by measurement.
#ifndef HSMA_VB_WARPS
#define HSMA_VB_WARPS 4
#endif
#ifndef HSMA_VB_MINB
#define HSMA_VB_MINB 3
#endif
// FP32 element types: the FP32 pipe leaves the kernel bound by load and
// barrier latency, so more CTAs per SM pay off (and fit: half the registers).
#ifndef HSMA_VB_MINB_F32
#define HSMA_VB_MINB_F32 6
#endif
#ifndef HSMA_VB_GMASK
#define HSMA_VB_GMASK 0xFu
#endif
// Single solve: four warps per CTA, one per SM sub-partition (each
// sub-partition has its own FP64 pipe, which bounds a warp's substitution
// steps), sharing one staged triangle.
constexpr int kWarpsSingle = 4;
constexpr int kWarpsBatched = HSMA_VB_WARPS;
constexpr unsigned kBatchedGMask = HSMA_VB_GMASK;

// packed strict-lower triangle: column i holds rows i+1 .. MMAX-1
__host__ __device__ constexpr int col_off(int i, int mmax) { return i * (mmax - 1) - (i * (i - 1)) / 2; }
__host__ __device__ constexpr int tri_elems(int mmax) { return col_off(mmax, mmax); }

// Index map from the solved lower-triangular form onto the caller's operand
// (the other left-side variants): with rev, row r of the form is row m-1-r of
// the operand (and of B); with tr, A is read transposed; with cj, conjugated.
// The identity map is the paper's left / lower / no-transpose case.
struct SmallMap {
  int rev, tr, cj;
};

template <class T, bool MAP>
__device__ __forceinline__ T map_ld(const T *A, int64_t lda, int m, int r, int i, SmallMap mp) {
  if constexpr (!MAP) return Elem<T>::ld(A + r + (int64_t)i * lda);
  int p = mp.rev ? m - 1 - r : r, q = mp.rev ? m - 1 - i : i;
  if (mp.tr) {
    const int t = p;
    p = q;
    q = t;
  }
  T v = Elem<T>::ld(A + p + (int64_t)q * lda);
  if constexpr (Elem<T>::kComplex) {
    if (mp.cj) v.im = -v.im;
  }
  return v;
}

template <class T>
struct SmemLayout {
  // triangle, then c_r = alpha/a_rr, then 1/a_rr
  __host__ __device__ static constexpr size_t bytes(int mmax) { return sizeof(T) * (tri_elems(mmax) + 2 * mmax); }
};

// Stage one instance: 1/a_rr and alpha/a_rr for every row r < MMAX (1 and 0
// past m), then the strict lower triangle with row r pre-multiplied by 1/a_rr,
// for the columns the substitution reads (i < m - 1) and rows i + 1 ..
// rows_used - 1 (zeros past m).  The threads walk those elements in packed
// order (consecutive elements in consecutive threads, four in flight), so
// every thread does useful work on every pass and the index arithmetic stays
// small.  All threads of the CTA take part; ends with a CTA barrier.
template <class T, int MMAX, int W, bool MAP>
__device__ __forceinline__ void stage(T *sTri, T *sC, T *sR, const T *__restrict__ A, int64_t lda, int m,
                                            int rows_used, T alpha, bool unit, SmallMap mp) {
  using E = Elem<T>;
  const int tid = threadIdx.x;
  for (int r = tid; r < MMAX; r += 32 * W) {
    T rv = E::one();
    if (r < m && !unit) rv = E::recip(map_ld<T, MAP>(A, lda, m, r, r, mp));
    sR[r] = rv;
    sC[r] = (r < m) ? E::mul(alpha, rv) : E::zero();
  }
  __syncthreads();
  int i = 0, loc = tid;
  auto advance = [&](int by) {
    loc += by;
    while (i < m - 1 && loc >= rows_used - 1 - i) {
      loc -= rows_used - 1 - i;
      ++i;
    }
  };
  advance(0);
  while (i < m - 1) {
    int rr[4], ii[4];
    T vv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {  // four elements in flight: loads first
      ii[u] = i;
      rr[u] = i + 1 + loc;
      vv[u] = (i < m - 1 && rr[u] < m) ? map_ld<T, MAP>(A, lda, m, rr[u], i, mp) : E::zero();
      advance(32 * W);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (ii[u] < m - 1) sTri[col_off(ii[u], MMAX) - ii[u] - 1 + rr[u]] = E::mul(sR[rr[u]], vv[u]);
  }
  __syncthreads();
}

// The B entries of a lane's rows in one column tile (zero outside the
// instance), loaded before the solve so that they can be in flight while the
// triangle is staged.
template <class T, int G, int MMAX, bool MAP, bool FULL = false>
__device__ __forceinline__ void warp_load_b(T (&b)[MMAX / G], const T *Bt, int64_t ldb, int m_, int ncols, int rev) {
  using E = Elem<T>;
  constexpr int R = MMAX / G;
  const int m = FULL ? MMAX : m_;
  const int lane = threadIdx.x & 31;
  const int g = lane % G, c = lane / G;
  const bool colok = c < ncols;
  const T *Bp = Bt + (int64_t)(colok ? c : 0) * ldb;
#pragma unroll
  for (int t = 0; t < R; ++t) {
    const int r = g + t * G;
    b[t] = E::zero();
    if (t * G < m) {
      if (colok && r < m) b[t] = E::ld(Bp + (MAP && rev ? m - 1 - r : r));
    }
  }
}

// One warp solves one column tile (up to 32/G columns starting at Bt) whose
// B entries warp_load_b has loaded.
// FULL: m == MMAX, known at compile time (the bound checks fold away).
template <class T, int G, int MMAX, bool MAP, bool FULL = false>
__device__ __forceinline__ void warp_solve_loaded(const T (&b)[MMAX / G], const T *sTri, const T *sC, T *Bt,
                                                  int64_t ldb, int m_, int ncols, int rev) {
  using E = Elem<T>;
  constexpr int R = MMAX / G;
  const int m = FULL ? MMAX : m_;
  const int lane = threadIdx.x & 31;
  const int g = lane % G, c = lane / G;
  const bool colok = c < ncols;
  T *Bp = Bt + (int64_t)(colok ? c : 0) * ldb;

  T s[R];
#pragma unroll
  for (int t = 0; t < R; ++t) {
    const int r = g + t * G;
    s[t] = E::zero();
    if (t * G < m) {
      if (colok && r < m) s[t] = E::mul(sC[r], b[t]);
    }
  }

#pragma unroll
  for (int i = 0; i < MMAX - 1; ++i) {
    if (i >= m - 1) break;  // warp-uniform: the last row updates nothing
    const int tb = i / G, gi = i % G;
    const T x = (G == 1) ? s[tb] : E::shfl(s[tb], c * G + gi);
    const T *col = sTri + col_off(i, MMAX) - i - 1;
    if (G > 1 && gi < G - 1) {
      // boundary slot: only rows strictly below i update
      const int r = g + tb * G;
      const int ra = r > i ? r : i + 1;
      const T ns = E::fms(col[ra], x, s[tb]);
      if (r > i) s[tb] = ns;
    }
#pragma unroll
    for (int t = tb + 1; t < R; ++t) {
      if (t * G >= m) break;  // warp-uniform
      s[t] = E::fms(col[g + t * G], x, s[t]);
    }
  }

#pragma unroll
  for (int t = 0; t < R; ++t) {
    const int r = g + t * G;
    if (t * G < m) {
      if (colok && r < m) E::st(Bp + (MAP && rev ? m - 1 - r : r), s[t]);
    }
  }
}

template <class T, int G, int MMAX, bool MAP, bool FULL = false>
__device__ __forceinline__ void warp_solve(const T *sTri, const T *sC, T *Bt, int64_t ldb, int m, int ncols,
                                           int rev) {
  T b[MMAX / G];
  warp_load_b<T, G, MMAX, MAP, FULL>(b, Bt, ldb, m, ncols, rev);
  warp_solve_loaded<T, G, MMAX, MAP, FULL>(b, sTri, sC, Bt, ldb, m, ncols, rev);
}

template <class T, int G, int MMAX, bool MAP, bool FULL = false>
__device__ __forceinline__ void solve_tiles(const T *sTri, const T *sC, T *B, int64_t ldb, int m, int n, int tile0,
                                            int tile_step, int rev) {
  constexpr int C = 32 / G;
  const int warp = threadIdx.x >> 5;
  const int ntiles = (n + C - 1) / C;
  for (int t = tile0 + warp; t < ntiles; t += tile_step) {
    const int col0 = t * C;
    const int nc = (n - col0) < C ? (n - col0) : C;
    warp_solve<T, G, MMAX, MAP, FULL>(sTri, sC, B + (int64_t)col0 * ldb, ldb, m, nc, rev);
  }
}

template <class T, int W>
__device__ __forceinline__ void zero_tiles(T *B, int64_t ldb, int m, int n) {
  for (int j = threadIdx.x >> 5; j < n; j += W)
    for (int r = threadIdx.x & 31; r < m; r += 32) Elem<T>::st(B + r + (int64_t)j * ldb, Elem<T>::zero());
}

// Dispatch over the row-group variants compiled into the batched kernel.
template <class T, bool MAP>
struct Variants {
  static constexpr bool kCplx = Elem<T>::kComplex;
  __device__ __forceinline__ static void run(int g, const T *sTri, const T *sC, T *B, int64_t ldb, int m, int n,
                                             int tile0, int step, int rev) {
    if constexpr ((kBatchedGMask & 1u) != 0) {
      if (g == 1) {
        solve_tiles<T, 1, kCplx ? HSMA_CPLX_G1_MMAX : 64, MAP>(sTri, sC, B, ldb, m, n, tile0, step, rev);
        return;
      }
    }
    if constexpr ((kBatchedGMask & 2u) != 0) {
      if (g == 2) {
        solve_tiles<T, 2, 64, MAP>(sTri, sC, B, ldb, m, n, tile0, step, rev);
        return;
      }
    }
    if constexpr ((kBatchedGMask & 4u) != 0) {
      if (g == 4) {
        solve_tiles<T, 4, 64, MAP>(sTri, sC, B, ldb, m, n, tile0, step, rev);
        return;
      }
    }
    if constexpr ((kBatchedGMask & 8u) != 0) {
      if (g == 8) {
        solve_tiles<T, 8, 64, MAP>(sTri, sC, B, ldb, m, n, tile0, step, rev);
        return;
      }
    }
  }
};

// The triangle's packed layout uses MMAX = 64 for every variant except the
// complex G = 1 one (MMAX = 32); stage with the variant's MMAX.
template <class T>
__device__ __forceinline__ int variant_mmax(int g) {
  return (Elem<T>::kComplex && g == 1) ? HSMA_CPLX_G1_MMAX : 64;
}

template <class T, int W, bool MAP>
__device__ __forceinline__ void stage_any(int g, T *sTri, T *sC, T *sR, const T *A, int64_t lda, int m, T alpha,
                                          bool unit, SmallMap mp) {
  const int rows_used = ((m + g - 1) / g) * g;
  if (variant_mmax<T>(g) == 32)
    stage<T, 32, W, MAP>(sTri, sC, sR, A, lda, m, rows_used, alpha, unit, mp);
  else
    stage<T, 64, W, MAP>(sTri, sC, sR, A, lda, m, rows_used, alpha, unit, mp);
}

template <class T>
__device__ __forceinline__ void smem_parts(unsigned char *smem, T *&sTri, T *&sC, T *&sR) {
  sTri = reinterpret_cast<T *>(smem);
  sC = sTri + tri_elems(64);
  sR = sC + 64;
}

// ---------------------------------------------------------------------------
// Single solve: CTA k stages the instance and its warps take column tiles
// k*W, k*W+1, ... (W warps per CTA).  MAP = false is the paper's case (no
// index remapping); FULL = true the m = MMAX case (no bound checks).
// ---------------------------------------------------------------------------
template <class T, int G, int MMAX, bool MAP, bool FULL>
__global__ void __launch_bounds__(32 * kWarpsSingle) small_single_kernel(const T *__restrict__ A, int64_t lda, T *B,
                                                                 int64_t ldb, int m_, int n, T alpha, int unit,
                                                                 SmallMap mp) {
  extern __shared__ __align__(16) unsigned char smem[];
  T *sTri, *sC, *sR;
  smem_parts<T>(smem, sTri, sC, sR);
  const int m = FULL ? MMAX : m_;
  if constexpr (FULL && !MAP) {
    // the warp's first column tile is loaded before staging, so its latency
    // overlaps the staging (a one-pass staging with every triangle load in
    // flight at once measured slower than this with warm caches: the kernel is
    // bound by dependent FP64 work on one warp per sub-partition, not by memory)
    constexpr int C = 32 / G;
    const int ntiles = (n + C - 1) / C;
    const int step = gridDim.x * kWarpsSingle;
    const int t0 = blockIdx.x * kWarpsSingle + (threadIdx.x >> 5);
    auto cols = [&](int t) { return (n - t * C) < C ? (n - t * C) : C; };
    T b[MMAX / G];
    if (t0 < ntiles) warp_load_b<T, G, MMAX, false, true>(b, B + (int64_t)t0 * C * ldb, ldb, m, cols(t0), 0);
    stage<T, MMAX, kWarpsSingle, false>(sTri, sC, sR, A, lda, m, MMAX, alpha, unit != 0, mp);
    for (int t = t0; t < ntiles; t += step) {
      T *Bt = B + (int64_t)t * C * ldb;
      if (t != t0) warp_load_b<T, G, MMAX, false, true>(b, Bt, ldb, m, cols(t), 0);
      warp_solve_loaded<T, G, MMAX, false, true>(b, sTri, sC, Bt, ldb, m, cols(t), 0);
    }
  } else {
    const int rows_used = ((m + G - 1) / G) * G;
    stage<T, MMAX, kWarpsSingle, MAP>(sTri, sC, sR, A, lda, m, rows_used, alpha, unit != 0, mp);
    solve_tiles<T, G, MMAX, MAP, FULL>(sTri, sC, B, ldb, m, n, blockIdx.x * kWarpsSingle,
                                       gridDim.x * kWarpsSingle, mp.rev);
  }
}

// ---------------------------------------------------------------------------
// Varlen batch.  A one-CTA pre-pass validates the instances, picks G per
// instance and writes a longest-first schedule (bucketed by estimated cost);
// the persistent kernel then pulls instances from an atomic counter.
//
// Scratch layout (int32): [0] next-item counter, [1] number of scheduled
// items, [2 .. 2+batch) schedule entries (instance | G << 24).
// ---------------------------------------------------------------------------
constexpr int kBuckets = 256;

__host__ __device__ inline int cost_bucket(long long cost) {
  // 8 buckets per octave: the octave and the three bits below the leading one
  if (cost < 16) return 0;
#ifdef __CUDA_ARCH__
  const int lead = 63 - __clzll(cost);
#else
  int lead = 0;
  while ((cost >> (lead + 1)) != 0) ++lead;
#endif
  const int b = lead * 8 + (int)((cost >> (lead - 3)) & 7);
  return b < kBuckets ? b : kBuckets - 1;
}

// The schedule entry of every (m, n) with m, n <= 64, real and complex:
// G | bucket << 8.  Computed on the host from the same closed-form cost model
// and copied to the device once per device, so the schedule pass does one
// lookup per instance instead of evaluating the model (64-bit divisions).
__device__ int32_t g_sched_tab[2 * 64 * 64];

int32_t sched_entry(int m, int n, bool cplx_) {
  const int g = hsma_small_pick_g_batched(m, n, cplx_, kWarpsBatched, kBatchedGMask);
  return g | (cost_bucket(hsma_small_cta_instr(m, n, g, cplx_, kWarpsBatched)) << 8);
}

// Device address of the table, filled on first use on this device; null when
// it is not yet filled and the stream is capturing (the pass then evaluates
// the model itself).
const int32_t *sched_table(cudaStream_t st) {
  static const int32_t *addr[64] = {nullptr};
  static std::mutex mu;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  if (addr[dev] != nullptr) return addr[dev];
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return nullptr;
  static int32_t host[2 * 64 * 64];
  static bool host_ready = false;
  if (!host_ready) {
    for (int c = 0; c < 2; ++c)
      for (int m = 1; m <= 64; ++m)
        for (int n = 1; n <= 64; ++n) host[c * 4096 + (m - 1) * 64 + (n - 1)] = sched_entry(m, n, c == 1);
    host_ready = true;
  }
  void *p = nullptr;
  if (cudaGetSymbolAddress(&p, g_sched_tab) != cudaSuccess) return nullptr;
  if (cudaMemcpy(p, host, sizeof host, cudaMemcpyHostToDevice) != cudaSuccess) return nullptr;
  addr[dev] = static_cast<const int32_t *>(p);
  return addr[dev];
}

template <class T>
__global__ void __launch_bounds__(1024) vbatched_schedule_kernel(int batch, const int32_t *__restrict__ dm,
                                                                 const int32_t *__restrict__ dn,
                                                                 const int32_t *__restrict__ dlda,
                                                                 const int32_t *__restrict__ dldb,
                                                                 const void *const *__restrict__ dA,
                                                                 void *const *__restrict__ dB, int32_t *scratch,
                                                                 uint32_t *status, const int32_t *__restrict__ tab,
                                                                 int skip_large) {
  __shared__ int hist[kBuckets];
  __shared__ int offs[kBuckets];
  const bool cplx_ = Elem<T>::kComplex;
  for (int k = threadIdx.x; k < kBuckets; k += blockDim.x) hist[k] = 0;
  __syncthreads();
  uint32_t err = 0;
  for (int b = threadIdx.x; b < batch; b += blockDim.x) {
    const int m = dm[b], n = dn[b];
    const int lo = m > 1 ? m : 1;
    if (skip_large && m > 64) continue;  // solved by the caller on the blocked path
    if (m < 0 || n < 0 || m > 64 || dlda[b] < lo || dldb[b] < lo) {
      err |= HSMA_DEVERR_BAD_SIZE;
      continue;
    }
    if (m == 0 || n == 0) continue;
    if (dA[b] == nullptr || dB[b] == nullptr) {
      err |= HSMA_DEVERR_NULL_PTR;
      continue;
    }
    int e;
    if (tab != nullptr && n <= 64) {
      e = tab[(cplx_ ? 4096 : 0) + (m - 1) * 64 + (n - 1)];
    } else {
      const int g = hsma_small_pick_g_batched(m, n, cplx_, kWarpsBatched, kBatchedGMask);
      e = g | (cost_bucket(hsma_small_cta_instr(m, n, g, cplx_, kWarpsBatched)) << 8);
    }
    atomicAdd(&hist[e >> 8], 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = 0;
    for (int k = kBuckets - 1; k >= 0; --k) {  // most expensive first
      offs[k] = run;
      run += hist[k];
    }
    scratch[0] = 0;
    scratch[1] = run;
  }
  __syncthreads();
  for (int b = threadIdx.x; b < batch; b += blockDim.x) {
    const int m = dm[b], n = dn[b];
    const int lo = m > 1 ? m : 1;
    if (m <= 0 || n <= 0 || m > 64 || dlda[b] < lo || dldb[b] < lo) continue;
    if (dA[b] == nullptr || dB[b] == nullptr) continue;
    int e;
    if (tab != nullptr && n <= 64) {
      e = tab[(cplx_ ? 4096 : 0) + (m - 1) * 64 + (n - 1)];
    } else {
      const int g = hsma_small_pick_g_batched(m, n, cplx_, kWarpsBatched, kBatchedGMask);
      e = g | (cost_bucket(hsma_small_cta_instr(m, n, g, cplx_, kWarpsBatched)) << 8);
    }
    const int pos = atomicAdd(&offs[e >> 8], 1);
    scratch[2 + pos] = b | ((e & 0xff) << 24);
  }
  if (err != 0 && status != nullptr) atomicOr(status, err);
}

template <class T, bool MAP>
__global__ void __launch_bounds__(32 * kWarpsBatched,
                                  (sizeof(T) == sizeof(float) || sizeof(T) == sizeof(cplxf)) && !std::is_same<T, double>::value
                                      ? HSMA_VB_MINB_F32
                                      : HSMA_VB_MINB) vbatched_solve_kernel(const int32_t *__restrict__ dm,
                                                                  const int32_t *__restrict__ dn,
                                                                  const int32_t *__restrict__ dlda,
                                                                  const int32_t *__restrict__ dldb,
                                                                  const void *const *__restrict__ dA,
                                                                  void *const *__restrict__ dB, T alpha, int unit,
                                                                  int32_t *scratch, SmallMap mp) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_item;
  T *sTri, *sC, *sR;
  smem_parts<T>(smem, sTri, sC, sR);
  const int nitems = *(volatile int32_t *)(scratch + 1);
  const bool azero = Elem<T>::is_zero(alpha);
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(scratch, 1);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= nitems) break;
    const int e = scratch[2 + item];
    const int b = e & 0xffffff, g = e >> 24;
    const int m = dm[b], n = dn[b];
    const T *A = static_cast<const T *>(dA[b]);
    T *B = static_cast<T *>(dB[b]);
    const int64_t lda = dlda[b], ldb = dldb[b];
    if (azero) {
      zero_tiles<T, kWarpsBatched>(B, ldb, m, n);
      continue;
    }
    stage_any<T, kWarpsBatched, MAP>(g, sTri, sC, sR, A, lda, m, alpha, unit != 0, mp);
    Variants<T, MAP>::run(g, sTri, sC, B, ldb, m, n, 0, kWarpsBatched, mp.rev);
    __syncthreads();  // the next item restages shared memory
  }
}

// ---------------------------------------------------------------------------
// Varlen batch of factor solves in one launch: the small solve fused with
// its consumer.  LU factors: per instance the CTA applies the row
// interchanges to B, stages the unit-lower factor and solves, then stages the
// upper factor in row-reversed form (the left / upper index map) and solves
// again on the intermediate result, which the same CTA has just written
// (cache resident).  Cholesky factors (A = L L^H): the lower factor, then its
// conjugate transpose through the reversed, transposed, conjugated map.
// ---------------------------------------------------------------------------

// Row interchanges k <-> ipiv[k]-1, k = 0..m-1 in order, applied to B as one
// gather (row r takes the old row perm[r]).  False, with B untouched, when a
// pivot lies outside [k, m).  All threads of the CTA take part.
template <class T>
__device__ __forceinline__ bool lu_permute_rows(T *B, int64_t ldb, int m, int n, const int32_t *__restrict__ ipiv,
                                                int *sPiv, int *sPerm, int *sBad) {
  using E = Elem<T>;
  for (int k = threadIdx.x; k < m; k += blockDim.x) sPiv[k] = ipiv[k] - 1;
  __syncthreads();
  if (threadIdx.x == 0) {
    int bad = 0;
    for (int r = 0; r < m; ++r) sPerm[r] = r;
    for (int k = 0; k < m && !bad; ++k) {
      const int p = sPiv[k];
      if (p < k || p >= m) {
        bad = 1;
      } else {
        const int t = sPerm[k];
        sPerm[k] = sPerm[p];
        sPerm[p] = t;
      }
    }
    *sBad = bad;
  }
  __syncthreads();
  if (*sBad) return false;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p0 = lane < m ? sPerm[lane] : 0, p1 = lane + 32 < m ? sPerm[lane + 32] : 0;
  for (int j = warp; j < n; j += kWarpsBatched) {  // warp-uniform: every lane shuffles
    T *col = B + (int64_t)j * ldb;
    const T v0 = lane < m ? E::ld(col + lane) : E::zero();
    const T v1 = lane + 32 < m ? E::ld(col + lane + 32) : E::zero();
    const T a0 = E::shfl(v0, p0 & 31), b0 = E::shfl(v1, p0 & 31);
    const T a1 = E::shfl(v0, p1 & 31), b1 = E::shfl(v1, p1 & 31);
    if (lane < m) E::st(col + lane, p0 < 32 ? a0 : b0);
    if (lane + 32 < m) E::st(col + lane + 32, p1 < 32 ? a1 : b1);
  }
  __syncthreads();
  return true;
}

// One triangular solve of the pair: stage (with the map) and solve every
// column tile.  Kept out of line so the compiler handles each of the two
// solves once, not the fused kernel as one body.
template <class T, bool MAP>
__device__ __noinline__ void lu_stage_solve(int g, T *sTri, T *sC, T *sR, const T *A, int64_t lda, T *B,
                                            int64_t ldb, int m, int n, T alpha, bool unit, SmallMap mp) {
  stage_any<T, kWarpsBatched, MAP>(g, sTri, sC, sR, A, lda, m, alpha, unit, mp);
  Variants<T, MAP>::run(g, sTri, sC, B, ldb, m, n, 0, kWarpsBatched, mp.rev);
}

template <class T>
__global__ void __launch_bounds__(32 * kWarpsBatched,
                                  (sizeof(T) == sizeof(float) || sizeof(T) == sizeof(cplxf)) && !std::is_same<T, double>::value
                                      ? HSMA_VB_MINB_F32
                                      : HSMA_VB_MINB) vbatched_lu_kernel(const int32_t *__restrict__ dm,
                                                                  const int32_t *__restrict__ dn,
                                                                  const int32_t *__restrict__ dlda,
                                                                  const int32_t *__restrict__ dldb,
                                                                  const void *const *__restrict__ dA,
                                                                  const int32_t *const *__restrict__ dipiv,
                                                                  void *const *__restrict__ dB, T alpha,
                                                                  int32_t *scratch, uint32_t *status, int chol) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_item, s_bad;
  __shared__ int s_piv[64], s_perm[64];
  T *sTri, *sC, *sR;
  smem_parts<T>(smem, sTri, sC, sR);
  const int nitems = *(volatile int32_t *)(scratch + 1);
  const bool azero = Elem<T>::is_zero(alpha);
  // second factor: U (upper), or L^H (lower read transposed and conjugated)
  const SmallMap lower{0, 0, 0}, second{1, chol, chol};
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(scratch, 1);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= nitems) break;
    const int e = scratch[2 + item];
    const int b = e & 0xffffff, g = e >> 24;
    const int m = dm[b], n = dn[b];
    const T *A = static_cast<const T *>(dA[b]);
    T *B = static_cast<T *>(dB[b]);
    const int64_t lda = dlda[b], ldb = dldb[b];
    const int32_t *ipiv = dipiv != nullptr ? dipiv[b] : nullptr;
    if (ipiv != nullptr && !lu_permute_rows<T>(B, ldb, m, n, ipiv, s_piv, s_perm, &s_bad)) {
      if (threadIdx.x == 0 && status != nullptr) atomicOr(status, HSMA_DEVERR_BAD_PIVOT);
      continue;
    }
    if (azero) {
      zero_tiles<T, kWarpsBatched>(B, ldb, m, n);
      continue;
    }
    // L Y = alpha P^T B (LU: unit diagonal, not read)
    lu_stage_solve<T, false>(g, sTri, sC, sR, A, lda, B, ldb, m, n, alpha, chol == 0, lower);
    __syncthreads();
    // U X = Y, or L^H X = Y
    lu_stage_solve<T, true>(g, sTri, sC, sR, A, lda, B, ldb, m, n, Elem<T>::one(), false, second);
    __syncthreads();  // the next item restages shared memory
  }
}

template <class T>
int lu_grid(int dev) {
  static int cached[64] = {0};
  if (dev >= 0 && dev < 64 && cached[dev] > 0) return cached[dev];
  int nsm = 0, per_sm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, vbatched_lu_kernel<T>, 32 * kWarpsBatched,
                                                SmemLayout<T>::bytes(64));
  int grid = nsm * (per_sm > 0 ? per_sm : 1);
  if (dev >= 0 && dev < 64) cached[dev] = grid;
  return grid;
}

template <class T, bool MAP>
int persistent_grid(int dev) {
  static int cached[64] = {0};
  if (dev >= 0 && dev < 64 && cached[dev] > 0) return cached[dev];
  int nsm = 0, per_sm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, vbatched_solve_kernel<T, MAP>, 32 * kWarpsBatched,
                                                SmemLayout<T>::bytes(64));
  int grid = nsm * (per_sm > 0 ? per_sm : 1);
  if (dev >= 0 && dev < 64) cached[dev] = grid;
  return grid;
}

template <class T>
hsma_status_t set_smem_attrs() {
  const int bytes = (int)SmemLayout<T>::bytes(64);
  HSMA_CUDA_TRY(
      cudaFuncSetAttribute(vbatched_solve_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  HSMA_CUDA_TRY(
      cudaFuncSetAttribute(vbatched_solve_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  return HSMA_OK;
}

template <class T, int G, int MMAX, bool MAP, bool FULL>
hsma_status_t launch_single_v(const T *A, int64_t lda, T *B, int64_t ldb, int m, int n, T alpha, int unit,
                              int grid, cudaStream_t st, SmallMap mp) {
  const size_t bytes = SmemLayout<T>::bytes(64);
  static DeviceFlags attr_done;
  if (!attr_done.test()) {
    HSMA_CUDA_TRY(cudaFuncSetAttribute(small_single_kernel<T, G, MMAX, MAP, FULL>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    attr_done.set();
  }
  HsmaTraceScope ts("small_single", st);
  small_single_kernel<T, G, MMAX, MAP, FULL><<<grid, 32 * kWarpsSingle, bytes, st>>>(A, lda, B, ldb, m, n, alpha,
                                                                                       unit, mp);
  HSMA_CUDA_TRY(cudaGetLastError());
  return HSMA_OK;
}

template <class T, int G, int MMAX>
hsma_status_t launch_single_g(const T *A, int64_t lda, T *B, int64_t ldb, int m, int n, T alpha, int unit,
                              int nsm, cudaStream_t st, SmallMap mp) {
  constexpr int C = 32 / G;
  const int tiles = (n + C - 1) / C;
  int grid = (tiles + kWarpsSingle - 1) / kWarpsSingle;
  const int cap = nsm * 16;
  if (grid > cap) grid = cap;
  const bool mapped = mp.rev != 0 || mp.tr != 0 || mp.cj != 0;
  if (mapped) return launch_single_v<T, G, MMAX, true, false>(A, lda, B, ldb, m, n, alpha, unit, grid, st, mp);
  if constexpr (G == 32 && MMAX == 64) {
    if (m == MMAX) return launch_single_v<T, G, MMAX, false, true>(A, lda, B, ldb, m, n, alpha, unit, grid, st, mp);
  }
  return launch_single_v<T, G, MMAX, false, false>(A, lda, B, ldb, m, n, alpha, unit, grid, st, mp);
}

}  // namespace

// ---------------------------------------------------------------------------
// Host entry points (internal; the C ABI validates arguments first).
// ---------------------------------------------------------------------------
static SmallMap make_map(int uplo, int trans) {
  const bool op_lower = (uplo == HSMA_LOWER) != (trans != HSMA_NO_TRANS);
  return SmallMap{op_lower ? 0 : 1, trans != HSMA_NO_TRANS ? 1 : 0, trans == HSMA_CONJ_TRANS ? 1 : 0};
}

template <class T>
static hsma_status_t small_single_impl(int g, const void *A, int64_t lda, void *B, int64_t ldb, int m, int n,
                                       const double *alpha, int unit, cudaStream_t st, SmallMap mp) {
  int dev = 0, nsm = 0;
  HSMA_CUDA_TRY(cudaGetDevice(&dev));
  HSMA_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const bool cplx_ = Elem<T>::kComplex;
  if (g == 0) g = hsma_small_pick_g_single(m, n, cplx_, nsm);
  if (!hsma_small_g_ok(g, m, cplx_)) return HSMA_ERR_INVALID_ARG;
  const T al = hsma_alpha_as<T>(alpha);
  const T *a = static_cast<const T *>(A);
  T *b = static_cast<T *>(B);
  if constexpr (Elem<T>::kComplex) {
    switch (g) {
      case 1: return launch_single_g<T, 1, 32>(a, lda, b, ldb, m, n, al, unit, nsm, st, mp);
      case 2: return launch_single_g<T, 2, 64>(a, lda, b, ldb, m, n, al, unit, nsm, st, mp);
      case 4: return launch_single_g<T, 4, 64>(a, lda, b, ldb, m, n, al, unit, nsm, st, mp);
      case 8: return launch_single_g<T, 8, 64>(a, lda, b, ldb, m, n, al, unit, nsm, st, mp);
      case 16: return launch_single_g<T, 16, 64>(a, lda, b, ldb, m, n, al, unit, nsm, st, mp);
      case 32: return launch_single_g<T, 32, 64>(a, lda, b, ldb, m, n, al, unit, nsm, st, mp);
      default: return HSMA_ERR_INVALID_ARG;
    }
  } else {
    switch (g) {
      case 1: return launch_single_g<T, 1, 64>(a, lda, b, ldb, m, n, al, unit, nsm, st, mp);
      case 2: return launch_single_g<T, 2, 64>(a, lda, b, ldb, m, n, al, unit, nsm, st, mp);
      case 4: return launch_single_g<T, 4, 64>(a, lda, b, ldb, m, n, al, unit, nsm, st, mp);
      case 8: return launch_single_g<T, 8, 64>(a, lda, b, ldb, m, n, al, unit, nsm, st, mp);
      case 16: return launch_single_g<T, 16, 64>(a, lda, b, ldb, m, n, al, unit, nsm, st, mp);
      case 32: return launch_single_g<T, 32, 64>(a, lda, b, ldb, m, n, al, unit, nsm, st, mp);
      default: return HSMA_ERR_INVALID_ARG;
    }
  }
}

hsma_status_t hsma_small_single(int dtype, int g, const void *A, int64_t lda, void *B, int64_t ldb, int m, int n,
                                const double *alpha, int unit, cudaStream_t st, int uplo, int trans) {
  const SmallMap mp = make_map(uplo, trans);
  switch (dtype) {
    case HSMA_C128: return small_single_impl<cplx>(g, A, lda, B, ldb, m, n, alpha, unit, st, mp);
    case HSMA_R32: return small_single_impl<float>(g, A, lda, B, ldb, m, n, alpha, unit, st, mp);
    case HSMA_C64: return small_single_impl<cplxf>(g, A, lda, B, ldb, m, n, alpha, unit, st, mp);
    default: return small_single_impl<double>(g, A, lda, B, ldb, m, n, alpha, unit, st, mp);
  }
}

template <class T>
static hsma_status_t vbatched_impl(int32_t batch, const int32_t *dm, const int32_t *dn, const double *alpha,
                                   const void *const *dA, const int32_t *dlda, void *const *dB,
                                   const int32_t *dldb, int unit, uint32_t *status, int32_t *scratch,
                                   cudaStream_t st, SmallMap mp, int skip_large) {
  int dev = 0;
  HSMA_CUDA_TRY(cudaGetDevice(&dev));
  static DeviceFlags attr_done;
  if (!attr_done.test()) {
    hsma_status_t s = set_smem_attrs<T>();
    if (s != HSMA_OK) return s;
    attr_done.set();
  }
  const T al = hsma_alpha_as<T>(alpha);
  {
    HsmaTraceScope ts("vbatched_schedule", st);
    vbatched_schedule_kernel<T><<<1, 1024, 0, st>>>(batch, dm, dn, dlda, dldb, dA, dB, scratch, status,
                                                    sched_table(st), skip_large);
  }
  HSMA_CUDA_TRY(cudaGetLastError());
  // the identity map (the paper's case) runs a kernel without the remapping arithmetic
  const bool mapped = mp.rev != 0 || mp.tr != 0 || mp.cj != 0;
  int grid = mapped ? persistent_grid<T, true>(dev) : persistent_grid<T, false>(dev);
  if (grid > batch) grid = batch;
  {
    HsmaTraceScope ts("vbatched_solve", st);
    if (mapped)
      vbatched_solve_kernel<T, true><<<grid, 32 * kWarpsBatched, SmemLayout<T>::bytes(64), st>>>(
          dm, dn, dlda, dldb, dA, dB, al, unit, scratch, mp);
    else
      vbatched_solve_kernel<T, false><<<grid, 32 * kWarpsBatched, SmemLayout<T>::bytes(64), st>>>(
          dm, dn, dlda, dldb, dA, dB, al, unit, scratch, mp);
  }
  HSMA_CUDA_TRY(cudaGetLastError());
  return HSMA_OK;
}

size_t hsma_vbatched_scratch_bytes(int32_t batch) { return sizeof(int32_t) * (2 + (size_t)(batch > 0 ? batch : 0)); }

hsma_status_t hsma_small_vbatched(int dtype, int32_t batch, const int32_t *dm, const int32_t *dn,
                                  const double *alpha, const void *const *dA, const int32_t *dlda,
                                  void *const *dB, const int32_t *dldb, int unit, uint32_t *status,
                                  int32_t *scratch, cudaStream_t st, int uplo, int trans, int skip_large) {
  const SmallMap mp = make_map(uplo, trans);
  switch (dtype) {
    case HSMA_C128: return vbatched_impl<cplx>(batch, dm, dn, alpha, dA, dlda, dB, dldb, unit, status, scratch, st, mp,
                                    skip_large);
    case HSMA_R32: return vbatched_impl<float>(batch, dm, dn, alpha, dA, dlda, dB, dldb, unit, status, scratch, st, mp,
                                    skip_large);
    case HSMA_C64: return vbatched_impl<cplxf>(batch, dm, dn, alpha, dA, dlda, dB, dldb, unit, status, scratch, st, mp,
                                    skip_large);
    default: return vbatched_impl<double>(batch, dm, dn, alpha, dA, dlda, dB, dldb, unit, status, scratch, st, mp,
                                    skip_large);
  }
}

template <class T>
static hsma_status_t getrs_impl(int32_t batch, const int32_t *dm, const int32_t *dn, const double *alpha,
                                const void *const *dLU, const int32_t *dlda, const int32_t *const *dipiv,
                                void *const *dB, const int32_t *dldb, uint32_t *status, int32_t *scratch,
                                cudaStream_t st, int chol, int skip_large) {
  int dev = 0;
  HSMA_CUDA_TRY(cudaGetDevice(&dev));
  static DeviceFlags attr_done;
  if (!attr_done.test()) {
    HSMA_CUDA_TRY(cudaFuncSetAttribute(vbatched_lu_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)SmemLayout<T>::bytes(64)));
    attr_done.set();
  }
  const T al = hsma_alpha_as<T>(alpha);
  {
    HsmaTraceScope ts("vbatched_schedule", st);
    vbatched_schedule_kernel<T><<<1, 1024, 0, st>>>(batch, dm, dn, dlda, dldb, dLU, dB, scratch, status,
                                                    sched_table(st), skip_large);
  }
  HSMA_CUDA_TRY(cudaGetLastError());
  int grid = lu_grid<T>(dev);
  if (grid > batch) grid = batch;
  {
    HsmaTraceScope ts("vbatched_lu", st);
    vbatched_lu_kernel<T><<<grid, 32 * kWarpsBatched, SmemLayout<T>::bytes(64), st>>>(dm, dn, dlda, dldb, dLU,
                                                                                       dipiv, dB, al, scratch,
                                                                                       status, chol);
  }
  HSMA_CUDA_TRY(cudaGetLastError());
  return HSMA_OK;
}

namespace {

// Row interchanges of a batch of LU-factor solves ahead of their two
// triangular solves (one warp per instance): P^T B by LAPACK's ipiv (row k
// swapped with row ipiv[k] - 1, k = 0, 1, ... in order), and the instance's
// size for the solves in m_eff: its m, or 0 when a pivot is out of range
// (HSMA_DEVERR_BAD_PIVOT; B untouched and both solves skip the instance).
// The swaps are composed into one permutation first (row r of P^T B is row
// perm[r] of B), so each column is one gather: loads of the column's rows,
// then stores, four columns in flight per step.
// Instances the solves reject (sizes, pointers) or leave to the blocked path
// (m > 64) are not permuted here.
template <class T>
__global__ void __launch_bounds__(256) lu_pivots_kernel(int32_t batch, const int32_t *__restrict__ dm,
                                                        const int32_t *__restrict__ dn,
                                                        const int32_t *__restrict__ dlda,
                                                        const int32_t *__restrict__ dldb,
                                                        const void *const *__restrict__ dA, void *const *dB,
                                                        const int32_t *const *__restrict__ dipiv, int32_t *m_eff,
                                                        uint32_t *status) {
  constexpr int kCols = 4;
  __shared__ int s_perm[8][64];
  const int lane = threadIdx.x & 31;
  int *perm = s_perm[threadIdx.x >> 5];
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < batch; b += nw) {
    const int m = dm[b], n = dn[b];
    if (lane == 0) m_eff[b] = m;
    const int32_t *ipiv = dipiv != nullptr ? dipiv[b] : nullptr;
    if (ipiv == nullptr || m <= 0 || n <= 0 || m > 64 || dlda[b] < m || dldb[b] < m || dA[b] == nullptr ||
        dB[b] == nullptr)
      continue;
    bool bad = false;
    for (int k = lane; k < m; k += 32) bad |= ipiv[k] <= k || ipiv[k] > m;  // LAPACK: ipiv[k] in [k+1, m]
    if (__any_sync(0xffffffffu, bad)) {
      if (lane == 0) {
        m_eff[b] = 0;
        if (status != nullptr) atomicOr(status, HSMA_DEVERR_BAD_PIVOT);
      }
      continue;
    }
    for (int r = lane; r < m; r += 32) perm[r] = r;
    __syncwarp();
    if (lane == 0) {
      for (int k = 0; k < m; ++k) {
        const int p = ipiv[k] - 1;
        const int t = perm[k];
        perm[k] = perm[p];
        perm[p] = t;
      }
    }
    __syncwarp();
    const int r0 = lane, r1 = lane + 32;
    const int q0 = r0 < m ? perm[r0] : 0, q1 = r1 < m ? perm[r1] : 0;
    __syncwarp();  // perm is rewritten by this warp's next instance
    T *B = static_cast<T *>(dB[b]);
    const int64_t ldb = dldb[b];
    for (int j0 = 0; j0 < n; j0 += kCols) {
      T v0[kCols], v1[kCols];
#pragma unroll
      for (int u = 0; u < kCols; ++u) {
        const T *col = B + (int64_t)(j0 + u) * ldb;
        if (j0 + u < n && r0 < m) v0[u] = col[q0];
        if (j0 + u < n && r1 < m) v1[u] = col[q1];
      }
      __syncwarp();  // every lane's loads of these columns before any store
#pragma unroll
      for (int u = 0; u < kCols; ++u) {
        T *col = B + (int64_t)(j0 + u) * ldb;
        if (j0 + u < n && r0 < m) col[r0] = v0[u];
        if (j0 + u < n && r1 < m) col[r1] = v1[u];
      }
      __syncwarp();
    }
  }
}

}  // namespace

hsma_status_t hsma_small_lu_pivots(int dtype, int32_t batch, const int32_t *dm, const int32_t *dn,
                                   const int32_t *dlda, const int32_t *dldb, const void *const *dA,
                                   void *const *dB, const int32_t *const *dipiv, int32_t *m_eff, uint32_t *status,
                                   cudaStream_t st) {
  if (batch <= 0) return HSMA_OK;
  int dev = 0, nsm = 0;
  HSMA_CUDA_TRY(cudaGetDevice(&dev));
  HSMA_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int grid = (int)std::min<int64_t>(((int64_t)batch + 7) / 8, 4 * (int64_t)nsm);
  HsmaTraceScope ts("vbatched_schedule", st);
  if (dtype == HSMA_C128)
    lu_pivots_kernel<cplx><<<grid, 256, 0, st>>>(batch, dm, dn, dlda, dldb, dA, dB, dipiv, m_eff, status);
  else if (dtype == HSMA_C64)
    lu_pivots_kernel<cplxf><<<grid, 256, 0, st>>>(batch, dm, dn, dlda, dldb, dA, dB, dipiv, m_eff, status);
  else if (dtype == HSMA_R32)
    lu_pivots_kernel<float><<<grid, 256, 0, st>>>(batch, dm, dn, dlda, dldb, dA, dB, dipiv, m_eff, status);
  else
    lu_pivots_kernel<double><<<grid, 256, 0, st>>>(batch, dm, dn, dlda, dldb, dA, dB, dipiv, m_eff, status);
  return hsma_from_cuda(cudaGetLastError());
}

hsma_status_t hsma_small_getrs_vbatched(int dtype, int32_t batch, const int32_t *dm, const int32_t *dn,
                                        const double *alpha, const void *const *dLU, const int32_t *dlda,
                                        const int32_t *const *dipiv, void *const *dB, const int32_t *dldb,
                                        uint32_t *status, int32_t *scratch, cudaStream_t st, int chol,
                                        int skip_large) {
  if (chol) dipiv = nullptr;
  switch (dtype) {
    case HSMA_C128:
      return getrs_impl<cplx>(batch, dm, dn, alpha, dLU, dlda, dipiv, dB, dldb, status, scratch, st, chol,
                                 skip_large);
    case HSMA_R32:
      return getrs_impl<float>(batch, dm, dn, alpha, dLU, dlda, dipiv, dB, dldb, status, scratch, st, chol,
                                 skip_large);
    case HSMA_C64:
      return getrs_impl<cplxf>(batch, dm, dn, alpha, dLU, dlda, dipiv, dB, dldb, status, scratch, st, chol,
                                 skip_large);
    default:
      return getrs_impl<double>(batch, dm, dn, alpha, dLU, dlda, dipiv, dB, dldb, status, scratch, st, chol,
                                 skip_large);
  }
}

// ---------------------------------------------------------------------------
// Allocation-free varlen batch.  The schedule scratch (next-item counter,
// item count and the per-instance schedule) lives in this file-scope device
// array instead of the stream-ordered pool.  Every GPU that loads the library
// keeps the array until the process exits.  Host code never hands the array's
// name to a kernel: it first looks up the array's device address, once per
// device, with that device current.
// ---------------------------------------------------------------------------
namespace {

constexpr int32_t kNoAllocMaxBatch = 65536;
__device__ __align__(256) int32_t g_noalloc_scratch[2 + kNoAllocMaxBatch];

int32_t *noalloc_scratch(cudaError_t *err) {
  static int32_t *addr[64] = {nullptr};
  static std::mutex mu;
  int dev = 0;
  *err = cudaGetDevice(&dev);
  if (*err != cudaSuccess) return nullptr;
  if (dev < 0 || dev >= 64) {
    *err = cudaErrorInvalidDevice;
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(mu);
  if (addr[dev] == nullptr) {
    int32_t *p = nullptr;
    *err = cudaGetSymbolAddress(reinterpret_cast<void **>(&p), g_noalloc_scratch);
    if (*err != cudaSuccess) return nullptr;
    addr[dev] = p;
  }
  return addr[dev];
}

}  // namespace

extern "C" HSMA_API hsma_status_t hsma_trsm_llnn_vbatched_noalloc(int dtype, int diag, int32_t batch,
                                                                  const int32_t *d_m, const int32_t *d_n,
                                                                  const void *alpha, const void *const *d_A,
                                                                  const int32_t *d_lda, void *const *d_B,
                                                                  const int32_t *d_ldb, int32_t max_m,
                                                                  int32_t max_n, uint32_t *d_status,
                                                                  void *stream) {
  if (!hsma_small_dtype(dtype)) {
    return (dtype == HSMA_R32_BF16 || dtype == HSMA_R64_IR) ? HSMA_ERR_UNSUPPORTED : HSMA_ERR_INVALID_ARG;
  }
  if ((diag != HSMA_NON_UNIT && diag != HSMA_UNIT) || batch < 0 || max_m < 0 || max_n < 0)
    return HSMA_ERR_INVALID_ARG;
  if (max_m > 64 || batch > kNoAllocMaxBatch) return HSMA_ERR_UNSUPPORTED;
  if (batch == 0) return HSMA_OK;
  if (alpha == nullptr || d_m == nullptr || d_n == nullptr || d_A == nullptr || d_lda == nullptr ||
      d_B == nullptr || d_ldb == nullptr)
    return HSMA_ERR_INVALID_ARG;
  cudaError_t e = cudaSuccess;
  int32_t *scratch = noalloc_scratch(&e);
  if (scratch == nullptr) return hsma_from_cuda(e);
  // the schedule pre-pass rewrites the counter and the item count on every call
  return hsma_small_vbatched(dtype, batch, d_m, d_n, static_cast<const double *>(alpha), d_A, d_lda, d_B, d_ldb,
                             diag == HSMA_UNIT, d_status, scratch, static_cast<cudaStream_t>(stream));
}
