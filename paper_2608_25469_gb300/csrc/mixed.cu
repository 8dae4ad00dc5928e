// Reduced-precision modes of the blocked solve (the paper lists mixed
// precision as future work, Section 6; the blocked algorithm is Section 4.3).
//
// FP32-result mode (HSMA_R32_BF16): phase 1 inverts the diagonal blocks in
// FP32; phase 2 forms X_r = D_r^{-1} B_r with FP32 FMAs and applies the
// trailing update B_{r+1:} -= A_{r+1:,r} X_r on the 5th-generation tensor
// cores: operands in BF16, products accumulated in FP32 in tensor memory
// (tcgen05.mma kind::f16, cta_group::1, 128 x 256 tiles, TMA loads with
// 128-byte swizzle).  With three terms per update the operands are split,
// a = hi(a) + lo(a), and the products hi*hi + hi*lo + lo*hi are accumulated in
// one pass by concatenating along K: [A_hi A_hi A_lo] [X_hi; X_lo; X_hi].
//
// FP64-result mode (HSMA_R64_IR): X_0 from the FP32-result solve of the
// rounded data, then iterative refinement: R = alpha B - L X in FP64 (FP64
// tensor products), C from the FP32-result solve of L C = R, X += C in FP64,
// until ||R||_F / (||L||_F ||X||_F + |alpha| ||B||_F) <= tol.  Every
// refinement kernel checks a device-side "converged" flag first, so the host
// enqueues the maximum number of steps without waiting on the device.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>

#include "blocked.h"
#include "common.cuh"
#include "mixed.h"
#include "tma.cuh"
#include "trace.h"
#include "workspace.h"

namespace {

// ---------------------------------------------------------------------------
// tcgen05 BF16 x BF16 -> FP32 update:  C (M x N, column-major fp32) =
// beta*C - A' B'^T with A' (M x K) and B' (N x K) row-major BF16 (K-major).
// ---------------------------------------------------------------------------
constexpr int TC_BM = 128, TC_BN = 256, TC_BK = 64, TC_STAGES = 4;
constexpr int TC_A_BYTES = TC_BM * TC_BK * 2;
constexpr int TC_B_BYTES = TC_BN * TC_BK * 2;
constexpr int TC_STAGE_BYTES = TC_A_BYTES + TC_B_BYTES;
constexpr int TC_SMEM = TC_STAGES * TC_STAGE_BYTES + 1024;
constexpr uint32_t TC_TMEM_COLS = 256;

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes in groups of 8 (1024 bytes apart).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1u << 16;              // leading-dimension offset (unused with this swizzle)
  d |= (uint64_t)(1024u >> 4) << 32;    // stride between 8-row groups
  d |= (uint64_t)1u << 46;              // descriptor version
  d |= (uint64_t)2u << 61;              // 128-byte swizzle
  return d;
}

// Instruction descriptor: FP32 accumulator, BF16 A and B, both K-major, M x N.
__host__ __device__ constexpr uint32_t tc_idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_BN >> 3) << 17) | ((uint32_t)(TC_BM >> 4) << 24);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Epilogues of the tensor-core product:
//   TC_F32:    C32 = beta*C32 - acc                    (the FP32-result update)
//   TC_F64ACC: C64 -= w * 2^(rexp[i] + cexp[j]) * acc  (one slice pair of an
//              emulated FP64 product; acc holds an exact integer)
enum { TC_F32 = 0, TC_F64ACC = 1 };

struct TcArgs {
  float *C32;
  double *C64;
  int64_t ldc;
  float beta;
  double w;
  const int *rexp;
  const double *cscale;  // 2^cexp[j]
  int M, N, K;
  int tri;          // row tile i0 needs k < i0 + TC_BM only
  const int *skip;  // device flag: when set, the launch does nothing
  unsigned int *err;
  uint64_t limit_ns;
};

// 32 lanes x 16 consecutive 32-bit tensor-memory columns into registers
// (completion awaited separately with tcgen05.wait::ld).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t *v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}

// Persistent, warp-specialised product: warp 0 loads operand stages by TMA,
// warp 1 issues the MMAs, warps 2..9 drain accumulators.  Two accumulators of
// 256 tensor-memory columns alternate between tiles, so the epilogue of one
// tile runs while the next tile's products accumulate.  Tiles are dealt
// round-robin to the CTAs (one per SM).
constexpr int TC_WARPS = 10;
constexpr int TC_EPI_WARPS = 8;

template <int MODE>
__global__ void __launch_bounds__(32 * TC_WARPS, 1) tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA,
                                                                   const __grid_constant__ CUtensorMap mapB,
                                                                   const TcArgs p) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[TC_STAGES];
  __shared__ __align__(8) uint64_t empty[TC_STAGES];
  __shared__ __align__(8) uint64_t acc_full[2];
  __shared__ __align__(8) uint64_t acc_empty[2];
  __shared__ __align__(8) uint64_t drained;
  __shared__ uint32_t tmem_base;
  if (p.skip != nullptr && *(volatile const int *)p.skip != 0) return;
  unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int M = p.M, N = p.N;
  const int tiles_m = (M + TC_BM - 1) / TC_BM, tiles_n = (N + TC_BN - 1) / TC_BN;
  const int ntiles = tiles_m * tiles_n;
  auto tile_k = [&](int t, int &m0, int &n0) {  // tile -> origin and K-block count
    m0 = (t % tiles_m) * TC_BM;
    n0 = (t / tiles_m) * TC_BN;
    const int kall = p.tri ? min(p.K, m0 + TC_BM) : p.K;
    return (kall + TC_BK - 1) / TC_BK;
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], TC_EPI_WARPS);
    }
    mbar_init(&drained, 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(2 * TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;

  if (warp == 0) {
    if (lane == 0) {
      // producer: TMA loads into a ring of stages, across tiles
      int it = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        int m0, n0;
        const int nk = tile_k(t, m0, n0);
        for (int kb = 0; kb < nk; ++kb, ++it) {
          const int s = it % TC_STAGES;
          if (it >= TC_STAGES && !mbar_wait_bounded(&empty[s], ((it / TC_STAGES) - 1) & 1, p.limit_ns, p.err)) {
            ok = false;
            break;
          }
          unsigned char *sa = smem + s * TC_STAGE_BYTES;
          mbar_arrive_expect_tx(&full[s], TC_STAGE_BYTES);
          tma_load_2d(sa, &mapA, &full[s], kb * TC_BK, m0);
          tma_load_2d(sa + TC_A_BYTES, &mapB, &full[s], kb * TC_BK, n0);
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer: per tile, wait for a drained accumulator, then four K = 16
      // steps per stage; each stage is released by a commit, the tile by another
      int it = 0, i = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++i) {
        int m0, n0;
        const int nk = tile_k(t, m0, n0);
        const int b = i & 1;
        if (i >= 2 && !mbar_wait_bounded(&acc_empty[b], ((i >> 1) - 1) & 1, p.limit_ns, p.err)) break;
        tc_fence_after();
        const uint32_t acc_cols = tmem + (uint32_t)(b * TC_TMEM_COLS);
        for (int kb = 0; kb < nk; ++kb, ++it) {
          const int s = it % TC_STAGES;
          if (!mbar_wait_bounded(&full[s], (it / TC_STAGES) & 1, p.limit_ns, p.err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = smem_u32(smem + s * TC_STAGE_BYTES);
          const uint64_t da = sw128_desc(sa), db = sw128_desc(sa + TC_A_BYTES);
#pragma unroll
          for (int kk = 0; kk < TC_BK / 16; ++kk) {
            const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
            asm volatile(
                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(acc_cols),
                "l"(da + 2ull * kk), "l"(db + 2ull * kk), "r"(tc_idesc()), "r"(acc)
                : "memory");
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           smem_u32(&empty[s]))
                       : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&acc_full[b]))
                     : "memory");
      }
      // every issued product has finished before tensor memory is released,
      // also when a wait above gave up
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&drained))
                   : "memory");
      mbar_wait_bounded(&drained, 0, p.limit_ns, p.err);
    }
    __syncwarp();
  } else {
    // epilogue warps: thread = one row of the 128-row tile (its tensor-memory
    // lane); two warps per lane quarter split the 256 columns.  The old values
    // of the next 32-column chunk are loaded before this chunk's stores.
    const int ew = warp - 2;
    const int quarter = warp & 3, half = ew >> 2;
    const int cbeg = half * (TC_BN / 2);
    using V = typename std::conditional<MODE == TC_F32, float, double>::type;
    int i = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
      int m0, n0;
      const int nk = tile_k(t, m0, n0);
      const int b = i & 1;
      const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&acc_full[b], (i >> 1) & 1, p.limit_ns, p.err));
      if (!ok) break;
      tc_fence_after();
      const int row = m0 + quarter * 32 + lane;
      const double rs = (MODE == TC_F64ACC && row < M) ? ldexp(p.w, p.rexp[row]) : 0.0;
      constexpr int CW = 16;  // columns per chunk: keeps ten warps within the register file
      V old[CW], nxt[CW];
      auto load_chunk = [&](int c0, V *dst) {
#pragma unroll
        for (int j = 0; j < CW; ++j) {
          const int col = n0 + c0 + j;
          if constexpr (MODE == TC_F32)
            dst[j] = (row < M && col < N) ? __ldcs(p.C32 + row + (int64_t)col * p.ldc) : 0.0f;
          else
            dst[j] = (row < M && col < N) ? __ldcs(p.C64 + row + (int64_t)col * p.ldc) : 0.0;
        }
      };
      load_chunk(cbeg, nxt);
#pragma unroll 1
      for (int c0 = cbeg; c0 < cbeg + TC_BN / 2; c0 += CW) {
#pragma unroll
        for (int j = 0; j < CW; ++j) old[j] = nxt[j];
        if (c0 + CW < cbeg + TC_BN / 2) load_chunk(c0 + CW, nxt);
        uint32_t v[CW];
        const uint32_t taddr = tmem + (uint32_t)(b * TC_TMEM_COLS) + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0;
#pragma unroll
        for (int h = 0; h < CW / 16; ++h) tmem_ld16(taddr + 16 * h, v + 16 * h);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (row < M && nk > 0) {
#pragma unroll
          for (int j = 0; j < CW; ++j) {
            const int col = n0 + c0 + j;
            if (col < N) {
              const float a = __uint_as_float(v[j]);
              if constexpr (MODE == TC_F32) {
                __stcs(p.C32 + row + (int64_t)col * p.ldc,
                       (p.beta == 1.0f) ? (old[j] - a) : fmaf(p.beta, old[j], -a));
              } else {
                __stcs(p.C64 + row + (int64_t)col * p.ldc, fma(-(rs * p.cscale[col]), (double)a, old[j]));
              }
            }
          }
        }
      }
      // this warp is done with accumulator b
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[b]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TC_TMEM_COLS)
                 : "memory");
  }
}

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
// Conversions to the tensor-core operand layouts.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16 &hi, __nv_bfloat16 &lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// A panel (rows x nb, column-major fp32, lda) -> A' rows x Kp row-major BF16:
// terms 1: [hi], terms 3: [hi | hi | lo]; columns past terms*nb are zero.
__global__ void __launch_bounds__(256) convert_panel_kernel(const float *__restrict__ A, int64_t lda, int rows,
                                                            int nb, int terms, int Kp, __nv_bfloat16 *out) {
  __shared__ float tile[32][33];
  const int i0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
  for (int kk = ty; kk < 32; kk += 8) {
    const int i = i0 + tx, k = k0 + kk;
    tile[kk][tx] = (i < rows && k < nb) ? A[i + (int64_t)k * lda] : 0.0f;
  }
  __syncthreads();
  for (int ii = ty; ii < 32; ii += 8) {
    const int i = i0 + ii, k = k0 + tx;
    if (i >= rows) continue;
    __nv_bfloat16 *o = out + (int64_t)i * Kp;
    if (k < nb) {
      __nv_bfloat16 hi, lo;
      split_bf16(tile[tx][ii], hi, lo);
      o[k] = hi;
      if (terms == 3) {
        o[nb + k] = hi;
        o[2 * nb + k] = lo;
      }
    }
    // zero padding columns [terms*nb, Kp)
    for (int kp = terms * nb + k0 + tx; kp < Kp && blockIdx.y == 0; kp += 32) o[kp] = __float2bfloat16_rn(0.0f);
  }
}

// X_r (nb x n, column-major fp32, ldx) -> X' n x Kp row-major BF16:
// terms 1: [hi], terms 3: [hi | lo | hi]; zero padding to Kp.
__global__ void __launch_bounds__(256) convert_x_kernel(const float *__restrict__ X, int64_t ldx, int nb, int n,
                                                        int terms, int Kp, __nv_bfloat16 *out, const int *skip) {
  if (skip != nullptr && *(volatile const int *)skip) return;
  const int64_t total = (int64_t)n * Kp;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / Kp), kp = (int)(e % Kp);
    const int part = kp / nb, k = kp % nb;
    float v = 0.0f;
    if (part < terms) {
      const float x = X[k + (int64_t)j * ldx];
      __nv_bfloat16 hi, lo;
      split_bf16(x, hi, lo);
      out[e] = (terms == 3 && part == 1) ? lo : hi;
      continue;
    }
    out[e] = __float2bfloat16_rn(v);
  }
}

int g_launch_grid(int64_t total) {
  int64_t b = (total + 255) / 256;
  return (int)std::min<int64_t>(std::max<int64_t>(b, 1), 152 * 32);
}

template <int MODE>
hsma_status_t tc_gemm(const __nv_bfloat16 *Ap, const __nv_bfloat16 *Bp, const TcArgs &a0, const char *phase,
                      cudaStream_t st) {
  if (a0.M <= 0 || a0.N <= 0) return HSMA_OK;
  if (a0.K % TC_BK != 0 || a0.K <= 0) return HSMA_ERR_INVALID_ARG;
  static DeviceFlags attr;
  if (!attr.test()) {
    HSMA_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
    attr.set();
  }
  CUtensorMap ma, mb;
  if (!hsma_make_map_2d(&ma, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, Ap, (uint64_t)a0.K, (uint64_t)a0.M, (uint64_t)a0.K,
                        TC_BK, TC_BM, CU_TENSOR_MAP_SWIZZLE_128B) ||
      !hsma_make_map_2d(&mb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, Bp, (uint64_t)a0.K, (uint64_t)a0.N, (uint64_t)a0.K,
                        TC_BK, TC_BN, CU_TENSOR_MAP_SWIZZLE_128B))
    return HSMA_ERR_CUDA;
  TcArgs a = a0;
  a.err = hsma_dev_error_ptr();
  if (a.err == nullptr) return HSMA_ERR_CUDA;
  if (a.limit_ns == 0) a.limit_ns = 4000000000ull;
  const int tiles = ((a.M + TC_BM - 1) / TC_BM) * ((a.N + TC_BN - 1) / TC_BN);
  static int nsm[64] = {0};
  int dev = 0;
  HSMA_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return HSMA_ERR_UNSUPPORTED;
  if (nsm[dev] == 0) HSMA_CUDA_TRY(cudaDeviceGetAttribute(&nsm[dev], cudaDevAttrMultiProcessorCount, dev));
  const int grid = tiles < nsm[dev] ? tiles : nsm[dev];
  HsmaTraceScope ts(phase, st);
  tc_gemm_kernel<MODE><<<grid, 32 * TC_WARPS, TC_SMEM, st>>>(ma, mb, a);
  HSMA_CUDA_TRY(cudaGetLastError());
  return HSMA_OK;
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
  return tc_gemm<TC_F32>(Ap, Bp, a, "update_bf16", st);
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
};

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
  const int64_t total = (int64_t)rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % rows, j = e / rows;
    dst[i + j * ldd] = src[i + j * lds];
  }
}

hsma_status_t r32_prepare(R32Plan &P, bool keep_panels, cudaStream_t st) {
  hsma_status_t s = hsma_diag_inverse(HSMA_R32_BF16, P.nb, P.A, P.lda, P.m, P.unit, P.Dinv, st);
  if (s != HSMA_OK || !keep_panels) return s;
  const int64_t nblk = (P.m + P.nb - 1) / P.nb;
  HsmaTraceScope ts("convert", st);
  for (int64_t r = 0; r + 1 < nblk; ++r) {
    const int64_t r0 = r * P.nb, sr = std::min<int64_t>(P.nb, P.m - r0);
    const int rows = (int)panel_rows(P, r);
    dim3 g1((rows + 31) / 32, (P.nb + 31) / 32);
    convert_panel_kernel<<<g1, 256, 0, st>>>(P.A + (r0 + sr) + r0 * P.lda, P.lda, rows, P.nb, P.terms, P.Kp,
                                             P.panels + panel_off(P, r));
  }
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
  const size_t w_b = sizeof(float) * (size_t)nb * n;
  const size_t a_b = P.panels ? 0 : sizeof(__nv_bfloat16) * (size_t)rows_max * Kp;
  const size_t x_b = sizeof(__nv_bfloat16) * (size_t)n * Kp;
  auto al = [](size_t v) { return (v + 1023) & ~(size_t)1023; };
  void *ws = nullptr;
  hsma_status_t s = hsma_ws_alloc(&ws, al(w_b) + al(a_b) + al(x_b), st);
  if (s != HSMA_OK) return s;
  unsigned char *base = static_cast<unsigned char *>(ws);
  float *W = reinterpret_cast<float *>(base);
  __nv_bfloat16 *Ap = reinterpret_cast<__nv_bfloat16 *>(base + al(w_b));
  __nv_bfloat16 *Xp = reinterpret_cast<__nv_bfloat16 *>(base + al(w_b) + al(a_b));
  for (int64_t r = 0; r < nblk && s == HSMA_OK; ++r) {
    const int64_t r0 = r * nb;
    const int sr = (int)std::min<int64_t>(nb, m - r0);
    {
      HsmaTraceScope ts("copy", st);
      copy_f32_kernel<<<g_launch_grid((int64_t)sr * n), 256, 0, st>>>(B + r0, ldb, W, nb, sr, n, skip);
    }
    s = sgemm_scale(P.Dinv + (size_t)r * nb * nb, nb, W, nb, B + r0, ldb, sr, (int)n, sr, r == 0 ? alpha : 1.0f, 1,
                    skip, st);
    if (s != HSMA_OK || r0 + sr >= m) break;
    const int rows = (int)(m - r0 - sr);
    const __nv_bfloat16 *panel = P.panels ? P.panels + panel_off(P, r) : Ap;
    {
      HsmaTraceScope ts("convert", st);
      if (!P.panels) {
        dim3 g1((rows + 31) / 32, (nb + 31) / 32);
        convert_panel_kernel<<<g1, 256, 0, st>>>(P.A + (r0 + sr) + r0 * P.lda, P.lda, rows, nb, P.terms, Kp, Ap);
      }
      convert_x_kernel<<<g_launch_grid((int64_t)n * Kp), 256, 0, st>>>(B + r0, ldb, nb, (int)n, P.terms, Kp, Xp,
                                                                       skip);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) {
        s = hsma_from_cuda(e);
        break;
      }
    }
    TcArgs a{};
    a.C32 = B + r0 + sr;
    a.ldc = ldb;
    a.beta = r == 0 ? alpha : 1.0f;
    a.M = rows;
    a.N = (int)n;
    a.K = Kp;
    a.skip = skip;
    s = tc_gemm<TC_F32>(panel, Xp, a, "update_bf16", st);
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
  void *ws = nullptr;
  hsma_status_t s = hsma_ws_alloc(&ws, sizeof(float) * (size_t)nblk * nb * nb, st);
  if (s != HSMA_OK) return s;
  P.Dinv = static_cast<float *>(ws);
  s = r32_prepare(P, false, st);
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
  const int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % rows, j = e / rows;
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
  const int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % rows, j = e / rows;
    const double c = (double)Cc[i + j * ldc];
    X[i + j * ldx] = assign ? c : X[i + j * ldx] + c;
  }
}

// sums[slot] += sum of squares (lower triangle only when lower; unit diagonal counts 1)
__global__ void sumsq_kernel(const double *__restrict__ M_, int64_t ld, int64_t rows, int64_t cols, int lower,
                             int unit, double *sums, int slot, const int *flag) {
  if (flag != nullptr && *(volatile const int *)flag) return;
  double acc = 0.0;
  const int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % rows, j = e / rows;
    if (lower && i < j) continue;
    const double v = (lower && unit && i == j) ? 1.0 : M_[i + j * ld];
    acc = fma(v, v, acc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(&sums[slot], acc);
}

// sums: [0] ||L||^2, [1] ||B||^2, [2] ||R||^2, [3] ||X||^2; state: [0] converged, [1] steps, [2..3] eta (double)
__global__ void check_kernel(double *sums, int *state, double alpha_abs, double tol, int step) {
  if (state[0]) return;
  const double nr = sqrt(sums[2]), den = sqrt(sums[0]) * sqrt(sums[3]) + alpha_abs * sqrt(sums[1]);
  const double eta = den > 0.0 ? nr / den : nr;
  *reinterpret_cast<double *>(state + 2) = eta;
  state[1] = step;
  if (eta <= tol) state[0] = 1;
  sums[2] = 0.0;
  sums[3] = 0.0;
}

// ---------------------------------------------------------------------------
// FP64 product emulated on the BF16 tensor cores (Ozaki-style exact slices).
//
// Each row i of L is scaled by 2^-e_i and each column j of X by 2^-f_j (powers
// of two, exact) so that every entry lies in (-1, 1); an entry a is then cut
// into kOzS signed digits, a = sum_p d_p 2^-b_p + r, b_p = 5 + 6(p-1), with
// d_p = rint(r_{p-1} 2^b_p) in [-32, 32] and r_p = r_{p-1} - d_p 2^-b_p, all
// exact in FP64.  A digit is exact in BF16 and a product of two digits is at
// most 2^10, so for K <= 2^14 every partial sum of a slice-pair product is an
// integer below 2^24: the FP32 tensor-memory accumulation is exact.  Pairs with
// p + q <= kOzS + 1 are kept and each is folded into the FP64 result with its
// weight 2^(e_i + f_j - b_p - b_q).  The dropped pairs and the digit remainders
// contribute below 2^-60 of |row scale| |column scale| per product.
// ---------------------------------------------------------------------------
constexpr int kOzS = 10;
constexpr int kOzMaxK = 1 << 14;
constexpr int kOzExpEmpty = -1100;  // exponent of an all-zero row or column

__host__ __device__ constexpr int oz_bits(int p) { return 5 + 6 * (p - 1); }

// e_i = exponent with |L_ik| < 2^e_i over the lower triangle (unit diagonal: 1)
__global__ void oz_rowexp_kernel(const double *__restrict__ A, int64_t lda, int M, int K, int unit, int *rexp) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  const int k0 = blockIdx.y * 64, k1 = min(K, k0 + 64);
  double mx = 0.0;
  for (int k = k0; k < k1 && k <= i; ++k) {
    const double v = (k == i && unit) ? 1.0 : fabs(A[i + (int64_t)k * lda]);
    mx = fmax(mx, v);
  }
  if (mx > 0.0) {
    int e;
    frexp(mx, &e);
    atomicMax(&rexp[i], e);
  }
}

// f_j and 2^f_j for the columns of X (one CTA per column)
__global__ void __launch_bounds__(256) oz_colexp_kernel(const double *__restrict__ X, int64_t ldx, int K, int *cexp,
                                                        double *cscale, const int *skip) {
  if (skip != nullptr && *(volatile const int *)skip) return;
  __shared__ double red[8];
  const int j = blockIdx.x;
  double mx = 0.0;
  for (int k = threadIdx.x; k < K; k += blockDim.x) mx = fmax(mx, fabs(X[k + (int64_t)j * ldx]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < 8; ++w) mx = fmax(mx, red[w]);
    int e = 0;
    if (mx > 0.0) frexp(mx, &e);
    cexp[j] = e;
    cscale[j] = ldexp(1.0, e);
  }
}

__device__ __forceinline__ void oz_digits(double a, __nv_bfloat16 *out, size_t stride) {
  double r = a;
#pragma unroll
  for (int p = 1; p <= kOzS; ++p) {
    const double t = ldexp(r, oz_bits(p));
    const double d = rint(t);
    r -= ldexp(d, -oz_bits(p));
    out[(size_t)(p - 1) * stride] = __float2bfloat16_rn((float)d);
  }
}

// slices of L (lower triangle of A): out[p][i][k], row-major M x Kp per slice
__global__ void __launch_bounds__(256) oz_slice_rows_kernel(const double *__restrict__ A, int64_t lda, int M, int K,
                                                            int Kp, int unit, const int *rexp, __nv_bfloat16 *out) {
  __shared__ double tile[32][33];
  const int i0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
  for (int kk = ty; kk < 32; kk += 8) {
    const int i = i0 + tx, k = k0 + kk;
    double v = 0.0;
    if (i < M && k < K && k <= i) v = (k == i && unit) ? 1.0 : A[i + (int64_t)k * lda];
    tile[kk][tx] = v;
  }
  __syncthreads();
  const size_t stride = (size_t)M * Kp;
  for (int ii = ty; ii < 32; ii += 8) {
    const int i = i0 + ii, k = k0 + tx;
    if (i >= M || k >= Kp) continue;
    const int e = rexp[i];
    const double a = e == kOzExpEmpty ? 0.0 : ldexp(tile[tx][ii], -e);
    oz_digits(a, out + (size_t)i * Kp + k, stride);
  }
}

// slices of X: out[q][j][k], row-major N x Kp per slice
__global__ void __launch_bounds__(256) oz_slice_cols_kernel(const double *__restrict__ X, int64_t ldx, int K, int N,
                                                            int Kp, const int *cexp, __nv_bfloat16 *out,
                                                            const int *skip) {
  if (skip != nullptr && *(volatile const int *)skip) return;
  const int64_t total = (int64_t)N * Kp;
  const size_t stride = (size_t)N * Kp;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / Kp), k = (int)(e % Kp);
    const double x = k < K ? X[k + (int64_t)j * ldx] : 0.0;
    oz_digits(ldexp(x, -cexp[j]), out + e, stride);
  }
}

__global__ void oz_fill_kernel(int *p, int n, int v) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) p[k] = v;
}

struct OzL {  // slices of L, built once per solve
  __nv_bfloat16 *slices = nullptr;
  int *rexp = nullptr;
  int M = 0, Kp = 0;
};

size_t oz_l_bytes(int64_t m) {
  const size_t Kp = (size_t)((m + TC_BK - 1) / TC_BK) * TC_BK;
  return kOzS * (size_t)m * Kp * sizeof(__nv_bfloat16) + 1024 + sizeof(int) * (size_t)m;
}

size_t oz_x_bytes(int64_t m, int64_t n) {
  const size_t Kp = (size_t)((m + TC_BK - 1) / TC_BK) * TC_BK;
  return kOzS * (size_t)n * Kp * sizeof(__nv_bfloat16) + 1024 + (sizeof(int) + sizeof(double)) * (size_t)n + 1024;
}

hsma_status_t oz_prepare_l(const double *A, int64_t lda, int unit, int64_t m, void *ws, OzL *L, cudaStream_t st) {
  const int Kp = (int)((m + TC_BK - 1) / TC_BK) * TC_BK;
  unsigned char *b = static_cast<unsigned char *>(ws);
  L->slices = reinterpret_cast<__nv_bfloat16 *>(b);
  L->rexp = reinterpret_cast<int *>(b + ((kOzS * (size_t)m * Kp * sizeof(__nv_bfloat16) + 1023) & ~(size_t)1023));
  L->M = (int)m;
  L->Kp = Kp;
  HsmaTraceScope ts("residual_slices", st);
  oz_fill_kernel<<<(unsigned)std::min<int64_t>((m + 255) / 256, 1024), 256, 0, st>>>(L->rexp, (int)m, kOzExpEmpty);
  oz_rowexp_kernel<<<dim3((unsigned)((m + 255) / 256), (unsigned)((m + 63) / 64)), 256, 0, st>>>(A, lda, (int)m,
                                                                                                 (int)m, unit,
                                                                                                 L->rexp);
  oz_slice_rows_kernel<<<dim3((unsigned)((m + 31) / 32), (unsigned)((Kp + 31) / 32)), 256, 0, st>>>(
      A, lda, (int)m, (int)m, Kp, unit, L->rexp, L->slices);
  HSMA_CUDA_TRY(cudaGetLastError());
  return HSMA_OK;
}

// R -= L X in emulated FP64 (R holds alpha B on entry); skip: device flag
hsma_status_t oz_residual(const OzL &L, const double *X, int64_t ldx, double *R, int64_t ldr, int64_t n, void *ws,
                          const int *skip, cudaStream_t st) {
  const int m = L.M, Kp = L.Kp;
  unsigned char *b = static_cast<unsigned char *>(ws);
  __nv_bfloat16 *XS = reinterpret_cast<__nv_bfloat16 *>(b);
  size_t off = (kOzS * (size_t)n * Kp * sizeof(__nv_bfloat16) + 1023) & ~(size_t)1023;
  int *cexp = reinterpret_cast<int *>(b + off);
  double *cscale = reinterpret_cast<double *>(b + ((off + sizeof(int) * (size_t)n + 1023) & ~(size_t)1023));
  {
    HsmaTraceScope ts("residual_slices", st);
    oz_colexp_kernel<<<(unsigned)n, 256, 0, st>>>(X, ldx, m, cexp, cscale, skip);
    oz_slice_cols_kernel<<<g_launch_grid((int64_t)n * Kp), 256, 0, st>>>(X, ldx, m, (int)n, Kp, cexp, XS, skip);
    HSMA_CUDA_TRY(cudaGetLastError());
  }
  for (int pa = 1; pa <= kOzS; ++pa)
    for (int qb = 1; pa + qb <= kOzS + 1; ++qb) {
      TcArgs a{};
      a.C64 = R;
      a.ldc = ldr;
      a.w = ldexp(1.0, -(oz_bits(pa) + oz_bits(qb)));
      a.rexp = L.rexp;
      a.cscale = cscale;
      a.M = m;
      a.N = (int)n;
      a.K = Kp;
      a.tri = 1;
      a.skip = skip;
      hsma_status_t s = tc_gemm<TC_F64ACC>(L.slices + (size_t)(pa - 1) * m * Kp, XS + (size_t)(qb - 1) * n * Kp, a,
                                           "residual", st);
      if (s != HSMA_OK) return s;
    }
  return HSMA_OK;
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
  const size_t ozl_b = emulated ? al(oz_l_bytes(m)) : 0;
  const size_t ozx_b = emulated ? al(oz_x_bytes(m, n)) : 0;
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
  OzL Lsl;
  P.A = A32;
  P.Dinv = reinterpret_cast<float *>(static_cast<unsigned char *>(ozx_ws) + ozx_b);
  P.panels = reinterpret_cast<__nv_bfloat16 *>(reinterpret_cast<unsigned char *>(P.Dinv) + dinv_b);
  const int grid = g_launch_grid(m * n);
  auto fail = [&](cudaError_t e) { return e == cudaSuccess ? HSMA_OK : hsma_from_cuda(e); };
  do {
    if ((s = fail(cudaMemsetAsync(sums, 0, st_b, st))) != HSMA_OK) break;
    if ((s = fail(cudaMemcpy2DAsync(B0, sizeof(double) * m, B, sizeof(double) * ldb, sizeof(double) * m, n,
                                    cudaMemcpyDeviceToDevice, st))) != HSMA_OK)
      break;
    {
      HsmaTraceScope ts("convert", st);
      f64_to_f32_kernel<<<g_launch_grid(m * m), 256, 0, st>>>(A, lda, A32, m, m, m, 1, nullptr);
      f64_to_f32_kernel<<<grid, 256, 0, st>>>(B, ldb, R32, m, m, n, 0, nullptr);
      sumsq_kernel<<<g_launch_grid(m * m), 256, 0, st>>>(A, lda, m, m, 1, unit, sums, 0, nullptr);
      sumsq_kernel<<<grid, 256, 0, st>>>(B0, m, m, n, 0, 0, sums, 1, nullptr);
      if ((s = fail(cudaGetLastError())) != HSMA_OK) break;
    }
    if (emulated && (s = oz_prepare_l(A, lda, unit, m, ozl_ws, &Lsl, st)) != HSMA_OK) break;
    // X_0 from the FP32-result solve of the rounded data
    if ((s = r32_prepare(P, true, st)) != HSMA_OK) break;
    if ((s = r32_apply(P, R32, m, n, (float)alpha, nullptr, st)) != HSMA_OK) break;
    {
      HsmaTraceScope ts("refine", st);
      accumulate_kernel<<<grid, 256, 0, st>>>(B, ldb, R32, m, m, n, 1, nullptr);
    }
    for (int it = 0; it <= itmax && s == HSMA_OK; ++it) {
      // R = alpha B - L X in FP64, then the stopping test
      if (emulated) {
        {
          HsmaTraceScope ts("refine", st);
          scale_copy_kernel<<<grid, 256, 0, st>>>(B0, R64, m * n, alpha, state);
        }
        if ((s = oz_residual(Lsl, B, ldb, R64, m, n, ozx_ws, state, st)) != HSMA_OK) break;
      } else {
        if ((s = fail(cudaMemcpy2DAsync(R64, sizeof(double) * m, B0, sizeof(double) * m, sizeof(double) * m, n,
                                        cudaMemcpyDeviceToDevice, st))) != HSMA_OK)
          break;
        if ((s = hsma_residual_f64(A, lda, unit, B, ldb, R64, m, m, n, alpha, state, st)) != HSMA_OK) break;
      }
      {
        HsmaTraceScope ts("refine", st);
        sumsq_kernel<<<grid, 256, 0, st>>>(R64, m, m, n, 0, 0, sums, 2, state);
        sumsq_kernel<<<grid, 256, 0, st>>>(B, ldb, m, n, 0, 0, sums, 3, state);
        check_kernel<<<1, 1, 0, st>>>(sums, state, std::fabs(alpha), tol, it);
        if (it == itmax) break;
        f64_to_f32_kernel<<<grid, 256, 0, st>>>(R64, m, R32, m, m, n, 0, state);
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
  if (A == nullptr || Bt == nullptr || C == nullptr || K == 0 || K % TC_BK != 0) return HSMA_ERR_INVALID_ARG;
  if (M > INT32_MAX || N > INT32_MAX || K > INT32_MAX) return HSMA_ERR_UNSUPPORTED;
  return bf16_update(static_cast<const __nv_bfloat16 *>(A), static_cast<const __nv_bfloat16 *>(Bt), (int)M, (int)N,
                     (int)K, beta, C, ldc, static_cast<cudaStream_t>(stream));
}
