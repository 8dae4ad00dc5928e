// Persistent, warp-specialised tcgen05 product (BF16 x BF16 -> FP32 in tensor
// memory) behind the FP32-result mode and the emulated FP64 products; used by
// mixed.cu only.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <type_traits>

#include "blocked.h"
#include "common.cuh"
#include "tma.cuh"
#include "trace.h"

namespace {

// ---------------------------------------------------------------------------
// tcgen05 BF16 x BF16 -> FP32 update:  C (M x N, column-major fp32) =
// beta*C - A' B'^T with A' (M x K) and B' (N x K) row-major BF16 (K-major).
// ---------------------------------------------------------------------------
// K-block of a pipeline stage: 64 BF16 values (128-byte rows, 128-byte
// swizzle, four 48 KB stages), or 32 (64-byte rows and swizzle, nine 24 KB
// stages: more bytes in flight behind the stage being multiplied).  Measured
// on GB300 the 32-wide ring is 20-25% slower on every product (emulated FP64
// 16384^2 solve 209 -> 258 ms, FP32-result 8192 x 4096 update 1.10 -> 1.20 ms),
// so the products are not bound by how many bytes the ring keeps in flight.
#ifndef HSMA_TC_BK
#define HSMA_TC_BK 64
#endif
constexpr int TC_BM = 128, TC_BN = 256, TC_BK = HSMA_TC_BK;
constexpr int TC_ROW_BYTES = TC_BK * 2;  // one K-row of a stage tile: the swizzle width
static_assert(TC_ROW_BYTES == 64 || TC_ROW_BYTES == 128, "K-blocks of 32 or 64 BF16 values");
constexpr int TC_A_BYTES = TC_BM * TC_BK * 2;
constexpr int TC_B_BYTES = TC_BN * TC_BK * 2;
constexpr int TC_STAGE_BYTES = TC_A_BYTES + TC_B_BYTES;
constexpr int TC_STAGES = TC_BK == 32 ? 9 : 4;
constexpr int TC_SMEM = TC_STAGES * TC_STAGE_BYTES + 1024;
static_assert(TC_SMEM <= 227 * 1024 - 256, "stages fit the shared memory of one CTA");
static_assert(TC_STAGE_BYTES % 1024 == 0, "every stage starts on a swizzle-pattern boundary");
constexpr uint32_t TC_TMEM_COLS = 256;

// Shared-memory matrix descriptor: K-major operand, rows of TC_ROW_BYTES in
// groups of 8 (8 * TC_ROW_BYTES apart), swizzled over the row width
// (layout codes: 2 = 128-byte, 4 = 64-byte swizzle).
__device__ __forceinline__ uint64_t sw_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1u << 16;                                // leading-dimension offset (unused when swizzled)
  d |= (uint64_t)((8u * TC_ROW_BYTES) >> 4) << 32;        // stride between 8-row groups
  d |= (uint64_t)1u << 46;                                // descriptor version
  d |= (uint64_t)(TC_ROW_BYTES == 128 ? 2u : 4u) << 61;   // swizzle mode
  return d;
}

// Instruction descriptor: FP32 accumulator, BF16 A and B, both K-major, M x N.
__host__ __device__ constexpr uint32_t tc_idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_BN >> 3) << 17) | ((uint32_t)(TC_BM >> 4) << 24);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Epilogues of the tensor-core product:
//   TC_F32: C32 = beta*C32 - acc                    (the FP32-result update)
//   TC_OZ:  C64 -/+= 2^(rexp[i] + cexp[j] + uexp[u]) * acc_u for every
//           accumulation unit u of the tile (an emulated FP64 product; each
//           acc_u holds an exact integer)
enum { TC_F32 = 0, TC_OZ = 1 };

// Emulated FP64 products (see the Ozaki section below): kOzS slices per
// operand, pairs p + q <= kOzS + 1.
constexpr int kOzS = 10;
constexpr int kOzPairs = kOzS * (kOzS + 1) / 2;
constexpr int kOzMaxUnits = 64;

struct TcArgs {
  float *C32;
  double *C64;
  int64_t ldc;
  float beta;      // TC_F32
  int beta0;       // TC_OZ: 0 = the first unit overwrites C64 (old values not read)
  int negate;      // TC_OZ: add the product instead of subtracting it
  const int *rexp;  // TC_OZ: row exponents of A
  const int *cexp;  // TC_OZ: column exponents of B
  int M, N, K;
  int tri;          // row tile i0 needs k < i0 + TC_BM only
  int nunits;       // accumulation units per tile (TC_F32: 1)
  int band;         // tile rows per band of the tile order (set by the launcher)
  uint8_t ubeg[kOzMaxUnits + 1];  // unit u accumulates pairs ubeg[u] .. ubeg[u+1]-1
  int8_t uexp[kOzMaxUnits];       // TC_OZ: weight exponent of unit u
  uint8_t pa[kOzPairs], pb[kOzPairs];  // slice of A and of B for each pair
  const int *skip;  // device flag: when set, the launch does nothing
  unsigned int *err;
  uint64_t limit_ns;
  // TC_F32 side outputs: BF16 splits of the stored values, the right operands
  // of the next products (null: none)
  __nv_bfloat16 *xs2;  // rows < rows2: [col][ld2] hi at k = row; terms2 = 3 adds lo at nb2 + row, hi at 2 nb2 + row
  int ld2, nb2, terms2, rows2;
  __nv_bfloat16 *xs3;  // rows r3 .. r3 + rows3 - 1: three exact slices [s][col][ld3] at k = row - r3, slice stride per3
  int64_t per3;
  int ld3, r3, rows3;
};

// x = hi + lo with hi, lo in BF16 (the split of the FP32-result products)
__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16 &hi, __nv_bfloat16 &lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// x = a + b + c exactly (24 bits in three BF16 slices)
__device__ __forceinline__ void split3_bf16(float x, __nv_bfloat16 &a, __nv_bfloat16 &b, __nv_bfloat16 &c) {
  a = __float2bfloat16_rn(x);
  float r = x - __bfloat162float(a);
  b = __float2bfloat16_rn(r);
  r -= __bfloat162float(b);
  c = __float2bfloat16_rn(r);
}

// 32 lanes x 16 consecutive 32-bit tensor-memory columns into registers
// (completion awaited separately with tcgen05.wait::ld).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t *v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}

// acc * 2^shift in FP64 for an FP32 accumulator value acc (bits f): the
// exponent is rebased with integer operations, so the FP64 pipe only sees the
// final addition; ldexp covers results outside the normal range.
__device__ __forceinline__ double oz_scale(uint32_t f, int shift) {
  if ((f & 0x7fffffffu) == 0) return 0.0;
  const int E = (int)((f >> 23) & 0xffu) + (1023 - 127) + shift;
  if (E >= 1 && E <= 2046)
    return __hiloint2double((int)((f & 0x80000000u) | ((uint32_t)E << 20) | ((f & 0x7fffffu) >> 3)), (int)(f << 29));
  return ldexp((double)__uint_as_float(f), shift);
}

// Persistent, warp-specialised product: warp 0 loads operand stages by TMA,
// warp 1 issues the MMAs, warps 2..9 drain accumulators.  Work items are
// (tile, accumulation unit); two accumulators of 256 tensor-memory columns
// alternate between items, so the epilogue of one item runs while the next
// item's products accumulate.  Tiles are dealt round-robin to the CTAs (one
// per SM).  Operands are 3-D: (K, rows, slice); a unit sums the products of
// its slice pairs over the whole K range in one accumulator.  Every CTA loads
// its own A and B tiles with plain (single-CTA) TMA.
constexpr int TC_WARPS = 10;
constexpr int TC_EPI_WARPS = 8;

template <int MODE>
__global__ void __launch_bounds__(32 * TC_WARPS, 1) tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA,
                                                                   const __grid_constant__ CUtensorMap mapB,
                                                                   const __grid_constant__ TcArgs p) {
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
  const int M = p.M, N = p.N, nunits = p.nunits;
  const int cid = blockIdx.x, ncl = gridDim.x;
  const int tiles_m = (M + TC_BM - 1) / TC_BM, tiles_n = (N + TC_BN - 1) / TC_BN;
  const int ntiles = tiles_m * tiles_n;
  // Tiles run in bands of p.band tile rows, column by column inside a band.
  // For short K the host picks 16 tile rows, so the tiles in flight at once
  // (one per SM) cover about 16 row tiles x 10 column tiles and their operand
  // slices stay in L2 while every slice pair re-reads them; for
  // long K one band spans all rows (column-major order), so the right operand's
  // slices are shared by every row tile in flight.
  const int G = max(1, p.band);
  auto tile_k = [&](int t, int &m0, int &n0) {  // tile -> its origin and K-block count
    const int band = t / (G * tiles_n);
    const int gb = min(G, tiles_m - band * G);
    const int idx = t - band * G * tiles_n;
    const int pm = band * G + idx % gb;
    m0 = pm * TC_BM;
    n0 = (idx / gb) * TC_BN;
    const int kall = p.tri ? min(p.K, (pm + 1) * TC_BM) : p.K;
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
      // producer: TMA loads into a ring of stages, across items
      int it = 0;
      bool ok = true;
      for (int t = cid; t < ntiles && ok; t += ncl) {
        int m0, n0;
        const int nk = tile_k(t, m0, n0);
        for (int q = 0; q < p.ubeg[nunits] && ok; ++q) {
          const int sa = p.pa[q], sb = p.pb[q];
          for (int kb = 0; kb < nk; ++kb, ++it) {
            const int s = it % TC_STAGES;
            if (it >= TC_STAGES && !mbar_wait_bounded(&empty[s], ((it / TC_STAGES) - 1) & 1, p.limit_ns, p.err)) {
              ok = false;
              break;
            }
            unsigned char *st = smem + s * TC_STAGE_BYTES;
            mbar_arrive_expect_tx(&full[s], TC_STAGE_BYTES);
            tma_load_3d(st, &mapA, &full[s], kb * TC_BK, m0, sa);
            tma_load_3d(st + TC_A_BYTES, &mapB, &full[s], kb * TC_BK, n0, sb);
          }
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer: per item, wait for a drained accumulator, then four K = 16
      // steps per stage; each stage is released by a commit, the item by another
      int it = 0, i = 0;
      bool ok = true;
      for (int t = cid; t < ntiles && ok; t += ncl) {
        int m0, n0;
        const int nk = tile_k(t, m0, n0);
        for (int u = 0; u < nunits && ok; ++u, ++i) {
          const int b = i & 1;
          if (i >= 2 && !mbar_wait_bounded(&acc_empty[b], ((i >> 1) - 1) & 1, p.limit_ns, p.err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t acc_cols = tmem + (uint32_t)(b * TC_TMEM_COLS);
          uint32_t accum = 0;
          for (int q = p.ubeg[u]; q < p.ubeg[u + 1] && ok; ++q) {
            for (int kb = 0; kb < nk; ++kb, ++it) {
              const int s = it % TC_STAGES;
              if (!mbar_wait_bounded(&full[s], (it / TC_STAGES) & 1, p.limit_ns, p.err)) {
                ok = false;
                break;
              }
              tc_fence_after();
              const uint32_t sa = smem_u32(smem + s * TC_STAGE_BYTES);
              const uint64_t da = sw_desc(sa), db = sw_desc(sa + TC_A_BYTES);
#pragma unroll
              for (int kk = 0; kk < TC_BK / 16; ++kk) {
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(acc_cols),
                    "l"(da + 2ull * kk), "l"(db + 2ull * kk), "r"(tc_idesc()), "r"(accum)
                    : "memory");
                accum = 1u;
              }
              asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                               smem_u32(&empty[s]))
                           : "memory");
            }
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           smem_u32(&acc_full[b]))
                       : "memory");
        }
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
    // of the next 16-column chunk are loaded before this chunk's stores.  The
    // units of a tile are drained in order by the same threads, so each
    // read-modify-write of C sees the previous unit's stores.
    const int ew = warp - 2;
    const int quarter = warp & 3, half = ew >> 2;
    const int cbeg = half * (TC_BN / 2);
    using V = typename std::conditional<MODE == TC_F32, float, double>::type;
    constexpr int CW = 16;  // columns per chunk: keeps ten warps within the register file
    int i = 0;
    bool ok = true;
    for (int t = cid; t < ntiles && ok; t += ncl) {
      int m0, n0;
      const int nk = tile_k(t, m0, n0);
      const int row = m0 + quarter * 32 + lane;
      const int rx = (MODE == TC_OZ && row < M) ? p.rexp[row] : 0;
      for (int u = 0; u < nunits; ++u, ++i) {
        const int b = i & 1;
        ok = __all_sync(0xffffffffu, mbar_wait_bounded(&acc_full[b], (i >> 1) & 1, p.limit_ns, p.err));
        if (!ok) break;
        tc_fence_after();
        const bool fresh = MODE == TC_OZ && u == 0 && p.beta0 == 0;
        const int ushift = MODE == TC_OZ ? rx + p.uexp[u] : 0;
        V old[CW], nxt[CW];
        auto load_chunk = [&](int c0, V *dst) {
#pragma unroll
          for (int j = 0; j < CW; ++j) {
            const int col = n0 + c0 + j;
            if constexpr (MODE == TC_F32)
              dst[j] = (p.beta != 0.0f && row < M && col < N) ? __ldcs(p.C32 + row + (int64_t)col * p.ldc) : 0.0f;
            else
              dst[j] = (!fresh && row < M && col < N) ? p.C64[row + (int64_t)col * p.ldc] : 0.0;
          }
        };
        load_chunk(cbeg, nxt);
#pragma unroll 1
        for (int c0 = cbeg; c0 < cbeg + TC_BN / 2; c0 += CW) {
#pragma unroll
          for (int j = 0; j < CW; ++j) old[j] = nxt[j];
          if (c0 + CW < cbeg + TC_BN / 2) load_chunk(c0 + CW, nxt);
          uint32_t v[CW];
          const uint32_t taddr =
              tmem + (uint32_t)(b * TC_TMEM_COLS) + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0;
#pragma unroll
          for (int h = 0; h < CW / 16; ++h) tmem_ld16(taddr + 16 * h, v + 16 * h);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          if (row < M && nk > 0) {
#pragma unroll
            for (int j = 0; j < CW; ++j) {
              const int col = n0 + c0 + j;
              if (col < N) {
                if constexpr (MODE == TC_F32) {
                  const float a = __uint_as_float(v[j]);
                  const float y = (p.beta == 1.0f) ? (old[j] - a) : fmaf(p.beta, old[j], -a);
                  __stcs(p.C32 + row + (int64_t)col * p.ldc, y);
                  if (p.xs2 != nullptr && row < p.rows2) {
                    __nv_bfloat16 hi, lo;
                    split_bf16(y, hi, lo);
                    __nv_bfloat16 *o = p.xs2 + (int64_t)col * p.ld2 + row;
                    o[0] = hi;
                    if (p.terms2 == 3) {
                      o[p.nb2] = lo;
                      o[2 * p.nb2] = hi;
                    }
                  }
                  if (p.xs3 != nullptr && row >= p.r3 && row < p.r3 + p.rows3) {
                    __nv_bfloat16 x0, x1, x2;
                    split3_bf16(y, x0, x1, x2);
                    __nv_bfloat16 *o = p.xs3 + (int64_t)col * p.ld3 + (row - p.r3);
                    o[0] = x0;
                    o[p.per3] = x1;
                    o[2 * p.per3] = x2;
                  }
                } else {
                  const double x = oz_scale(v[j], ushift + __ldg(p.cexp + col));
                  p.C64[row + (int64_t)col * p.ldc] = p.negate ? old[j] + x : old[j] - x;
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
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TC_TMEM_COLS)
                 : "memory");
  }
}

// 3-D tensor map over BF16 operand slices (K contiguous, rows, slice), one
// box = TC_BK K-values x box_rows rows of one slice, swizzled over its row
// width as the shared-memory descriptor expects.
bool make_slice_map(CUtensorMap *map, const void *base, uint64_t K, uint64_t rows, uint64_t slices,
                    uint32_t box_rows, uint64_t ld, uint64_t sst) {
  PFN_encodeTiled enc = hsma_encode_fn();
  if (enc == nullptr || (uintptr_t)base % 16 != 0 || (ld * 2) % 16 != 0 || (sst * 2) % 16 != 0 || K > ld) return false;
  const cuuint64_t dims[3] = {K, rows, slices};
  const cuuint64_t strides[2] = {ld * 2, sst * 2};
  const cuuint32_t box[3] = {(cuuint32_t)TC_BK, box_rows, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, TC_ROW_BYTES == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Layout of an operand's slice stack in memory: rows, K extent addressable
// from the base (0: the product's K), row stride and slice stride in elements
// (0: dense, ld = K extent, sst = rows * ld).  A view into a larger stack (a
// row and K offset) keeps the stack's strides.
struct SliceLayout {
  int64_t rows = 0, kext = 0, ld = 0, sst = 0;
};

// Launch the persistent product.  A: sa slices of M x K (row-major), B: sb
// slices of N x K; the unit table of a0 names the slice pairs (TC_F32: one
// unit, one pair, filled in here unless given).  One CTA per SM.
template <int MODE>
hsma_status_t tc_gemm(const __nv_bfloat16 *Ap, int sa, const __nv_bfloat16 *Bp, int sb, const TcArgs &a0,
                      const char *phase, cudaStream_t st, SliceLayout la = {}, SliceLayout lb = {}) {
  if (a0.M <= 0 || a0.N <= 0) return HSMA_OK;
  if (a0.K % TC_BK != 0 || a0.K <= 0) return HSMA_ERR_INVALID_ARG;
  static DeviceFlags attr;
  if (!attr.test()) {
    HSMA_CUDA_TRY(
        cudaFuncSetAttribute(tc_gemm_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
    attr.set();
  }
  const int tiles_m = (a0.M + TC_BM - 1) / TC_BM, tiles_n = (a0.N + TC_BN - 1) / TC_BN;
  CUtensorMap ma, mb;
  auto dense = [&](SliceLayout l, int64_t rows) {
    if (l.rows == 0) l.rows = rows;
    if (l.kext == 0) l.kext = a0.K;
    if (l.ld == 0) l.ld = l.kext;
    if (l.sst == 0) l.sst = l.rows * l.ld;
    return l;
  };
  la = dense(la, a0.M);
  lb = dense(lb, a0.N);
  if (la.kext < a0.K || lb.kext < a0.K) return HSMA_ERR_INVALID_ARG;
  if (!make_slice_map(&ma, Ap, (uint64_t)la.kext, (uint64_t)la.rows, (uint64_t)sa, TC_BM, (uint64_t)la.ld,
                      (uint64_t)la.sst) ||
      !make_slice_map(&mb, Bp, (uint64_t)lb.kext, (uint64_t)lb.rows, (uint64_t)sb, TC_BN, (uint64_t)lb.ld,
                      (uint64_t)lb.sst))
    return HSMA_ERR_CUDA;
  TcArgs a = a0;
  if (MODE == TC_F32 && a.nunits == 0) {
    a.nunits = 1;
    a.ubeg[0] = 0;
    a.ubeg[1] = 1;
    a.pa[0] = a.pb[0] = 0;
  }
  if (a.nunits < 1 || a.nunits > kOzMaxUnits) return HSMA_ERR_INVALID_ARG;
  for (int q = 0; q < a.ubeg[a.nunits]; ++q)
    if (a.pa[q] >= sa || a.pb[q] >= sb) return HSMA_ERR_INVALID_ARG;
  a.err = hsma_dev_error_ptr();
  if (a.err == nullptr) return HSMA_ERR_CUDA;
  if (a.limit_ns == 0) a.limit_ns = 4000000000ull;
  static int nsm[64] = {0};
  int dev = 0;
  HSMA_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return HSMA_ERR_UNSUPPORTED;
  if (nsm[dev] == 0) HSMA_CUDA_TRY(cudaDeviceGetAttribute(&nsm[dev], cudaDevAttrMultiProcessorCount, dev));
  const int ntiles = tiles_m * tiles_n;
  a.band = a.K <= 2048 ? 16 : tiles_m;
  const int grid = std::max(1, std::min(ntiles, nsm[dev]));
  HsmaTraceScope ts(phase, st);
  tc_gemm_kernel<MODE><<<grid, 32 * TC_WARPS, TC_SMEM, st>>>(ma, mb, a);
  HSMA_CUDA_TRY(cudaGetLastError());
  return HSMA_OK;
}

}  // namespace
