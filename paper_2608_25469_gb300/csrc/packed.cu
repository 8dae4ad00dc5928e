// Column-packed varlen batch of small solves (m <= 64), the paper's
// left / lower / no-transpose case (Section 4.2.1's direct solve, batched).
//
// The FP64 pipe bounds this work, and a warp-wide FP64 instruction costs the
// same whether 1 or 32 of its lanes do useful work.  Solving instance by
// instance leaves lanes idle whenever n is not a multiple of a warp's column
// count, and warps of a CTA idle while the busiest one finishes the instance.
// Here the columns of ALL instances with the same m form one stream: a warp
// takes 32/G consecutive columns of that stream, which may belong to several
// instances, so every warp tile is full except the last one of each m.
//
//  1. schedule (one CTA): validates the instances, groups them by m, orders
//     the groups by the cost of one warp tile (longest first), and writes
//     per position in that order the instance and its first column in the
//     stream (staged triangles lie position by position);
//  2. prep (all SMs, one warp per instance): 1/a_rr, alpha/a_rr and the
//     strict lower triangle with row r pre-multiplied by 1/a_rr, packed by
//     columns into a workspace (the same products the shared-memory staging
//     of the per-instance kernel computes, so results agree bit for bit);
//  3. solve (persistent, independent warps): each warp pulls a tile, finds
//     the instance and column of each of its lanes, keeps its columns of X in
//     registers (lane group g of G lanes holds rows g, g+G, ...) and runs the
//     forward substitution, reading the staged triangles through the L1/L2
//     caches: at this GPU's FP64 rate one 16-byte operand per 64-cycle warp
//     instruction is far below what the caches deliver.
#include <cuda_runtime.h>

#include "common.cuh"
#include "small.h"
#include "trace.h"

namespace {

constexpr int kPkWarps = 4;     // warps per CTA of the solve kernel (independent)
constexpr int kPkMinBlocks = 3;  // resident CTAs per SM (register cap of the solve kernel)

// Index map from the solved lower-triangular form onto the caller's operand
// for the other left-side variants (the per-instance kernel's map): with rev,
// row r of the form is row m-1-r of the operand and of B; with tr, A is read
// transposed; with cj, conjugated.  The identity is the paper's case.
struct PkMap {
  int rev, tr, cj;
};
constexpr int kPkHeaderWords = 8;

// Rows per lane group G of the packed solve: FP64 complex values take four
// registers each, so m > 32 spreads a column over two lanes; every other
// element type keeps whole columns of up to 64 rows in one lane.
template <class T>
__host__ __device__ constexpr bool pk_two_lanes() {
  return sizeof(T) == 16;
}
__host__ __device__ inline int pk_groups(int m, bool two_lanes) { return (two_lanes && m > 32) ? 2 : 1; }
// rows stored per column of a staged triangle: m rounded up to the lane groups
__host__ __device__ inline int pk_rows(int m, int g) { return ((m + g - 1) / g) * g; }
// packed strict-lower triangle of `rows` rows: column i holds rows i+1 .. rows-1
__host__ __device__ inline int64_t pk_col_off(int i, int rows) {
  return (int64_t)i * (rows - 1) - ((int64_t)i * (i - 1)) / 2;
}
__host__ __device__ inline int64_t pk_tri_elems(int rows) { return pk_col_off(rows, rows); }
// staged elements per instance: the triangle, then alpha/a_rr for every row
__host__ __device__ inline int64_t pk_stage_elems(int m, bool two_lanes) {
  const int rows = pk_rows(m, pk_groups(m, two_lanes));
  return pk_tri_elems(rows) + rows;
}

// Scratch layout (bytes, each part 256-aligned):
//   header  int32[8]       [0] next tile, [1] tiles, [2] groups, [3] positions
//   counts  per m (1..64): instances (int32), columns (uint64), and the
//           placement cursor (uint64: instances << 40 | columns); zeroed
//           before every call
//   groups  int32[64][16]  per group of equal m, in schedule order: m, G,
//                          first tile, first position, end position, staged
//                          elements per instance, first stream column
//                          (int64, words 6..7), first staged element (int64,
//                          words 8..9)
//   inst    int32[batch]   instance at each position
//   colpref int64[batch+1] first stream column of each position
//   stage   T[...]         staged triangles, position by position
struct PkLayout {
  size_t counts, groups, inst, colpref, stage, total;
};

struct PkCounts {
  unsigned long long csum[65], cur[65];
  int cnt[65];
};

constexpr int kPkGroupWords = 16;

// Groups in schedule order: m values by decreasing FP64 instructions of one
// warp tile (longest first), computed on the host.
struct PkOrder {
  uint8_t m[64];
};

inline size_t pk_align(size_t v) { return (v + 255) & ~(size_t)255; }

PkLayout pk_layout(int32_t batch, int max_m, int esize, bool two_lanes) {
  PkLayout L;
  const size_t b = (size_t)(batch > 0 ? batch : 0);
  const int mm = (max_m <= 0 || max_m > 64) ? 64 : max_m;
  L.counts = pk_align(sizeof(int32_t) * kPkHeaderWords);
  L.groups = L.counts + pk_align(sizeof(PkCounts));
  L.inst = L.groups + pk_align(sizeof(int32_t) * 64 * kPkGroupWords);
  L.colpref = L.inst + pk_align(sizeof(int32_t) * b);
  L.stage = L.colpref + pk_align(sizeof(int64_t) * (b + 1));
  // every instance's staged size is at most that of an m = max_m instance
  int64_t per = 0;
  for (int m = 1; m <= mm; ++m) per = per > pk_stage_elems(m, two_lanes) ? per : pk_stage_elems(m, two_lanes);
  L.total = L.stage + pk_align((size_t)per * b * (size_t)esize);
  return L;
}

PkOrder pk_order(bool two_lanes, bool cplx_) {
  PkOrder o;
  long long cost[64];
  int n = 0;
  for (int m = 64; m >= 1; --m) {
    const long long c = hsma_small_tile_instr(m, pk_groups(m, two_lanes), cplx_);
    int k = n++;
    while (k > 0 && cost[k - 1] < c) {
      o.m[k] = o.m[k - 1];
      cost[k] = cost[k - 1];
      --k;
    }
    o.m[k] = (uint8_t)m;
    cost[k] = c;
  }
  return o;
}

// ---------------------------------------------------------------------------
// 1. Schedule, in two grid-wide passes over the instances (one instance per
// thread).  Instances with m = 0 or n = 0 are valid and need no work; invalid
// ones set a status bit and are skipped (as the per-instance kernel does).
// An instance above mmax (the caller's bound, which sized the staging
// workspace) counts as invalid, unless skip_large is set: then instances with
// m > 64 are left to the caller (solved elsewhere) without a status bit.
//   count: per m, the instances and their columns (CTA totals in shared
//          memory, then one global atomic per m and CTA);
//   place: every CTA derives the group table from the totals (CTA 0 writes
//          it), gives its instances of each m consecutive slots with one
//          shared 64-bit atomic each (slot in the high bits, first column in
//          the low bits, so stream columns increase with the position), and
//          reserves the CTA's range of each m with one global atomic.
// ---------------------------------------------------------------------------
constexpr int kPkSchedThreads2 = 512;
constexpr int kPkColBits = 40;

__device__ __forceinline__ bool pk_valid(int b, const int32_t *__restrict__ dm, const int32_t *__restrict__ dn,
                                         const int32_t *__restrict__ dlda, const int32_t *__restrict__ dldb,
                                         const void *const *__restrict__ dA, void *const *__restrict__ dB, int mmax,
                                         int skip_large, int &m, int &n, uint32_t &err) {
  m = dm[b];
  n = dn[b];
  const int lda = dlda[b], ldb = dldb[b];
  const bool nul = dA[b] == nullptr || dB[b] == nullptr;
  const int lo = m > 1 ? m : 1;
  if (skip_large && m > 64) return false;
  if (m < 0 || n < 0 || m > mmax || lda < lo || ldb < lo) {
    err |= HSMA_DEVERR_BAD_SIZE;
    return false;
  }
  if (m == 0 || n == 0) return false;
  if (nul) {
    err |= HSMA_DEVERR_NULL_PTR;
    return false;
  }
  return true;
}

template <class T>
__global__ void __launch_bounds__(kPkSchedThreads2) packed_count_kernel(
    int batch, const int32_t *__restrict__ dm, const int32_t *__restrict__ dn, const int32_t *__restrict__ dlda,
    const int32_t *__restrict__ dldb, const void *const *__restrict__ dA, void *const *__restrict__ dB,
    unsigned char *scratch, PkLayout L, int mmax, int skip_large, uint32_t *status) {
  __shared__ int cnt[65];
  __shared__ unsigned long long csum[65];
  PkCounts *g = reinterpret_cast<PkCounts *>(scratch + L.counts);
  for (int k = threadIdx.x; k < 65; k += blockDim.x) {
    cnt[k] = 0;
    csum[k] = 0;
  }
  __syncthreads();
  uint32_t err = 0;
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < batch; b += gridDim.x * blockDim.x) {
    int m, n;
    if (!pk_valid(b, dm, dn, dlda, dldb, dA, dB, mmax, skip_large, m, n, err)) continue;
    atomicAdd(&cnt[m], 1);
    atomicAdd(&csum[m], (unsigned long long)n);
  }
  __syncthreads();
  for (int m = threadIdx.x; m <= 64; m += blockDim.x) {
    if (cnt[m] == 0) continue;
    atomicAdd(&g->cnt[m], cnt[m]);
    atomicAdd(&g->csum[m], csum[m]);
  }
  if (err != 0 && status != nullptr) atomicOr(status, err);
}

template <class T>
__global__ void __launch_bounds__(kPkSchedThreads2) packed_place_kernel(
    int batch, const int32_t *__restrict__ dm, const int32_t *__restrict__ dn, const int32_t *__restrict__ dlda,
    const int32_t *__restrict__ dldb, const void *const *__restrict__ dA, void *const *__restrict__ dB,
    unsigned char *scratch, PkLayout L, int mmax, int skip_large, PkOrder order) {
  constexpr bool two = pk_two_lanes<T>();
  __shared__ int gpos0[65];
  __shared__ long long gcol0[65];
  __shared__ unsigned long long ccur[65], cbase[65], tcsum[65];
  __shared__ int tcnt[65];
  __shared__ int s_over;
  PkCounts *g = reinterpret_cast<PkCounts *>(scratch + L.counts);
  int32_t *hdr = reinterpret_cast<int32_t *>(scratch);
  int32_t *grp = reinterpret_cast<int32_t *>(scratch + L.groups);
  int32_t *inst = reinterpret_cast<int32_t *>(scratch + L.inst);
  int64_t *colpref = reinterpret_cast<int64_t *>(scratch + L.colpref);
  for (int k = threadIdx.x; k < 65; k += blockDim.x) {
    tcnt[k] = g->cnt[k];
    tcsum[k] = g->csum[k];
  }
  __syncthreads();
  // The group table, in schedule order (every CTA derives the same one): the
  // first 64 threads take one schedule slot each and two warp scans give the
  // running positions, tiles, columns and staged elements.
  __shared__ long long wsum[2][4];
  __shared__ int wng[2];
  const int t = threadIdx.x;
  int c = 0, tiles = 0, se = 0, gg = 1, m = 0;
  unsigned long long cs = 0;
  if (t < 64) {
    m = order.m[t];
    c = tcnt[m];
    cs = tcsum[m];
    gg = pk_groups(m, two);
    tiles = c == 0 ? 0 : (int)(gg == 1 ? ((long long)cs + 31) >> 5 : ((long long)cs + 15) >> 4);
    se = (int)pk_stage_elems(m, two);
  }
  const int over_t = (t < 64 && cs >= (1ull << kPkColBits)) ? 1 : 0;
  const int over = __syncthreads_or(over_t);
  long long v[4] = {c, tiles, (long long)cs, (long long)c * se};
  int nz = c != 0 ? 1 : 0;
  const int lane = t & 31, w = t >> 5;
  if (t < 64) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {  // inclusive warp scans
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const long long y = __shfl_up_sync(0xffffffffu, v[q], o);
        if (lane >= o) v[q] += y;
      }
      const int y = __shfl_up_sync(0xffffffffu, nz, o);
      if (lane >= o) nz += y;
    }
    if (lane == 31) {
#pragma unroll
      for (int q = 0; q < 4; ++q) wsum[w][q] = v[q];
      wng[w] = nz;
    }
  }
  __syncthreads();
  if (t < 64) {
    // exclusive prefixes (warp 1 adds warp 0's totals)
    long long ex[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) ex[q] = v[q] - (q == 0 ? c : q == 1 ? tiles : q == 2 ? (long long)cs : (long long)c * se) +
                                        (w == 1 ? wsum[0][q] : 0);
    const int k = nz - (c != 0 ? 1 : 0) + (w == 1 ? wng[0] : 0);  // index among the non-empty groups
    if (c != 0) {
      gpos0[m] = (int)ex[0];
      gcol0[m] = ex[2];
      if (blockIdx.x == 0 && !over) {
        int32_t *e = grp + k * kPkGroupWords;
        e[0] = m;
        e[1] = gg;
        e[2] = (int)ex[1];
        e[3] = (int)ex[0];
        e[4] = (int)ex[0] + c;
        e[5] = se;
        *reinterpret_cast<long long *>(e + 6) = ex[2];
        *reinterpret_cast<long long *>(e + 8) = ex[3];
      }
    }
    if (t == 63 && blockIdx.x == 0) {  // totals; a column count beyond the cursor's low bits: nothing is solved
      const long long pos = v[0] + wsum[0][0], tile = v[1] + wsum[0][1], col = v[2] + wsum[0][2];
      hdr[0] = 0;
      hdr[1] = over ? 0 : (int)tile;
      hdr[2] = over ? 0 : nz + wng[0];
      hdr[3] = over ? 0 : (int)pos;
      colpref[over ? 0 : pos] = over ? 0 : col;
    }
  }
  if (t == 0) s_over = over;
  __syncthreads();
  if (s_over) return;
  uint32_t err = 0;
  const int stride = gridDim.x * blockDim.x;
  for (int b0 = blockIdx.x * blockDim.x; b0 < batch; b0 += stride) {
    for (int k = threadIdx.x; k < 65; k += blockDim.x) ccur[k] = 0;
    __syncthreads();
    const int b = b0 + threadIdx.x;
    int m = 0, n = 0;
    const bool ok = b < batch && pk_valid(b, dm, dn, dlda, dldb, dA, dB, mmax, skip_large, m, n, err);
    unsigned long long mine = 0;
    if (ok) mine = atomicAdd(&ccur[m], (1ull << kPkColBits) + (unsigned long long)n);
    __syncthreads();
    for (int k = threadIdx.x; k <= 64; k += blockDim.x)
      if (ccur[k] != 0) cbase[k] = atomicAdd(&g->cur[k], ccur[k]);
    __syncthreads();
    if (ok) {
      const unsigned long long at = cbase[m] + mine;
      const int p = gpos0[m] + (int)(at >> kPkColBits);
      inst[p] = b;
      colpref[p] = gcol0[m] + (long long)(at & ((1ull << kPkColBits) - 1));
    }
    __syncthreads();  // ccur and cbase are reused by the next chunk
  }
}

// Copy the group table into shared memory (every thread of the CTA).
__device__ __forceinline__ int pk_load_groups(const unsigned char *scratch, const PkLayout &L, int32_t *sgrp) {
  const int32_t *hdr = reinterpret_cast<const int32_t *>(scratch);
  const int32_t *grp = reinterpret_cast<const int32_t *>(scratch + L.groups);
  const int ng = hdr[2];
  for (int k = threadIdx.x; k < ng * kPkGroupWords; k += blockDim.x) sgrp[k] = grp[k];
  __syncthreads();
  return ng;
}

// ---------------------------------------------------------------------------
// 2. Prep: one warp per position.  The reciprocals of the diagonal go to a
// per-warp shared row table; then the lanes walk the packed triangle element
// by element (consecutive elements in consecutive lanes), so every lane of
// every FP64 instruction produces a staged value.
// ---------------------------------------------------------------------------
constexpr int kPkPrepWarps = 8;

template <class T, bool MAP>
__global__ void __launch_bounds__(32 * kPkPrepWarps) packed_prep_kernel(const int32_t *__restrict__ dm,
                                                                       const void *const *__restrict__ dA,
                                                                       const int32_t *__restrict__ dlda,
                                                                       const unsigned char *__restrict__ scratch,
                                                                       PkLayout L, T *stage, T alpha, int unit,
                                                                       int a_packed, PkMap mp) {
  using E = Elem<T>;
  __shared__ __align__(16) int32_t sgrp[64 * kPkGroupWords];
  __shared__ T sR[kPkPrepWarps][64];
  const int ng = pk_load_groups(scratch, L, sgrp);
  const int32_t *hdr = reinterpret_cast<const int32_t *>(scratch);
  const int32_t *inst = reinterpret_cast<const int32_t *>(scratch + L.inst);
  const int np = hdr[3];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int wid = blockIdx.x * kPkPrepWarps + w, nw = gridDim.x * kPkPrepWarps;
  T *rinv = sR[w];
  int k = 0;
  for (int p = wid; p < np; p += nw) {
    while (k + 1 < ng && sgrp[(k + 1) * kPkGroupWords + 3] <= p) ++k;  // positions only grow
    const int32_t *e = sgrp + k * kPkGroupWords;
    const int m = e[0], rows = pk_rows(m, e[1]);
    const int64_t off = *reinterpret_cast<const long long *>(e + 8) + (int64_t)(p - e[3]) * e[5];
    const int b = inst[p];
    const T *A = static_cast<const T *>(dA[b]);
    const int64_t lda = dlda[b];
    // element (r, c), r >= c, of the lower-triangular form: from the operand
    // through the index map (column-major with lda), or (a_packed, identity
    // map only) LAPACK's packed lower storage, column c holding rows c .. m-1
    // from c (2m - c + 1) / 2
    auto at = [&](int r, int c) -> T {
      if (a_packed) return E::ld(A + (int64_t)c * (2 * m - c + 1) / 2 + (r - c));
      if constexpr (!MAP) return E::ld(A + r + (int64_t)c * lda);
      int pr = mp.rev ? m - 1 - r : r, pc = mp.rev ? m - 1 - c : c;
      if (mp.tr) {
        const int t = pr;
        pr = pc;
        pc = t;
      }
      T v = E::ld(A + pr + (int64_t)pc * lda);
      if constexpr (E::kComplex) {
        if (mp.cj) v.im = -v.im;
      }
      return v;
    };
    T *tri = stage + off;
    T *sc = tri + pk_tri_elems(rows);
    __syncwarp();
    for (int r = lane; r < rows; r += 32) {  // warp-uniform trip count per 32 rows
      T rv = E::one();
      if (r < m && !unit) rv = E::recip(at(r, r));
      rinv[r] = rv;
      sc[r] = r < m ? E::mul(alpha, rv) : E::zero();
    }
    __syncwarp();
    // element q of the packed triangle: column i, row i + 1 + local index;
    // eight elements per lane in flight (loads first)
    const int total = (int)pk_tri_elems(rows);
    int i = 0, loc = lane;
    auto advance = [&](int by) {
      loc += by;
      while (i < rows - 1 && loc >= rows - 1 - i) {
        loc -= rows - 1 - i;
        ++i;
      }
    };
    advance(0);
    for (int q0 = 0; q0 < total; q0 += 8 * 32) {
      int rr[8];
      T vv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int q = q0 + u * 32 + lane;
        rr[u] = i + 1 + loc;
        vv[u] = (q < total && rr[u] < m) ? at(rr[u], i) : E::zero();
        advance(32);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int q = q0 + u * 32 + lane;
        if (q < total) tri[q] = E::mul(rinv[rr[u]], vv[u]);
      }
    }
  }
}

// Staged values are 16-byte aligned: complex128 is read as one vector.
template <class T>
__device__ __forceinline__ T pk_ld(const T *p) {
  return Elem<T>::ld(p);
}
template <>
__device__ __forceinline__ cplx pk_ld<cplx>(const cplx *p) {
  const double2 v = __ldg(reinterpret_cast<const double2 *>(p));
  return cplx{v.x, v.y};
}

// ---------------------------------------------------------------------------
// 3. Solve.  A warp tile: C = 32/G columns of one m's stream; lane l holds
// column c = l / G of the tile, rows g + t*G (g = l % G) in register slot t.
// ---------------------------------------------------------------------------
template <class T, int G, int MMAX, bool REV, int KS>
__device__ __forceinline__ void packed_tile(const T *tri, const T *sc, T *Bp, bool active, int m, int rows,
                                            bool azero) {
  using E = Elem<T>;
  constexpr int R = MMAX / G;
  const int lane = threadIdx.x & 31;
  const int g = lane % G, c = lane / G;
  // row r = g + t G of the form is row r of B, or (REV) row m - 1 - r: one
  // base per lane and a compile-time step per slot t
  T *const Bg = REV ? Bp + (m - 1 - g) : Bp + g;
  constexpr int kStep = REV ? -G : G;
  if (azero) {
#pragma unroll
    for (int t = 0; t < R; ++t) {
      const int r = g + t * G;
      if (t * G < m && active && r < m) E::st(Bg + t * kStep, E::zero());
    }
    return;
  }
  T s[R];
#pragma unroll
  for (int t = 0; t < R; ++t) {
    const int r = g + t * G;
    s[t] = E::zero();
    if (t * G < m) {
      if (active && r < m) s[t] = E::mul(pk_ld(sc + r), E::ld(Bg + t * kStep));
    }
  }
  // slots below KS hold rows below m for every m the caller sends to this
  // form (KS G < m), so their loads need no run-time bound check and the
  // compiler may issue them together
  int64_t base = -1;  // column i of the staged triangle starts at tri + base + i + 1
#pragma unroll
  for (int i = 0; i < MMAX - 1; ++i) {
    if (i >= m - 1) break;  // warp-uniform: the last row updates nothing
    const int tb = i / G, gi = i % G;
    const T x = (G == 1) ? s[tb] : E::shfl(s[tb], c * G + gi);
    const T *col = tri + base;
    if (G > 1 && gi < G - 1) {
      // boundary slot: only rows strictly below i update
      const int r = g + tb * G;
      const int ra = r > i ? r : i + 1;
      const T ns = E::fms(pk_ld(col + ra), x, s[tb]);
      if (r > i) s[tb] = ns;
    }
#pragma unroll
    for (int t = tb + 1; t < R; ++t) {
      if (t >= KS && t * G >= m) break;  // warp-uniform
      s[t] = E::fms(pk_ld(col + g + t * G), x, s[t]);
    }
    base += rows - 2 - i;
  }
#pragma unroll
  for (int t = 0; t < R; ++t) {
    const int r = g + t * G;
    if (t * G < m) {
      if (active && r < m) E::st(Bg + t * kStep, s[t]);
    }
  }
}

template <class T, bool REV>
__global__ void __launch_bounds__(32 * kPkWarps, kPkMinBlocks) packed_solve_kernel(
    void *const *__restrict__ dB, const int32_t *__restrict__ dldb, unsigned char *scratch, PkLayout L,
    const T *__restrict__ stage, int azero) {
  constexpr bool two = pk_two_lanes<T>();
  __shared__ __align__(16) int32_t sgrp[64 * kPkGroupWords];
  int32_t *hdr = reinterpret_cast<int32_t *>(scratch);
  const int32_t *inst = reinterpret_cast<const int32_t *>(scratch + L.inst);
  const int64_t *colpref = reinterpret_cast<const int64_t *>(scratch + L.colpref);
  const int ng = pk_load_groups(scratch, L, sgrp);
  const int ntiles = *(volatile const int32_t *)(hdr + 1);
  const int lane = threadIdx.x & 31;
  for (;;) {
    int tile = 0;
    if (lane == 0) tile = atomicAdd(hdr, 1);
    tile = __shfl_sync(0xffffffffu, tile, 0);
    if (tile >= ntiles) break;
    int k = 0;
    while (k + 1 < ng && sgrp[(k + 1) * kPkGroupWords + 2] <= tile) ++k;  // warp-uniform
    const int32_t *e = sgrp + k * kPkGroupWords;
    const int m = e[0], G = e[1], pos0 = e[3], pos1 = e[4];
    const long long col0 = *reinterpret_cast<const long long *>(e + 6);
    const long long colend = colpref[pos1];
    const int C = 32 / G;
    const long long gc = col0 + (long long)(tile - e[2]) * C + lane / G;
    const bool active = gc < colend;
    // position of the lane's instance: last p in [pos0, pos1) with colpref[p] <= gc
    int p = pos0;
    if (active) {
      int lo = pos0, hi = pos1 - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (colpref[mid] <= gc) lo = mid;
        else hi = mid - 1;
      }
      p = lo;
    }
    const int p_lane0 = __shfl_sync(0xffffffffu, p, 0);  // lane 0 is always active
    if (!active) p = p_lane0;
    const int b = inst[p];
    const long long j = active ? gc - colpref[p] : 0;
    T *Bp = static_cast<T *>(dB[b]) + j * (int64_t)dldb[b];
    const int rows = pk_rows(m, G);
    const T *tri = stage + *reinterpret_cast<const long long *>(e + 8) + (int64_t)(p - pos0) * e[5];
    const T *sc = tri + pk_tri_elems(rows);
    if constexpr (two) {
      // the bound-check-free slot prefix by m: KS slots with KS G < m
      if (G == 1) {
        if (m > 8)
          packed_tile<T, 1, 32, REV, 9>(tri, sc, Bp, active, m, rows, azero != 0);
        else
          packed_tile<T, 1, 32, REV, 1>(tri, sc, Bp, active, m, rows, azero != 0);
      } else {
        packed_tile<T, 2, 64, REV, 17>(tri, sc, Bp, active, m, rows, azero != 0);
      }
    } else {
      packed_tile<T, 1, 64, REV, 1>(tri, sc, Bp, active, m, rows, azero != 0);
    }
  }
}

template <class T, bool REV>
int packed_grid(int dev) {
  static int cached[64] = {0};
  if (dev >= 0 && dev < 64 && cached[dev] > 0) return cached[dev];
  int nsm = 0, per_sm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, packed_solve_kernel<T, REV>, 32 * kPkWarps, 0);
  const int grid = nsm * (per_sm > 0 ? per_sm : 1);
  if (dev >= 0 && dev < 64) cached[dev] = grid;
  return grid;
}

int sm_count(int dev) {
  static int cached[64] = {0};
  if (dev >= 0 && dev < 64 && cached[dev] > 0) return cached[dev];
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (dev >= 0 && dev < 64) cached[dev] = nsm;
  return nsm;
}

template <class T>
hsma_status_t packed_impl(int32_t batch, int max_m, const int32_t *dm, const int32_t *dn, const double *alpha,
                          const void *const *dA, const int32_t *dlda, void *const *dB, const int32_t *dldb, int unit,
                          uint32_t *status, void *scratch, cudaStream_t st, int a_packed, PkMap mp) {
  int dev = 0;
  HSMA_CUDA_TRY(cudaGetDevice(&dev));
  const PkLayout L = pk_layout(batch, max_m, (int)sizeof(T), pk_two_lanes<T>());
  unsigned char *scr = static_cast<unsigned char *>(scratch);
  T *stage = reinterpret_cast<T *>(scr + L.stage);
  const T al = hsma_alpha_as<T>(alpha);
  const bool azero = Elem<T>::kComplex ? (alpha[0] == 0.0 && alpha[1] == 0.0) : alpha[0] == 0.0;
  {
    static const PkOrder order = pk_order(pk_two_lanes<T>(), Elem<T>::kComplex);
    const int mmax = (max_m <= 0 || max_m > 64) ? 64 : max_m;
    const int skip_large = max_m > 64 ? 1 : 0;
    const int nsm = sm_count(dev);
    int blocks = (batch + kPkSchedThreads2 - 1) / kPkSchedThreads2;
    if (blocks > 4 * nsm) blocks = 4 * nsm;
    HsmaTraceScope ts("vbatched_schedule", st, 2);
    HSMA_CUDA_TRY(cudaMemsetAsync(scr + L.counts, 0, sizeof(PkCounts), st));
    packed_count_kernel<T><<<blocks, kPkSchedThreads2, 0, st>>>(batch, dm, dn, dlda, dldb, dA, dB, scr, L, mmax,
                                                                skip_large, status);
    packed_place_kernel<T><<<blocks, kPkSchedThreads2, 0, st>>>(batch, dm, dn, dlda, dldb, dA, dB, scr, L, mmax,
                                                                skip_large, order);
  }
  HSMA_CUDA_TRY(cudaGetLastError());
  if (!azero) {
    // one warp per instance, up to 32 warps per SM over the whole GPU
    const int nsm = sm_count(dev);
    int blocks = (batch + kPkPrepWarps - 1) / kPkPrepWarps;
    if (blocks > 4 * nsm) blocks = 4 * nsm;
    HsmaTraceScope ts("vbatched_prep", st);
    const bool mapped = mp.rev || mp.tr || mp.cj;
    if (mapped)
      packed_prep_kernel<T, true><<<blocks, 32 * kPkPrepWarps, 0, st>>>(dm, dA, dlda, scr, L, stage, al, unit,
                                                                        a_packed, mp);
    else
      packed_prep_kernel<T, false><<<blocks, 32 * kPkPrepWarps, 0, st>>>(dm, dA, dlda, scr, L, stage, al, unit,
                                                                         a_packed, mp);
    HSMA_CUDA_TRY(cudaGetLastError());
  }
  {
    HsmaTraceScope ts("vbatched_solve", st);
    if (mp.rev)
      packed_solve_kernel<T, true><<<packed_grid<T, true>(dev), 32 * kPkWarps, 0, st>>>(dB, dldb, scr, L, stage,
                                                                                     azero ? 1 : 0);
    else
      packed_solve_kernel<T, false><<<packed_grid<T, false>(dev), 32 * kPkWarps, 0, st>>>(dB, dldb, scr, L, stage,
                                                                                       azero ? 1 : 0);
  }
  HSMA_CUDA_TRY(cudaGetLastError());
  return HSMA_OK;
}

}  // namespace

size_t hsma_vbatched_packed_scratch_bytes(int dtype, int32_t batch, int32_t max_m) {
  const int es = hsma_small_esize(dtype);
  return pk_layout(batch, max_m, es, es == 16).total;
}

hsma_status_t hsma_small_vbatched_packed(int dtype, int32_t batch, int32_t max_m, const int32_t *dm,
                                         const int32_t *dn, const double *alpha, const void *const *dA,
                                         const int32_t *dlda, void *const *dB, const int32_t *dldb, int unit,
                                         uint32_t *status, void *scratch, cudaStream_t st, int a_packed, int uplo,
                                         int trans) {
  // the per-instance kernel's map: an upper operand (after op) is solved with
  // its rows and columns reversed
  const bool op_lower = (uplo == HSMA_LOWER) != (trans != HSMA_NO_TRANS);
  const PkMap mp{op_lower ? 0 : 1, trans != HSMA_NO_TRANS ? 1 : 0, trans == HSMA_CONJ_TRANS ? 1 : 0};
  if (a_packed && (mp.rev || mp.tr)) return HSMA_ERR_UNSUPPORTED;
  switch (dtype) {
    case HSMA_C128:
      return packed_impl<cplx>(batch, max_m, dm, dn, alpha, dA, dlda, dB, dldb, unit, status, scratch, st,
                               a_packed, mp);
    default:
      return HSMA_ERR_UNSUPPORTED;
  }
}
