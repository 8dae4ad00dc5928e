// Internal helpers shared by the CUDA translation units of the library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/hsma.h"

#define HSMA_CUDA_TRY(expr)                                  \
  do {                                                       \
    cudaError_t hsma_e_ = (expr);                            \
    if (hsma_e_ != cudaSuccess) return hsma_from_cuda(hsma_e_); \
  } while (0)

static inline hsma_status_t hsma_from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return HSMA_OK;
  if (e == cudaErrorMemoryAllocation) return HSMA_ERR_NO_MEMORY;
  return HSMA_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// Element types.  `cplx` is the interleaved (re, im) layout of complex128,
// `cplxf` that of complex64.
// ---------------------------------------------------------------------------
struct cplx {
  double re, im;
};

struct __align__(8) cplxf {
  float re, im;
};

template <class T>
struct Elem;

template <>
struct Elem<double> {
  static constexpr bool kComplex = false;
  static constexpr int kFlopsPerFma = 1;  // DFMA instructions per multiply-add
  __device__ __forceinline__ static double zero() { return 0.0; }
  __device__ __forceinline__ static double one() { return 1.0; }
  __device__ __forceinline__ static double mul(double a, double b) { return a * b; }
  // s - a*x, one fused multiply-add
  __device__ __forceinline__ static double fms(double a, double x, double s) { return fma(-a, x, s); }
  __device__ __forceinline__ static double recip(double a) { return 1.0 / a; }
  __device__ __forceinline__ static double shfl(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }
  __device__ __forceinline__ static double ld(const double *p) { return __ldg(p); }
  __device__ __forceinline__ static void st(double *p, double v) { *p = v; }
  __device__ __forceinline__ static bool is_zero(double a) { return a == 0.0; }
};

template <>
struct Elem<float> {
  static constexpr bool kComplex = false;
  static constexpr int kFlopsPerFma = 1;
  __device__ __forceinline__ static float zero() { return 0.0f; }
  __device__ __forceinline__ static float one() { return 1.0f; }
  __device__ __forceinline__ static float mul(float a, float b) { return a * b; }
  __device__ __forceinline__ static float fms(float a, float x, float s) { return fmaf(-a, x, s); }
  __device__ __forceinline__ static float recip(float a) { return 1.0f / a; }
  __device__ __forceinline__ static float shfl(float v, int src) { return __shfl_sync(0xffffffffu, v, src); }
  __device__ __forceinline__ static float ld(const float *p) { return __ldg(p); }
  __device__ __forceinline__ static void st(float *p, float v) { *p = v; }
  __device__ __forceinline__ static bool is_zero(float a) { return a == 0.0f; }
};

template <>
struct Elem<cplx> {
  static constexpr bool kComplex = true;
  static constexpr int kFlopsPerFma = 4;
  __device__ __forceinline__ static cplx zero() { return cplx{0.0, 0.0}; }
  __device__ __forceinline__ static cplx one() { return cplx{1.0, 0.0}; }
  __device__ __forceinline__ static cplx mul(cplx a, cplx b) {
    cplx r;
    r.re = fma(a.re, b.re, -(a.im * b.im));
    r.im = fma(a.re, b.im, a.im * b.re);
    return r;
  }
  // s - a*x with four fused multiply-adds
  __device__ __forceinline__ static cplx fms(cplx a, cplx x, cplx s) {
    s.re = fma(-a.re, x.re, s.re);
    s.re = fma(a.im, x.im, s.re);
    s.im = fma(-a.re, x.im, s.im);
    s.im = fma(-a.im, x.re, s.im);
    return s;
  }
  // 1/a, scaled by the larger component of a (Smith's algorithm with numerator
  // 1), with two divisions: t/d is taken as t (1/d), one rounding more than a
  // third division (relative error below 2 ulps instead of 1).  Written with
  // selects rather than a branch: lanes of a warp that take different branches
  // would otherwise run both branches' divisions.
  //   |re| >= |im|: t = im/re, d = re + im t, 1/a = (1/d, -t/d)
  //   otherwise:    t = re/im, d = re t + im, 1/a = (t/d, -1/d)
  __device__ __forceinline__ static cplx recip(cplx a) {
    const bool big = fabs(a.re) >= fabs(a.im);
    const double p = big ? a.re : a.im, q = big ? a.im : a.re;  // larger, smaller
    const double t = q / p;
    const double d = fma(q, t, p);
    const double u = 1.0 / d, v = t * u;
    return big ? cplx{u, -v} : cplx{v, -u};
  }
  __device__ __forceinline__ static cplx shfl(cplx v, int src) {
    cplx r;
    r.re = __shfl_sync(0xffffffffu, v.re, src);
    r.im = __shfl_sync(0xffffffffu, v.im, src);
    return r;
  }
  __device__ __forceinline__ static cplx ld(const cplx *p) {
    const double *q = reinterpret_cast<const double *>(p);
    return cplx{__ldg(q), __ldg(q + 1)};
  }
  __device__ __forceinline__ static void st(cplx *p, cplx v) {
    double *q = reinterpret_cast<double *>(p);
    q[0] = v.re;
    q[1] = v.im;
  }
  __device__ __forceinline__ static bool is_zero(cplx a) { return a.re == 0.0 && a.im == 0.0; }
};

template <>
struct Elem<cplxf> {
  static constexpr bool kComplex = true;
  static constexpr int kFlopsPerFma = 4;
  __device__ __forceinline__ static cplxf zero() { return cplxf{0.0f, 0.0f}; }
  __device__ __forceinline__ static cplxf one() { return cplxf{1.0f, 0.0f}; }
  __device__ __forceinline__ static cplxf mul(cplxf a, cplxf b) {
    cplxf r;
    r.re = fmaf(a.re, b.re, -(a.im * b.im));
    r.im = fmaf(a.re, b.im, a.im * b.re);
    return r;
  }
  __device__ __forceinline__ static cplxf fms(cplxf a, cplxf x, cplxf s) {
    s.re = fmaf(-a.re, x.re, s.re);
    s.re = fmaf(a.im, x.im, s.re);
    s.im = fmaf(-a.re, x.im, s.im);
    s.im = fmaf(-a.im, x.re, s.im);
    return s;
  }
  // Smith's algorithm with numerator 1 (selects, two divisions, as for cplx)
  __device__ __forceinline__ static cplxf recip(cplxf a) {
    const bool big = fabsf(a.re) >= fabsf(a.im);
    const float p = big ? a.re : a.im, q = big ? a.im : a.re;
    const float t = q / p;
    const float d = fmaf(q, t, p);
    const float u = 1.0f / d, v = t * u;
    return big ? cplxf{u, -v} : cplxf{v, -u};
  }
  __device__ __forceinline__ static cplxf shfl(cplxf v, int src) {
    return cplxf{__shfl_sync(0xffffffffu, v.re, src), __shfl_sync(0xffffffffu, v.im, src)};
  }
  __device__ __forceinline__ static cplxf ld(const cplxf *p) {
    const float2 v = __ldg(reinterpret_cast<const float2 *>(p));
    return cplxf{v.x, v.y};
  }
  __device__ __forceinline__ static void st(cplxf *p, cplxf v) {
    *reinterpret_cast<float2 *>(p) = make_float2(v.re, v.im);
  }
  __device__ __forceinline__ static bool is_zero(cplxf a) { return a.re == 0.0f && a.im == 0.0f; }
};

// alpha (host double, or double[2] for complex) in the element type
template <class T>
inline T hsma_alpha_as(const double *a);
template <>
inline double hsma_alpha_as<double>(const double *a) { return a[0]; }
template <>
inline float hsma_alpha_as<float>(const double *a) { return (float)a[0]; }
template <>
inline cplx hsma_alpha_as<cplx>(const double *a) { return cplx{a[0], a[1]}; }
template <>
inline cplxf hsma_alpha_as<cplxf>(const double *a) { return cplxf{(float)a[0], (float)a[1]}; }

// ---------------------------------------------------------------------------
// Element loops over a rows x cols column-major block without integer
// division: blockIdx.y strides the columns, blockIdx.x and the threads the
// rows.  hsma_grid_rc gives the matching launch grid (256 threads).
// ---------------------------------------------------------------------------
#define HSMA_FOR_RC(i, j, rows, cols)                                                       \
  for (int64_t j = blockIdx.y; j < (int64_t)(cols); j += gridDim.y)                         \
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)(rows); \
         i += (int64_t)gridDim.x * blockDim.x)

inline dim3 hsma_grid_rc(int64_t rows, int64_t cols) {
  // about 16 CTAs of 256 threads per SM in total; the loops stride the rest
  int64_t bx = (rows + 255) / 256;
  bx = bx < 1 ? 1 : (bx > 64 ? 64 : bx);
  const int64_t cap = 2432 / bx;
  int64_t by = cols < cap ? cols : cap;
  by = by < 1 ? 1 : by;
  return dim3((unsigned)bx, (unsigned)by);
}

// ---------------------------------------------------------------------------
// Small-path cost model (Section 4.2 kernel as laid out on this GPU).
//
// A warp holds C = 32/G columns of X; each column's rows are spread over G
// lanes (row r lives in lane group r % G, register slot r / G).  FP64 lanes
// that are masked off still occupy the FP64 pipe, so the cost of a solve is
// the number of warp-wide FP64 instructions it issues:
//   per column tile: K * ( R + sum_{i=0}^{m-2} (R - floor((i+1)/G)) ),
//   R = ceil(m/G) register slots, K = FP64 instructions per multiply-add
//   (1 real, 4 complex); the first R term is the alpha*diag^{-1} scaling.
// Staging the scaled triangle costs K * sum_i ceil((R*G - 1 - i)/32) per CTA.
// ---------------------------------------------------------------------------
// Rows a complex warp holds with G = 1 (two registers per value): 32 keeps the
// batched kernel at three CTAs per SM.
#ifndef HSMA_CPLX_G1_MMAX
#define HSMA_CPLX_G1_MMAX 32
#endif
__host__ __device__ inline int hsma_small_rmax(int g, bool cplx_) {
  // register slots available per lane: 64 rows for any G, except complex G=1
  // which is limited to 32 rows (128 registers of X per lane)
  return (cplx_ && g == 1) ? HSMA_CPLX_G1_MMAX : 64 / g;
}

__host__ __device__ inline bool hsma_small_g_ok(int g, int m, bool cplx_) {
  return m <= hsma_small_rmax(g, cplx_) * g;
}

// closed form of sum_{k=1}^{N} floor(k/g)
__host__ __device__ inline long long hsma_sum_floor(long long N, long long g) {
  if (N <= 0) return 0;
  const long long q = N / g, r = N % g;
  return g * q * (q - 1) / 2 + q * (r + 1);
}

// closed form of sum_{v=0}^{V} ceil(v/32)  (0 for V < 0)
__host__ __device__ inline long long hsma_sum_ceil32(long long V) {
  if (V <= 0) return 0;
  const long long a = V / 32, b = V % 32;
  return 32 * a * (a + 1) / 2 + (a + 1) * b;
}

__host__ __device__ inline long long hsma_small_tile_instr(int m, int g, bool cplx_) {
  const long long K = cplx_ ? 4 : 1;
  const long long R = (m + g - 1) / g;
  return K * (R + (long long)(m - 1) * R - hsma_sum_floor(m - 1, g));
}

__host__ __device__ inline long long hsma_small_stage_instr(int m, int g, bool cplx_) {
  const long long K = cplx_ ? 4 : 1;
  const long long RG = (long long)((m + g - 1) / g) * g;
  return K * (hsma_sum_ceil32(RG - 1) - hsma_sum_ceil32(RG - m - 1));
}

// FP64 warp instructions issued for one (m, n) solve with row groups g
__host__ __device__ inline long long hsma_small_total_instr(int m, int n, int g, bool cplx_) {
  const int C = 32 / g;
  const long long tiles = (n + C - 1) / C;
  return tiles * hsma_small_tile_instr(m, g, cplx_) + hsma_small_stage_instr(m, g, cplx_);
}

// As above, but with the tiles dealt round-robin to the W warps of a CTA that
// share one staged triangle: the CTA holds its warps until the busiest is done.
__host__ __device__ inline long long hsma_small_cta_instr(int m, int n, int g, bool cplx_, int W) {
  const int C = 32 / g;
  const long long tiles = (n + C - 1) / C;
  const long long rounds = (tiles + W - 1) / W;
  return rounds * W * hsma_small_tile_instr(m, g, cplx_) + hsma_small_stage_instr(m, g, cplx_);
}

// Row-group choice of the batched kernel: the allowed set is a bit mask
// (bit log2(G)), the cost the CTA-level one above.
__host__ __device__ inline int hsma_small_pick_g_batched(int m, int n, bool cplx_, int W, unsigned gmask) {
  int best = 0;
  long long bc = 0;
  for (int lg = 0; lg < 6; ++lg) {
    const int g = 1 << lg;
    if (!(gmask & (1u << lg)) || !hsma_small_g_ok(g, m, cplx_)) continue;
    const long long c = hsma_small_cta_instr(m, n, g, cplx_, W);
    if (best == 0 || c < bc) {
      best = g;
      bc = c;
    }
  }
  return best;
}

// Device constants of this GPU's FP64 pipe used by the latency-aware choice
// for a single solve: a warp-wide FP64 instruction occupies a sub-partition
// for 64 cycles; a dependent step costs one FP64 latency plus, for G > 1, a
// shuffle round trip.
__host__ __device__ inline double hsma_small_time_model(int m, int n, int g, bool cplx_, int nsm) {
  const double tile = (double)hsma_small_tile_instr(m, g, cplx_);
  const int C = 32 / g;
  const int tiles = (n + C - 1) / C;
  const double stage = (double)hsma_small_stage_instr(m, g, cplx_);
  // every CTA (four warps) stages the triangle once
  const double total = tiles * tile + stage * ((tiles + 3) / 4);
  // whole-GPU pipe: 4 sub-partitions per SM, ~84% of nominal measured
  const double tput = total * 64.0 / (4.0 * nsm * 0.84);
  // one warp alone on its sub-partition, with staging split over four warps
  const double warp = (tile + 0.25 * stage) * 64.0;
  // dependent chain: per step one multiply-add latency (two for complex) plus a shuffle
  const double chain = (m - 1) * ((cplx_ ? 128.0 : 64.0) + (g > 1 ? 40.0 : 0.0));
  const double busy = tput > warp ? tput : warp;
  return busy > chain ? busy : chain;
}

__host__ __device__ inline int hsma_small_pick_g_single(int m, int n, bool cplx_, int nsm) {
  const int cands[6] = {1, 2, 4, 8, 16, 32};
  int best = 0;
  double bc = 0.0;
  for (int k = 0; k < 6; ++k) {
    const int g = cands[k];
    if (!hsma_small_g_ok(g, m, cplx_)) continue;
    const double c = hsma_small_time_model(m, n, g, cplx_, nsm);
    if (best == 0 || c < bc) {
      best = g;
      bc = c;
    }
  }
  return best;
}

// One flag per device (e.g. "kernel attribute already set on this device").
struct DeviceFlags {
  static constexpr int kMax = 64;
  volatile int flag[kMax] = {0};
  bool test() const {
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= kMax) return false;
    return flag[d] != 0;
  }
  void set() {
    int d = 0;
    if (cudaGetDevice(&d) == cudaSuccess && d >= 0 && d < kMax) flag[d] = 1;
  }
};
