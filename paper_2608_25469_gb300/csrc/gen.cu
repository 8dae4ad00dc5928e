// Device-side seeded input generator (not part of the solve).
//
// Same definition as the host generator in inputs.py: counter-based
// SplitMix64 (S. Vigna; finaliser of Steele, Lea and Flood, OOPSLA 2014),
//   key(seed, s)    = mix64(seed*G + s*H + G)
//   u64(seed, s, i) = mix64(key + (i+1)*G),   u01 = (u64 >> 11) * 2^-53,
// streams A_RE=0, B_RE=1, A_IM=2, B_IM=3 offset by (inst+1) << 8.
// A (m x m): (2u-1)/m below the diagonal, 1+u on it, 0 above.  B: 2u-1.
// Packed LU factors (kind 2): A's entries below the diagonal; on and above
// it U(i, j) = T(j, i), T drawn like A from streams U_RE=4, U_IM=5.
// Element index is i + j*m (the logical, unpadded column-major index).
#include <cuda_runtime.h>

#include "common.cuh"
#include "gen.h"
#include "trace.h"

namespace {

constexpr uint64_t kG = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kH = 0xD1B54A32D192ED03ull;

__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ uint64_t stream_key(uint64_t seed, uint64_t stream) {
  return mix64(seed * kG + stream * kH + kG);
}

__device__ __forceinline__ double u01(uint64_t key, uint64_t idx) {
  return (double)(mix64(key + (idx + 1) * kG) >> 11) * 0x1.0p-53;
}

__device__ __forceinline__ double a_entry(uint64_t key, int64_t i, int64_t j, int64_t m) {
  if (i < j) return 0.0;
  const double u = u01(key, (uint64_t)(i + j * m));
  if (i == j) return 1.0 + u;
  return __ddiv_rn(2.0 * u - 1.0, (double)m);
}

__global__ void gen_kernel(int cplx_, int kind, uint64_t key_re, uint64_t key_im, uint64_t ukey_re,
                           uint64_t ukey_im, int64_t m, int64_t cols, double *dst, int64_t ld) {
  const int64_t total = m * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % m, j = e / m;
    double re, im = 0.0;
    if (kind == 2 && i <= j) {
      re = a_entry(ukey_re, j, i, m);
      if (cplx_) im = a_entry(ukey_im, j, i, m);
    } else if (kind != 1) {
      re = a_entry(key_re, i, j, m);
      if (cplx_) im = a_entry(key_im, i, j, m);
    } else {
      re = 2.0 * u01(key_re, (uint64_t)e) - 1.0;
      if (cplx_) im = 2.0 * u01(key_im, (uint64_t)e) - 1.0;
    }
    if (cplx_) {
      dst[2 * (i + j * ld)] = re;
      dst[2 * (i + j * ld) + 1] = im;
    } else {
      dst[i + j * ld] = re;
    }
  }
}

}  // namespace

hsma_status_t hsma_gen_launch(int dtype, int kind, uint64_t seed, int64_t inst, int64_t m, int64_t cols, void *dst,
                              int64_t ld, cudaStream_t st) {
  const uint64_t base_re = kind == 1 ? 1 : 0, base_im = kind == 1 ? 3 : 2;
  const uint64_t hi = (uint64_t)(inst + 1) << 8;
  const uint64_t kre = stream_key(seed, base_re + hi), kim = stream_key(seed, base_im + hi);
  const uint64_t ukre = stream_key(seed, 4 + hi), ukim = stream_key(seed, 5 + hi);
  const int64_t total = m * cols;
  if (total == 0) return HSMA_OK;
  static int nsm[64] = {0};
  int dev = 0;
  HSMA_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return HSMA_ERR_UNSUPPORTED;
  if (nsm[dev] == 0) HSMA_CUDA_TRY(cudaDeviceGetAttribute(&nsm[dev], cudaDevAttrMultiProcessorCount, dev));
  int64_t blocks = (total + 255) / 256;
  if (blocks > (int64_t)nsm[dev] * 64) blocks = (int64_t)nsm[dev] * 64;
  gen_kernel<<<(unsigned)blocks, 256, 0, st>>>(dtype == HSMA_C128, kind, kre, kim, ukre, ukim, m, cols,
                                               static_cast<double *>(dst), ld);
  hsma_count_launches(1);
  HSMA_CUDA_TRY(cudaGetLastError());
  return HSMA_OK;
}
