// FP32 inverses of the N_B x N_B diagonal blocks for the FP32-result solve
// (phase 1 of the blocked algorithm, Section 4.3, in the reduced-precision
// mode the paper leaves to future work, Section 6), by doubling.
//
// Inverting a 512-row block by substitution is a 512-step dependent chain.
// Here the substitution kernel inverts 64 x 64 blocks only (a 64-step chain),
// and each level joins adjacent h x h inverses into a 2h x 2h one: for
//   T = [A 0; C D],   T^-1 = [A^-1 0; -D^-1 C A^-1  D^-1],
// the new lower-left block takes two FP32 products, W = C A^-1 and then
// -D^-1 W, for every pair of the level in one launch each (levels h = 64,
// 128, ..., N_B / 2).  The operands are the triangular inverses already in
// place (zeros above their diagonals) and the strictly lower block C of the
// matrix, so the matrix's upper triangle and its diagonal (unit case) are not
// read here.
#include <cuda_runtime.h>

#include <algorithm>

#include "blocked.h"
#include "common.cuh"
#include "mixed.h"
#include "trace.h"
#include "workspace.h"

namespace {

constexpr int kInvBase = 64;  // blocks inverted by substitution
constexpr int kDT = 64;       // output tile of the doubling products
constexpr int kDK = 16;       // K step

// Copy the inverse of base block b (64 x 64, contiguous) onto the diagonal of
// its N_B-row outer block (ld N_B): one CTA per base block.
__global__ void __launch_bounds__(256) inv_place_kernel(const float *__restrict__ base, int64_t m, int nb,
                                                        float *Dinv) {
  const int64_t b = blockIdx.x, r0 = b * kInvBase;
  const int s = (int)std::min<int64_t>(kInvBase, m - r0);
  const int64_t R = r0 / nb;
  const int l = (int)(r0 % nb);
  float *Y = Dinv + R * nb * nb;
  const float *src = base + b * kInvBase * kInvBase;
  for (int e = threadIdx.x; e < kInvBase * kInvBase; e += blockDim.x) {
    const int i = e % kInvBase, j = e / kInvBase;
    if (i < s && j < s) Y[(l + i) + (int64_t)(l + j) * nb] = src[i + j * kInvBase];
  }
}

// One 64 x 64 output tile of out = sign * P Q (P: M x K, Q: K x N, all
// column-major), zero outside the sizes, over the K range [kb, ke) (the
// terms outside it are known zeros of a triangular operand).  256 threads,
// 4 x 4 outputs each.
__device__ __forceinline__ void tile_product(const float *__restrict__ P, int64_t ldp, const float *__restrict__ Q,
                                             int64_t ldq, float *out, int64_t ldo, int M, int N, int K, int r0,
                                             int c0, float sign, int kb, int ke) {
  __shared__ __align__(16) float sP[kDK][kDT];
  __shared__ __align__(16) float sQ[kDK][kDT];
  const int t = threadIdx.x;
  const int tx = t % 16, ty = t / 16;
  const int pk = t / 16, pi = (t % 16) * 4;  // P loader: k, 4 rows
  const int qj = t / 4, qk = (t % 4) * 4;    // Q loader: column, 4 k
  float acc[4][4] = {};
  ke = ke < K ? ke : K;
  for (int k0 = kb; k0 < ke; k0 += kDK) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = r0 + pi + u, k = k0 + pk;
      sP[pk][pi + u] = (i < M && k < ke) ? P[i + (int64_t)k * ldp] : 0.0f;
      const int kq = k0 + qk + u, j = c0 + qj;
      sQ[qk + u][qj] = (kq < ke && j < N) ? Q[kq + (int64_t)j * ldq] : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kDK; ++kk) {
      const float4 a = *reinterpret_cast<const float4 *>(&sP[kk][tx * 4]);
      const float4 b = *reinterpret_cast<const float4 *>(&sQ[kk][ty * 4]);
      const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(av[x], bv[y], acc[x][y]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int y = 0; y < 4; ++y) {
    const int j = c0 + ty * 4 + y;
    if (j >= N) continue;
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      const int i = r0 + tx * 4 + x;
      if (i < M) out[i + (int64_t)j * ldo] = sign * acc[x][y];
    }
  }
}

// Level h of the doubling.  blockIdx.y = pair p (rows i0 = 2hp .. of the
// matrix, inside outer block i0 / N_B), blockIdx.x = output tile.  Pass 0:
// W_p = C A^-1 (h x h scratch per pair, ld h); pass 1: the lower-left block
// of the 2h inverse, -D^-1 W_p.  A partial last pair (m not a multiple of 2h)
// has a shorter D; a pair without a D block does nothing.
template <int PASS>
__global__ void __launch_bounds__(256) inv_double_kernel(const float *__restrict__ A, int64_t lda, int64_t m, int nb,
                                                         int h, float *Dinv, float *W) {
  const int64_t i0 = (int64_t)blockIdx.y * 2 * h;
  const int sa = (int)std::min<int64_t>(h, m - i0);
  const int sd = (int)std::min<int64_t>(h, m - i0 - h);
  if (sd <= 0) return;
  const int tiles = (h + kDT - 1) / kDT;
  const int r0 = (blockIdx.x % tiles) * kDT, c0 = (blockIdx.x / tiles) * kDT;
  float *Y = Dinv + (i0 / nb) * nb * nb;
  const int l0 = (int)(i0 % nb);
  float *Wp = W + (int64_t)blockIdx.y * h * h;
  // A^-1 is lower triangular: column tile c0 of C A^-1 takes k >= c0 only;
  // D^-1 is too: row tile r0 of D^-1 W takes k < r0 + 64 only
  if (PASS == 0)
    tile_product(A + (i0 + h) + i0 * lda, lda, Y + l0 + (int64_t)l0 * nb, nb, Wp, h, sd, sa, sa, r0, c0, 1.0f, c0,
                 sa);
  else
    tile_product(Y + (l0 + h) + (int64_t)(l0 + h) * nb, nb, Wp, h, Y + (l0 + h) + (int64_t)l0 * nb, nb, sd, sa, sd,
                 r0, c0, -1.0f, 0, r0 + kDT);
}

}  // namespace

hsma_status_t hsma_r32_diag_inverse(int nb, const float *A, int64_t lda, int64_t m, int unit, float *Dinv,
                                    cudaStream_t st) {
  if (nb < 2 * kInvBase || nb % (2 * kInvBase) != 0 || (nb & (nb - 1)) != 0)
    return hsma_diag_inverse(HSMA_R32_BF16, nb, A, lda, m, unit, Dinv, st);
  const int64_t nblk = (m + nb - 1) / nb;
  const int64_t nbase = (m + kInvBase - 1) / kInvBase;
  auto al = [](size_t v) { return (v + 1023) & ~(size_t)1023; };
  const size_t base_b = al(sizeof(float) * (size_t)nbase * kInvBase * kInvBase);
  // pair scratch: an outer block holds N_B / 2h pairs of h^2 floats at level
  // h, at most (N_B / 2)^2 in all (the last level)
  const size_t w_b = al(sizeof(float) * (size_t)nblk * (nb / 2) * (nb / 2));
  void *ws = nullptr;
  hsma_status_t s = hsma_ws_alloc(&ws, base_b + w_b, st);
  if (s != HSMA_OK) return s;
  float *base = static_cast<float *>(ws);
  float *W = reinterpret_cast<float *>(static_cast<unsigned char *>(ws) + base_b);
  do {
    if ((s = hsma_diag_inverse(HSMA_R32_BF16, kInvBase, A, lda, m, unit, base, st)) != HSMA_OK) break;
    int levels = 0;
    for (int h = kInvBase; h < nb; h *= 2) ++levels;
    HsmaTraceScope ts("diag_inverse", st, 1 + 2 * levels);
    if ((s = hsma_from_cuda(cudaMemsetAsync(Dinv, 0, sizeof(float) * (size_t)nblk * nb * nb, st))) != HSMA_OK) break;
    inv_place_kernel<<<(unsigned)nbase, 256, 0, st>>>(base, m, nb, Dinv);
    for (int h = kInvBase; h < nb; h *= 2) {
      const int64_t pairs = (m + 2 * h - 1) / (2 * h);
      if (pairs > 65535) {
        s = HSMA_ERR_UNSUPPORTED;
        break;
      }
      const int tiles = (h + kDT - 1) / kDT;
      const dim3 grid((unsigned)(tiles * tiles), (unsigned)pairs);
      inv_double_kernel<0><<<grid, 256, 0, st>>>(A, lda, m, nb, h, Dinv, W);
      inv_double_kernel<1><<<grid, 256, 0, st>>>(A, lda, m, nb, h, Dinv, W);
    }
    if (s == HSMA_OK) s = hsma_from_cuda(cudaGetLastError());
  } while (0);
  hsma_status_t f = hsma_ws_free(ws, st);
  return s != HSMA_OK ? s : f;
}
