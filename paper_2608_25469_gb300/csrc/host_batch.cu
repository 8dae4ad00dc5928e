// Varlen batch of small solves whose matrices live in host memory: the batch
// is cut into chunks of consecutive instances, and each chunk's host-to-device
// copy, solve (the persistent batched kernel) and device-to-host copy run on
// one of three internal streams, so the copies of some chunks overlap the
// solves of others (the copy engines and the SMs work at the same time).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "../../include/hsma.h"
#include "common.cuh"
#include "small.h"
#include "trace.h"
#include "workspace.h"

namespace {

constexpr int kSlots = 3;

struct SlotStreams {
  cudaStream_t s[kSlots] = {};
  bool ok = false;
};

// internal non-blocking streams, created once per device
hsma_status_t slot_streams(cudaStream_t out[kSlots]) {
  static SlotStreams per_dev[64];
  static std::mutex mu;
  int d = 0;
  HSMA_CUDA_TRY(cudaGetDevice(&d));
  if (d < 0 || d >= 64) return HSMA_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(mu);
  SlotStreams &S = per_dev[d];
  if (!S.ok) {
    for (int k = 0; k < kSlots; ++k) HSMA_CUDA_TRY(cudaStreamCreateWithFlags(&S.s[k], cudaStreamNonBlocking));
    S.ok = true;
  }
  for (int k = 0; k < kSlots; ++k) out[k] = S.s[k];
  return HSMA_OK;
}

// device pointers and leading dimensions of one chunk from its offsets
__global__ void chunk_meta_kernel(int count, const int32_t *__restrict__ m, const int64_t *__restrict__ offA,
                                  const int64_t *__restrict__ offB, int64_t baseA, int64_t baseB, char *dA, char *dB,
                                  int es, const void **pA, void **pB, int32_t *ld) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  pA[i] = dA + (offA[i] - baseA) * es;
  pB[i] = dB + (offB[i] - baseB) * es;
  ld[i] = m[i] > 1 ? m[i] : 1;
}

}  // namespace

extern "C" HSMA_API hsma_status_t hsma_trsm_llnn_vbatched_host(int dtype, int diag, int32_t batch,
                                                                const int32_t *h_m, const int32_t *h_n,
                                                                const void *alpha, const void *hA,
                                                                const int64_t *h_offA, const void *hB,
                                                                const int64_t *h_offB, void *hX, int32_t chunks,
                                                                void *stream) {
  if (!hsma_small_dtype(dtype)) {
    return (dtype == HSMA_R32_BF16 || dtype == HSMA_R64_IR) ? HSMA_ERR_UNSUPPORTED : HSMA_ERR_INVALID_ARG;
  }
  if ((diag != HSMA_NON_UNIT && diag != HSMA_UNIT) || batch < 0 || chunks < 0) return HSMA_ERR_INVALID_ARG;
  if (batch == 0) return HSMA_OK;
  if (h_m == nullptr || h_n == nullptr || alpha == nullptr || hA == nullptr || h_offA == nullptr ||
      hB == nullptr || h_offB == nullptr || hX == nullptr)
    return HSMA_ERR_INVALID_ARG;
  for (int32_t i = 0; i < batch; ++i) {
    if (h_m[i] < 0 || h_n[i] < 0 || h_offA[i] < 0 || h_offB[i] < 0) return HSMA_ERR_INVALID_ARG;
    if (h_m[i] > 64) return HSMA_ERR_UNSUPPORTED;
    if (i > 0 && (h_offA[i] < h_offA[i - 1] + (int64_t)h_m[i - 1] * h_m[i - 1] ||
                  h_offB[i] < h_offB[i - 1] + (int64_t)h_m[i - 1] * h_n[i - 1]))
      return HSMA_ERR_INVALID_ARG;
  }
  const int es = hsma_small_esize(dtype);
  const int nch = std::min<int32_t>(batch, chunks > 0 ? chunks : 8);
  const int32_t per = (batch + nch - 1) / nch;
  // element extents of each chunk in the packed buffers
  auto extA = [&](int32_t b, int32_t e) { return h_offA[e - 1] + (int64_t)h_m[e - 1] * h_m[e - 1] - h_offA[b]; };
  auto extB = [&](int32_t b, int32_t e) { return h_offB[e - 1] + (int64_t)h_m[e - 1] * h_n[e - 1] - h_offB[b]; };
  int64_t maxA = 0, maxB = 0;
  for (int c = 0; c < nch; ++c) {
    const int32_t b = c * per, e = std::min(batch, b + per);
    if (b >= e) continue;
    maxA = std::max(maxA, extA(b, e));
    maxB = std::max(maxB, extB(b, e));
  }
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  const size_t a_b = al((size_t)maxA * es), b_b = al((size_t)maxB * es);
  const size_t meta_b = al(sizeof(int32_t) * per) * 3 + al(sizeof(int64_t) * per) * 2 + al(sizeof(void *) * per) * 2;
  const size_t scr_b = al(hsma_vbatched_scratch_bytes(per));
  const size_t slot_b = a_b + b_b + meta_b + scr_b;
  cudaStream_t caller = static_cast<cudaStream_t>(stream);
  cudaStream_t ss[kSlots];
  hsma_status_t s = slot_streams(ss);
  if (s != HSMA_OK) return s;
  void *ws = nullptr;
  if ((s = hsma_ws_alloc(&ws, slot_b * kSlots, caller)) != HSMA_OK) return s;
  cudaEvent_t start = nullptr, done[kSlots] = {};
  auto fail = [](cudaError_t e) { return e == cudaSuccess ? HSMA_OK : hsma_from_cuda(e); };
  do {
    if ((s = fail(cudaEventCreateWithFlags(&start, cudaEventDisableTiming))) != HSMA_OK) break;
    if ((s = fail(cudaEventRecord(start, caller))) != HSMA_OK) break;
    for (int k = 0; k < kSlots && s == HSMA_OK; ++k) {
      s = fail(cudaEventCreateWithFlags(&done[k], cudaEventDisableTiming));
      if (s == HSMA_OK) s = fail(cudaStreamWaitEvent(ss[k], start, 0));
    }
    for (int c = 0; c < nch && s == HSMA_OK; ++c) {
      const int32_t b = c * per, e = std::min(batch, b + per), cnt = e - b;
      if (cnt <= 0) continue;
      cudaStream_t st = ss[c % kSlots];
      char *slot = static_cast<char *>(ws) + slot_b * (c % kSlots);
      char *dA = slot, *dB = slot + a_b;
      char *meta = slot + a_b + b_b;
      int32_t *dm = reinterpret_cast<int32_t *>(meta);
      int32_t *dn = reinterpret_cast<int32_t *>(meta + al(sizeof(int32_t) * per));
      int32_t *dld = reinterpret_cast<int32_t *>(meta + 2 * al(sizeof(int32_t) * per));
      int64_t *doA = reinterpret_cast<int64_t *>(meta + 3 * al(sizeof(int32_t) * per));
      int64_t *doB = reinterpret_cast<int64_t *>(reinterpret_cast<char *>(doA) + al(sizeof(int64_t) * per));
      const void **pA = reinterpret_cast<const void **>(reinterpret_cast<char *>(doB) + al(sizeof(int64_t) * per));
      void **pB = reinterpret_cast<void **>(reinterpret_cast<char *>(pA) + al(sizeof(void *) * per));
      int32_t *scr = reinterpret_cast<int32_t *>(meta + meta_b);
      {
        HsmaTraceScope ts("host_h2d", st);
        const char *srcA = static_cast<const char *>(hA) + h_offA[b] * es;
        const char *srcB = static_cast<const char *>(hB) + h_offB[b] * es;
        if ((s = fail(cudaMemcpyAsync(dA, srcA, (size_t)extA(b, e) * es, cudaMemcpyHostToDevice, st))) != HSMA_OK)
          break;
        if ((s = fail(cudaMemcpyAsync(dB, srcB, (size_t)extB(b, e) * es, cudaMemcpyHostToDevice, st))) != HSMA_OK)
          break;
        if ((s = fail(cudaMemcpyAsync(dm, h_m + b, sizeof(int32_t) * cnt, cudaMemcpyHostToDevice, st))) != HSMA_OK)
          break;
        if ((s = fail(cudaMemcpyAsync(dn, h_n + b, sizeof(int32_t) * cnt, cudaMemcpyHostToDevice, st))) != HSMA_OK)
          break;
        if ((s = fail(cudaMemcpyAsync(doA, h_offA + b, sizeof(int64_t) * cnt, cudaMemcpyHostToDevice, st))) !=
            HSMA_OK)
          break;
        if ((s = fail(cudaMemcpyAsync(doB, h_offB + b, sizeof(int64_t) * cnt, cudaMemcpyHostToDevice, st))) !=
            HSMA_OK)
          break;
      }
      chunk_meta_kernel<<<(cnt + 255) / 256, 256, 0, st>>>(cnt, dm, doA, doB, h_offA[b], h_offB[b], dA, dB, es, pA,
                                                           pB, dld);
      if ((s = fail(cudaGetLastError())) != HSMA_OK) break;
      s = hsma_small_vbatched(dtype, cnt, dm, dn, static_cast<const double *>(alpha), pA, dld, pB, dld,
                              diag == HSMA_UNIT, nullptr, scr, st);
      if (s != HSMA_OK) break;
      {
        HsmaTraceScope ts("host_d2h", st);
        char *dst = static_cast<char *>(hX) + h_offB[b] * es;
        if ((s = fail(cudaMemcpyAsync(dst, dB, (size_t)extB(b, e) * es, cudaMemcpyDeviceToHost, st))) != HSMA_OK)
          break;
      }
    }
    for (int k = 0; k < kSlots; ++k) {
      if (done[k] == nullptr) continue;
      hsma_status_t r = fail(cudaEventRecord(done[k], ss[k]));
      if (r == HSMA_OK) r = fail(cudaStreamWaitEvent(caller, done[k], 0));
      if (s == HSMA_OK) s = r;
    }
  } while (0);
  if (start) cudaEventDestroy(start);
  for (int k = 0; k < kSlots; ++k)
    if (done[k]) cudaEventDestroy(done[k]);
  hsma_status_t f = hsma_ws_free(ws, caller);
  return s != HSMA_OK ? s : f;
}
