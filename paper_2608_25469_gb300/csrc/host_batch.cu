// Varlen batch of small solves whose matrices live in host memory: the batch
// is cut into chunks of consecutive instances; chunk copies to the device,
// solves (the persistent batched kernel) and copies back run on separate
// internal streams, so the copies of some chunks overlap the solves of others
// (the copy engines and the SMs work at the same time).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/hsma.h"
#include "blocked.h"
#include "common.cuh"
#include "small.h"
#include "trace.h"
#include "workspace.h"

namespace {

constexpr int kStreams = 4;
constexpr int32_t kMaxChunks = 256;

struct PipeStreams {
  cudaStream_t s[kStreams] = {};
  bool ok = false;
};

// internal non-blocking streams (copy-in, two compute, copy-out), created
// once per device
hsma_status_t pipe_streams(cudaStream_t out[kStreams]) {
  static PipeStreams per_dev[64];
  static std::mutex mu;
  int d = 0;
  HSMA_CUDA_TRY(cudaGetDevice(&d));
  if (d < 0 || d >= 64) return HSMA_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(mu);
  PipeStreams &S = per_dev[d];
  if (!S.ok) {
    for (int k = 0; k < kStreams; ++k) HSMA_CUDA_TRY(cudaStreamCreateWithFlags(&S.s[k], cudaStreamNonBlocking));
    S.ok = true;
  }
  for (int k = 0; k < kStreams; ++k) out[k] = S.s[k];
  return HSMA_OK;
}

// device pointers and leading dimensions of the instances from their offsets
__global__ void chunk_meta_kernel(int count, const int32_t *__restrict__ m, const int64_t *__restrict__ offA,
                                  const int64_t *__restrict__ offB, int64_t baseA, int64_t baseB, char *dA, char *dB,
                                  int es, const void **pA, void **pB, int32_t *ld) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  pA[i] = dA + (offA[i] - baseA) * es;
  pB[i] = dB + (offB[i] - baseB) * es;
  ld[i] = m[i] > 1 ? m[i] : 1;
}

// Packed lower triangles (column j holds rows j..m-1, m(m+1)/2 elements) of
// instances [b0, b1) into their square device layout (ld = m): one warp per
// instance; the strict upper triangle of a square is left as it is (never
// read).  src offsets are the host's packed offsets minus baseP.
template <class T>
__global__ void unpack_tri_kernel(int b0, int b1, const int32_t *__restrict__ m, const int64_t *__restrict__ offP,
                                  int64_t baseP, const int64_t *__restrict__ offS, const T *__restrict__ src, T *dst) {
  const int lane = threadIdx.x & 31;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  for (int b = b0 + w; b < b1; b += nw) {
    const int mb = m[b];
    const T *s = src + (offP[b] - baseP);
    T *d = dst + offS[b];
    int64_t q = 0;  // packed index of column j's diagonal
    for (int j = 0; j < mb; ++j) {
      for (int r = j + lane; r < mb; r += 32) d[r + (int64_t)j * mb] = s[q + (r - j)];
      q += mb - j;
    }
  }
}

template <class T>
void launch_unpack(int b0, int b1, const int32_t *m, const int64_t *offP, int64_t baseP, const int64_t *offS,
                   const void *src, void *dst, cudaStream_t st) {
  const int blocks = std::max(1, std::min((b1 - b0 + 7) / 8, 4 * hsma_sm_count()));
  unpack_tri_kernel<T><<<blocks, 256, 0, st>>>(b0, b1, m, offP, baseP, offS, static_cast<const T *>(src),
                                               static_cast<T *>(dst));
}

hsma_status_t unpack_chunk(int dtype, int b0, int b1, const int32_t *m, const int64_t *offP, int64_t baseP,
                           const int64_t *offS, const void *src, void *dst, cudaStream_t st) {
  HsmaTraceScope ts("host_unpack", st);
  switch (hsma_small_esize(dtype)) {
    case 16: launch_unpack<double2>(b0, b1, m, offP, baseP, offS, src, dst, st); break;
    case 8: launch_unpack<double>(b0, b1, m, offP, baseP, offS, src, dst, st); break;
    default: launch_unpack<float>(b0, b1, m, offP, baseP, offS, src, dst, st); break;
  }
  return hsma_from_cuda(cudaGetLastError());
}

// The whole batch's A and B get device buffers: the copy-in stream copies the
// sizes and offsets, fills every instance's pointers, then copies A and B
// chunk by chunk; each chunk's solve runs on one of two compute streams (so a
// solve's tail overlaps the next one's start) once its copy has landed; the
// copy-out stream returns each chunk's X as soon as it is solved.
// tri = 1: A_i is stored as packed lower triangles on the host (m(m+1)/2
// elements each); they are copied packed, and read packed by the complex128
// batch or expanded on the device for the other dtypes.
inline int64_t a_elems(int32_t m, int tri) { return tri ? (int64_t)m * (m + 1) / 2 : (int64_t)m * m; }

hsma_status_t full_pipeline(int dtype, int diag, int32_t batch, const int32_t *h_m, const int32_t *h_n,
                            const void *alpha, const void *hA, const int64_t *h_offA, const void *hB,
                            const int64_t *h_offB, void *hX, int nch, int32_t per, int es, cudaStream_t caller,
                            const cudaStream_t ss[kStreams], int tri) {
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  const int64_t extA = h_offA[batch - 1] + a_elems(h_m[batch - 1], tri) - h_offA[0];
  // complex128 runs the column-packed batch, whose prep pass reads packed
  // triangles directly; the per-instance kernel of the other dtypes reads a
  // square layout, so their packed triangles are expanded on the device
  const bool packed = hsma_vbatched_packed_dtype(dtype);
  const bool expand = tri && !packed;
  // square offsets of the expanded triangles, computed here and copied once
  std::vector<int64_t> sq;
  int64_t extS = 0;
  if (expand) {
    sq.resize((size_t)batch);
    for (int32_t i = 0; i < batch; ++i) {
      sq[i] = extS;
      extS += (int64_t)h_m[i] * h_m[i];
    }
  }
  const int64_t extB = h_offB[batch - 1] + (int64_t)h_m[batch - 1] * h_n[batch - 1] - h_offB[0];
  const size_t mi_b = al(sizeof(int32_t) * batch), oi_b = al(sizeof(int64_t) * batch);
  const size_t p_b = al(sizeof(void *) * batch);
  const size_t a_b = al((size_t)extA * es), b_b = al((size_t)extB * es), s_b = al((size_t)extS * es);
  const size_t sq_b = expand ? al(sizeof(int64_t) * batch) : 0;
  // chunks on one compute stream run in order, so each stream needs one scratch
  int32_t max_m = 0;
  for (int32_t i = 0; i < batch; ++i) max_m = std::max(max_m, h_m[i]);
  const size_t scr_b = al(packed ? hsma_vbatched_packed_scratch_bytes(dtype, per, max_m)
                                 : hsma_vbatched_scratch_bytes(per));
  const int nscr = nch < 2 ? nch : 2;
  const size_t total = a_b + b_b + s_b + sq_b + 3 * mi_b + 2 * oi_b + 2 * p_b + scr_b * nscr;
  std::unique_ptr<cudaEvent_t[]> evs(new (std::nothrow) cudaEvent_t[2 * nch]());  // copied-in, solved
  if (!evs) return HSMA_ERR_NO_MEMORY;
  cudaEvent_t *ev = evs.get();
  void *ws = nullptr;
  hsma_status_t s = hsma_ws_alloc(&ws, total, caller);
  if (s != HSMA_OK) return s;
  char *q = static_cast<char *>(ws);
  char *dA = q, *dB = q + a_b;  // dA: the host's layout of A (packed triangles when tri)
  q += a_b + b_b;
  char *dS = expand ? q : dA;  // the layout the kernels read
  q += s_b;
  int64_t *gSq = expand ? reinterpret_cast<int64_t *>(q) : nullptr;
  q += sq_b;
  int32_t *gm = reinterpret_cast<int32_t *>(q), *gn = reinterpret_cast<int32_t *>(q + mi_b);
  int32_t *gld = reinterpret_cast<int32_t *>(q + 2 * mi_b);
  q += 3 * mi_b;
  int64_t *goA = reinterpret_cast<int64_t *>(q), *goB = reinterpret_cast<int64_t *>(q + oi_b);
  q += 2 * oi_b;
  const void **pA = reinterpret_cast<const void **>(q);
  void **pB = reinterpret_cast<void **>(q + p_b);
  q += 2 * p_b;
  int32_t *scr0 = reinterpret_cast<int32_t *>(q);
  cudaStream_t s_in = ss[0], s_out = ss[3];
  const cudaStream_t s_k[2] = {ss[1], ss[2]};
  auto fail = [](cudaError_t e) { return e == cudaSuccess ? HSMA_OK : hsma_from_cuda(e); };
  cudaEvent_t start = nullptr, fin = nullptr;
  do {
    if ((s = fail(cudaEventCreateWithFlags(&start, cudaEventDisableTiming))) != HSMA_OK) break;
    if ((s = fail(cudaEventCreateWithFlags(&fin, cudaEventDisableTiming))) != HSMA_OK) break;
    for (int k = 0; k < 2 * nch && s == HSMA_OK; ++k) s = fail(cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming));
    if (s != HSMA_OK) break;
    if ((s = fail(cudaEventRecord(start, caller))) != HSMA_OK) break;
    for (int k = 0; k < kStreams && s == HSMA_OK; ++k) s = fail(cudaStreamWaitEvent(ss[k], start, 0));
    if (s != HSMA_OK) break;
    {
      HsmaTraceScope ts("host_h2d", s_in, 0);
      if ((s = fail(cudaMemcpyAsync(gm, h_m, sizeof(int32_t) * batch, cudaMemcpyHostToDevice, s_in))) != HSMA_OK)
        break;
      if ((s = fail(cudaMemcpyAsync(gn, h_n, sizeof(int32_t) * batch, cudaMemcpyHostToDevice, s_in))) != HSMA_OK)
        break;
      if ((s = fail(cudaMemcpyAsync(goA, h_offA, sizeof(int64_t) * batch, cudaMemcpyHostToDevice, s_in))) !=
          HSMA_OK)
        break;
      if ((s = fail(cudaMemcpyAsync(goB, h_offB, sizeof(int64_t) * batch, cudaMemcpyHostToDevice, s_in))) !=
          HSMA_OK)
        break;
    }
    if (expand) {
      HsmaTraceScope ts("host_h2d", s_in, 0);
      if ((s = fail(cudaMemcpyAsync(gSq, sq.data(), sizeof(int64_t) * batch, cudaMemcpyHostToDevice, s_in))) !=
          HSMA_OK)
        break;
    }
    chunk_meta_kernel<<<(batch + 255) / 256, 256, 0, s_in>>>(batch, gm, expand ? gSq : goA, goB,
                                                             expand ? 0 : h_offA[0], h_offB[0], dS, dB, es, pA, pB,
                                                             gld);
    hsma_count_launches(1);
    if ((s = fail(cudaGetLastError())) != HSMA_OK) break;
    for (int c = 0; c < nch && s == HSMA_OK; ++c) {
      const int32_t b = c * per, e = std::min(batch, b + per), cnt = e - b;
      if (cnt <= 0) {
        s = fail(cudaEventRecord(ev[2 * c], s_in));
        if (s == HSMA_OK) s = fail(cudaEventRecord(ev[2 * c + 1], s_in));
        continue;
      }
      const int64_t a0 = h_offA[b] - h_offA[0], b0 = h_offB[b] - h_offB[0];
      const int64_t na = h_offA[e - 1] + a_elems(h_m[e - 1], tri) - h_offA[b];
      const int64_t nbx = h_offB[e - 1] + (int64_t)h_m[e - 1] * h_n[e - 1] - h_offB[b];
      {
        HsmaTraceScope ts("host_h2d", s_in, 0);
        if ((s = fail(cudaMemcpyAsync(dA + a0 * es, static_cast<const char *>(hA) + h_offA[b] * es, (size_t)na * es,
                                      cudaMemcpyHostToDevice, s_in))) != HSMA_OK)
          break;
        if ((s = fail(cudaMemcpyAsync(dB + b0 * es, static_cast<const char *>(hB) + h_offB[b] * es,
                                      (size_t)nbx * es, cudaMemcpyHostToDevice, s_in))) != HSMA_OK)
          break;
      }
      if ((s = fail(cudaEventRecord(ev[2 * c], s_in))) != HSMA_OK) break;
      cudaStream_t sk = s_k[c & 1];
      if ((s = fail(cudaStreamWaitEvent(sk, ev[2 * c], 0))) != HSMA_OK) break;
      if (expand && (s = unpack_chunk(dtype, b, e, gm, goA, h_offA[0], gSq, dA, dS, sk)) != HSMA_OK) break;
      int32_t *scr = reinterpret_cast<int32_t *>(reinterpret_cast<char *>(scr0) + scr_b * (c & 1));
      if (packed)
        s = hsma_small_vbatched_packed(dtype, cnt, max_m, gm + b, gn + b, static_cast<const double *>(alpha), pA + b,
                                       gld + b, pB + b, gld + b, diag == HSMA_UNIT, nullptr, scr, sk, tri);
      else
        s = hsma_small_vbatched(dtype, cnt, gm + b, gn + b, static_cast<const double *>(alpha), pA + b, gld + b,
                                pB + b, gld + b, diag == HSMA_UNIT, nullptr, scr, sk);
      if (s != HSMA_OK) break;
      if ((s = fail(cudaEventRecord(ev[2 * c + 1], sk))) != HSMA_OK) break;
      if ((s = fail(cudaStreamWaitEvent(s_out, ev[2 * c + 1], 0))) != HSMA_OK) break;
      {
        HsmaTraceScope ts("host_d2h", s_out, 0);
        if ((s = fail(cudaMemcpyAsync(static_cast<char *>(hX) + h_offB[b] * es, dB + b0 * es, (size_t)nbx * es,
                                      cudaMemcpyDeviceToHost, s_out))) != HSMA_OK)
          break;
      }
    }
    // the caller's stream resumes when every internal stream is done
    for (int k = 0; k < kStreams; ++k) {
      hsma_status_t r = fail(cudaEventRecord(fin, ss[k]));
      if (r == HSMA_OK) r = fail(cudaStreamWaitEvent(caller, fin, 0));
      if (s == HSMA_OK) s = r;
    }
  } while (0);
  if (start) cudaEventDestroy(start);
  if (fin) cudaEventDestroy(fin);
  for (int k = 0; k < 2 * nch; ++k)
    if (ev[k]) cudaEventDestroy(ev[k]);
  hsma_status_t f = hsma_ws_free(ws, caller);
  return s != HSMA_OK ? s : f;
}

}  // namespace

namespace {

hsma_status_t host_batch_entry(int dtype, int diag, int32_t batch, const int32_t *h_m, const int32_t *h_n,
                               const void *alpha, const void *hA, const int64_t *h_offA, const void *hB,
                               const int64_t *h_offB, void *hX, int32_t chunks, void *stream, int tri) {
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
    if (i > 0 && (h_offA[i] < h_offA[i - 1] + a_elems(h_m[i - 1], tri) ||
                  h_offB[i] < h_offB[i - 1] + (int64_t)h_m[i - 1] * h_n[i - 1]))
      return HSMA_ERR_INVALID_ARG;
  }
  const int es = hsma_small_esize(dtype);
  // default chunk counts measured fastest on GB300 for the 8192-instance
  // complex128 batch: 8 with square A, 6 with packed triangles (fewer bytes
  // per chunk to copy, so fewer and longer solves pay)
  const int nch = std::min<int32_t>(batch, chunks > 0 ? std::min<int32_t>(chunks, kMaxChunks) : (tri ? 6 : 8));
  const int32_t per = (batch + nch - 1) / nch;
  cudaStream_t caller = static_cast<cudaStream_t>(stream);
  cudaStream_t ss[kStreams];
  hsma_status_t s = pipe_streams(ss);
  if (s != HSMA_OK) return s;
  return full_pipeline(dtype, diag, batch, h_m, h_n, alpha, hA, h_offA, hB, h_offB, hX, nch, per, es, caller, ss,
                       tri);
}

}  // namespace

extern "C" HSMA_API hsma_status_t hsma_trsm_llnn_vbatched_host(int dtype, int diag, int32_t batch,
                                                                const int32_t *h_m, const int32_t *h_n,
                                                                const void *alpha, const void *hA,
                                                                const int64_t *h_offA, const void *hB,
                                                                const int64_t *h_offB, void *hX, int32_t chunks,
                                                                void *stream) {
  return host_batch_entry(dtype, diag, batch, h_m, h_n, alpha, hA, h_offA, hB, h_offB, hX, chunks, stream, 0);
}

extern "C" HSMA_API hsma_status_t hsma_trsm_llnn_vbatched_host_tp(int dtype, int diag, int32_t batch,
                                                                   const int32_t *h_m, const int32_t *h_n,
                                                                   const void *alpha, const void *hAp,
                                                                   const int64_t *h_offA, const void *hB,
                                                                   const int64_t *h_offB, void *hX, int32_t chunks,
                                                                   void *stream) {
  return host_batch_entry(dtype, diag, batch, h_m, h_n, alpha, hAp, h_offA, hB, h_offB, hX, chunks, stream, 1);
}
