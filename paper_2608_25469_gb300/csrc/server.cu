// Serving loop: continuous batching of triangular solves on one GPU.
//
// Requests (fp64 or complex128, any m, n; a triangular solve, or a solve with
// LU or Cholesky factors) are submitted from any host thread and stamped with
// their arrival time.  A scheduler thread admits pending requests in arrival
// order while their device memory (A, B, pivots and the blocked path's
// workspace) fits the budget, brings their data onto the device (generated
// there from a seed, or copied from host memory), and launches them without
// waiting for earlier work: requests with m <= 64 that are ready together are
// grouped into one varlen batched launch per dtype and kind (the factor
// solves through the fused factor-solve batch); larger requests run the
// blocked path on a ring of streams, so their work overlaps on the device.  A completion event per launch frees the memory and records the
// latency (arrival to completion).  Results are the same as solving each
// request alone, because each request's arithmetic does not depend on what
// runs beside it.
//
// With HSMA_SERVER_FP64_EMULATED the blocked requests with m >= 384 use FP64
// products emulated on the BF16 tensor cores (the fp64_products option); below
// that the FP64 tensor products of a few block steps take no longer than the
// emulated path's extra slicing launches.
//
// A fake-device mode (HSMA_SERVER_FAKE_DEVICE) runs the same admission and
// queue logic with no GPU: each "launch" completes after a modelled time.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/hsma.h"
#include "common.cuh"
#include "gen.h"
#include "mixed.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
  hsma_request_t r;
  Clock::time_point arrival;
  size_t need = 0;
  void *dA = nullptr, *dB = nullptr, *dPiv = nullptr;
  int stream = 0;
  std::atomic<int> done{0};
  double latency = 0.0;
  hsma_status_t status = HSMA_OK;
};

struct Flight {  // one launch in flight: a batched group or one blocked solve
  std::vector<Req *> reqs;  // owned by hsma_server::all; a Req never moves
  cudaEvent_t ev = nullptr;
  void *meta = nullptr;  // device arrays of a batched group
  Clock::time_point fake_done;
};

size_t esize(int dtype) { return dtype == HSMA_C128 ? 16 : 8; }

}  // namespace

struct hsma_server {
  size_t budget = 0;
  int nstreams = 1;
  unsigned flags = 0;
  bool fake = false;
  std::vector<cudaStream_t> streams;
  cudaMemPool_t pool = nullptr;
  int device = 0;

  std::mutex mu;
  std::condition_variable cv;
  // Every request, indexed by ticket.  The deque is only touched under `mu`;
  // the scheduler works on the Req objects themselves (which never move) so
  // it never indexes the deque while a submit may be growing it.
  std::deque<std::unique_ptr<Req>> all;
  std::deque<Req *> inbox;    // submitted, not yet seen by the scheduler
  std::deque<Req *> pending;  // waiting for admission
  std::vector<Flight> flights;
  bool stop = false;
  std::thread worker;
  int next_stream = 1;

  // statistics
  std::atomic<uint64_t> n_sub{0}, n_adm{0}, n_done{0}, n_batched{0}, n_blocked{0};
  size_t in_use = 0, peak = 0;
  hsma_status_t sticky = HSMA_OK;
};

namespace {

constexpr int64_t kEmulatedMinM = 384;  // smallest m served with emulated products

bool use_emulated(const hsma_request_t &r, unsigned flags) {
  return (flags & HSMA_SERVER_FP64_EMULATED) != 0 && r.m >= kEmulatedMinM;
}

size_t request_bytes(const hsma_request_t &r, unsigned flags) {
  const size_t es = esize(r.dtype);
  size_t b = es * (size_t)r.m * (size_t)r.m + es * (size_t)r.m * (size_t)r.n;
  if (r.ipiv_host != nullptr) b += sizeof(int32_t) * (size_t)r.m;
  if (r.m > 64 && r.kind != HSMA_REQ_TRSM) {
    // the factor solves: permutation and a gathered copy of B, then two
    // triangular solves one after the other (their workspaces never coexist)
    b += sizeof(int32_t) * (size_t)r.m + es * (size_t)r.m * (size_t)r.n;
  }
  if (use_emulated(r, flags)) {
    hsma_opts_t o;
    std::memset(&o, 0, sizeof o);
    o.fp64_products = 1;
    hsma_plan_t p;
    if (hsma_make_plan(r.dtype, r.m, r.n, &o, &p) != HSMA_OK) p.nb = kHsmaEmulatedNb, p.panel_cols = 0;
    return b + hsma_blocked_emulated_ws_bytes(r.dtype, p.nb, p.panel_cols, r.m, r.n);
  }
  if (r.m > 64) {
    hsma_plan_t p;
    hsma_plan(r.dtype, r.m, r.n, &p);
    const size_t nb = (size_t)(p.nb > 0 ? p.nb : 256);
    const size_t nblk = ((size_t)r.m + nb - 1) / nb;
    b += es * (nblk * nb * nb + nb * (size_t)r.n);  // Dinv + block-row copy
  }
  return b;
}

hsma_status_t dev_alloc(hsma_server *s, void **p, size_t bytes, cudaStream_t st) {
  *p = nullptr;
  if (bytes == 0) return HSMA_OK;
  cudaError_t e = cudaMallocFromPoolAsync(p, bytes, s->pool, st);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? HSMA_ERR_NO_MEMORY : HSMA_ERR_CUDA;
  }
  return HSMA_OK;
}

// bring one admitted request's inputs onto the device (stream-ordered)
hsma_status_t stage_inputs(hsma_server *s, Req &q) {
  const hsma_request_t &r = q.r;
  cudaStream_t st = s->streams[q.stream];
  const size_t es = esize(r.dtype);
  hsma_status_t rc = dev_alloc(s, &q.dA, es * r.m * r.m, st);
  if (rc == HSMA_OK) rc = dev_alloc(s, &q.dB, es * r.m * r.n, st);
  if (rc == HSMA_OK && r.ipiv_host != nullptr) rc = dev_alloc(s, &q.dPiv, sizeof(int32_t) * r.m, st);
  if (rc != HSMA_OK) return rc;
  if (r.ipiv_host != nullptr)
    HSMA_CUDA_TRY(cudaMemcpyAsync(q.dPiv, r.ipiv_host, sizeof(int32_t) * r.m, cudaMemcpyHostToDevice, st));
  if (r.A_host != nullptr) {
    HSMA_CUDA_TRY(cudaMemcpy2DAsync(q.dA, es * r.m, r.A_host, es * r.lda, es * r.m, r.m, cudaMemcpyHostToDevice, st));
    HSMA_CUDA_TRY(cudaMemcpy2DAsync(q.dB, es * r.m, r.B_host, es * r.ldb, es * r.m, r.n, cudaMemcpyHostToDevice, st));
    return HSMA_OK;
  }
  rc = hsma_gen_launch(r.dtype, r.kind == HSMA_REQ_GETRS ? 2 : 0, r.gen_seed, r.gen_inst, r.m, r.m, q.dA, r.m, st);
  if (rc == HSMA_OK) rc = hsma_gen_launch(r.dtype, 1, r.gen_seed, r.gen_inst, r.m, r.n, q.dB, r.m, st);
  return rc;
}

hsma_status_t fetch_output(hsma_server *s, Req &q) {
  const hsma_request_t &r = q.r;
  if (r.X_host == nullptr) return HSMA_OK;
  const size_t es = esize(r.dtype);
  HSMA_CUDA_TRY(cudaMemcpy2DAsync(r.X_host, es * r.ldx, q.dB, es * r.m, es * r.m, r.n, cudaMemcpyDeviceToHost,
                                  s->streams[q.stream]));
  return HSMA_OK;
}

double fake_seconds(const hsma_request_t &r) {
  // modelled device time: counted flops at 1 TFLOP/s plus 20 us per launch
  const double f = (double)r.m * r.m * r.n * (r.dtype == HSMA_C128 ? 4.0 : 1.0);
  return 20e-6 + f / 1e12;
}

void finish(hsma_server *s, Req &q, Clock::time_point now) {
  q.latency = std::chrono::duration<double>(now - q.arrival).count();
  q.done.store(1);
  s->n_done.fetch_add(1);
}

// One varlen batched launch for the requests of group g (one dtype and kind,
// all with m <= 64) on stream 0: the triangular-solve batch, or the fused
// factor-solve batch.  Requests whose alpha (or, for triangular solves, diag)
// differs from the first one's run as single solves of the same kind.
Flight launch_group(hsma_server *s, int dt, int kind, const std::vector<Req *> &g) {
  cudaStream_t st = s->streams[0];
  const int nb = (int)g.size();
  // host staging of the group's size and pointer arrays (pageable copies are fine: small)
  std::vector<int32_t> hm(nb), hn(nb);
  std::vector<void *> ha(nb), hb(nb), hp(nb);
  for (int k = 0; k < nb; ++k) {
    hm[k] = (int32_t)g[k]->r.m;
    hn[k] = (int32_t)g[k]->r.n;
    ha[k] = g[k]->dA;
    hb[k] = g[k]->dB;
    hp[k] = g[k]->dPiv;
  }
  Flight f;
  f.reqs = g;
  const size_t bytes = (size_t)nb * (3 * sizeof(int32_t) + 3 * sizeof(void *)) + 64;
  hsma_status_t rc = dev_alloc(s, &f.meta, bytes, st);
  hsma_status_t rc2 = HSMA_OK;
  if (rc == HSMA_OK) {
    unsigned char *base = static_cast<unsigned char *>(f.meta);
    void **dpa = reinterpret_cast<void **>(base);
    void **dpb = dpa + nb;
    void **dpp = dpb + nb;
    int32_t *dm = reinterpret_cast<int32_t *>(dpp + nb);
    int32_t *dn = dm + nb;
    cudaMemcpyAsync(dpa, ha.data(), sizeof(void *) * nb, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(dpb, hb.data(), sizeof(void *) * nb, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(dpp, hp.data(), sizeof(void *) * nb, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(dm, hm.data(), sizeof(int32_t) * nb, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(dn, hn.data(), sizeof(int32_t) * nb, cudaMemcpyHostToDevice, st);
    const hsma_request_t &r0 = g[0]->r;
    bool uniform = true;
    for (Req *q : g) {
      const hsma_request_t &r = q->r;
      uniform &= r.alpha[0] == r0.alpha[0] && r.alpha[1] == r0.alpha[1] &&
                 (kind != HSMA_REQ_TRSM || r.diag == r0.diag);
    }
    if (uniform) {
      if (kind == HSMA_REQ_GETRS)
        rc2 = hsma_getrs_vbatched(dt, nb, dm, dn, r0.alpha, (const void *const *)dpa, dm,
                                  (const int32_t *const *)dpp, (void *const *)dpb, dm, 64, 0, nullptr, st);
      else if (kind == HSMA_REQ_POTRS)
        rc2 = hsma_potrs_vbatched(dt, nb, dm, dn, r0.alpha, (const void *const *)dpa, dm, (void *const *)dpb, dm, 64,
                                  0, nullptr, st);
      else
        rc2 = hsma_trsm_llnn_vbatched(dt, r0.diag, nb, dm, dn, r0.alpha, (const void *const *)dpa, dm,
                                      (void *const *)dpb, dm, 64, 0, nullptr, st);
    } else {
      for (Req *qp : g) {
        Req &q = *qp;
        hsma_status_t r1;
        if (kind == HSMA_REQ_GETRS)
          r1 = hsma_getrs(dt, q.r.m, q.r.n, q.r.alpha, q.dA, q.r.m, static_cast<const int32_t *>(q.dPiv), q.dB,
                          q.r.m, st, nullptr);
        else if (kind == HSMA_REQ_POTRS)
          r1 = hsma_potrs(dt, q.r.m, q.r.n, q.r.alpha, q.dA, q.r.m, q.dB, q.r.m, st, nullptr);
        else
          r1 = hsma_trsm_llnn(dt, q.r.diag, q.r.m, q.r.n, q.r.alpha, q.dA, q.r.m, q.dB, q.r.m, st);
        if (r1 != HSMA_OK) rc2 = r1;
      }
    }
    for (Req *q : g) fetch_output(s, *q);
    s->n_batched.fetch_add(1);
  }
  if (rc != HSMA_OK || rc2 != HSMA_OK)
    for (Req *q : g) q->status = rc != HSMA_OK ? rc : rc2;
  cudaEventCreateWithFlags(&f.ev, cudaEventDisableTiming);
  cudaEventRecord(f.ev, st);
  return f;
}

// Launch what was admitted in this tick.  Called with the lock NOT held.
void launch(hsma_server *s, std::vector<Req *> &small_group, std::vector<Req *> &large) {
  std::vector<Flight> out;
  if (s->fake) {
    auto now = Clock::now();
    double tsum = 0.0;
    Flight f;
    for (Req *q : small_group) tsum += fake_seconds(q->r);
    if (!small_group.empty()) {
      f.reqs = small_group;
      f.fake_done = now + std::chrono::microseconds((long)(tsum * 1e6));
      out.push_back(f);
    }
    for (Req *q : large) {
      Flight g;
      g.reqs = {q};
      g.fake_done = now + std::chrono::microseconds((long)(fake_seconds(q->r) * 1e6));
      out.push_back(g);
    }
  } else {
    cudaSetDevice(s->device);
    // one batched launch per dtype and kind for the small requests, on stream 0
    for (int dt = HSMA_R64; dt <= HSMA_C128; ++dt) {
      for (int kind = HSMA_REQ_TRSM; kind <= HSMA_REQ_POTRS; ++kind) {
        std::vector<Req *> g;
        for (Req *q : small_group)
          if (q->r.dtype == dt && q->r.kind == kind) g.push_back(q);
        if (!g.empty()) out.push_back(launch_group(s, dt, kind, g));
      }
    }
    for (Req *qp : large) {
      Req &q = *qp;
      cudaStream_t st = s->streams[q.stream];
      hsma_opts_t o;
      std::memset(&o, 0, sizeof o);
      o.fp64_products = use_emulated(q.r, s->flags) ? 1 : 0;
      hsma_status_t rc;
      if (q.r.kind == HSMA_REQ_GETRS)
        rc = hsma_getrs(q.r.dtype, q.r.m, q.r.n, q.r.alpha, q.dA, q.r.m, static_cast<const int32_t *>(q.dPiv), q.dB,
                        q.r.m, st, &o);
      else if (q.r.kind == HSMA_REQ_POTRS)
        rc = hsma_potrs(q.r.dtype, q.r.m, q.r.n, q.r.alpha, q.dA, q.r.m, q.dB, q.r.m, st, &o);
      else
        rc = hsma_trsm_llnn_ex(q.r.dtype, q.r.diag, q.r.m, q.r.n, q.r.alpha, q.dA, q.r.m, q.dB, q.r.m, st, &o,
                               nullptr);
      if (rc == HSMA_OK) rc = fetch_output(s, q);
      q.status = rc;
      s->n_blocked.fetch_add(1);
      Flight f;
      f.reqs = {qp};
      cudaEventCreateWithFlags(&f.ev, cudaEventDisableTiming);
      cudaEventRecord(f.ev, st);
      out.push_back(f);
    }
  }
  std::lock_guard<std::mutex> lk(s->mu);
  for (auto &f : out) s->flights.push_back(f);
}

void worker_loop(hsma_server *s) {
  if (!s->fake) cudaSetDevice(s->device);
  for (;;) {
    std::vector<Req *> small_group, large;
    bool idle = true;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (s->stop && s->inbox.empty() && s->pending.empty() && s->flights.empty()) break;
      while (!s->inbox.empty()) {
        s->pending.push_back(s->inbox.front());
        s->inbox.pop_front();
      }
      // admission in arrival order: a request that does not fit waits; later
      // ones that fit may go first (the budget is much larger than one request)
      for (auto it = s->pending.begin(); it != s->pending.end();) {
        Req &q = **it;
        if (q.need > s->budget) {  // can never fit
          q.status = HSMA_ERR_NO_MEMORY;
          finish(s, q, Clock::now());
          it = s->pending.erase(it);
          continue;
        }
        if (s->in_use + q.need > s->budget) {
          ++it;
          continue;
        }
        s->in_use += q.need;
        s->peak = std::max(s->peak, s->in_use);
        s->n_adm.fetch_add(1);
        if (q.r.m <= 64) {
          q.stream = 0;
          small_group.push_back(*it);
        } else {
          q.stream = s->nstreams > 1 ? s->next_stream : 0;
          if (s->nstreams > 1) s->next_stream = 1 + (s->next_stream % (s->nstreams - 1));
          large.push_back(*it);
        }
        it = s->pending.erase(it);
      }
    }
    if (!small_group.empty() || !large.empty()) {
      idle = false;
      if (!s->fake) {
        for (Req *q : small_group) {
          hsma_status_t rc = stage_inputs(s, *q);
          if (rc != HSMA_OK) q->status = rc;
        }
        for (Req *q : large) {
          hsma_status_t rc = stage_inputs(s, *q);
          if (rc != HSMA_OK) q->status = rc;
        }
      }
      launch(s, small_group, large);
    }
    // completions
    {
      std::vector<Flight> done;
      {
        std::lock_guard<std::mutex> lk(s->mu);
        auto now = Clock::now();
        for (auto it = s->flights.begin(); it != s->flights.end();) {
          bool ready;
          if (s->fake) {
            ready = now >= it->fake_done;
          } else {
            cudaError_t e = cudaEventQuery(it->ev);
            ready = e != cudaErrorNotReady;
            if (e != cudaSuccess && e != cudaErrorNotReady) {
              for (Req *q : it->reqs) q->status = HSMA_ERR_CUDA;
              (void)cudaGetLastError();
            }
          }
          if (ready) {
            done.push_back(*it);
            it = s->flights.erase(it);
          } else {
            ++it;
          }
        }
      }
      if (!done.empty()) {
        idle = false;
        auto now = Clock::now();
        for (auto &f : done) {
          if (!s->fake) {
            for (Req *qp : f.reqs) {
              Req &q = *qp;
              cudaFreeAsync(q.dA, s->streams[q.stream]);
              cudaFreeAsync(q.dB, s->streams[q.stream]);
              if (q.dPiv) cudaFreeAsync(q.dPiv, s->streams[q.stream]);
              q.dA = q.dB = q.dPiv = nullptr;
            }
            if (f.meta) cudaFreeAsync(f.meta, s->streams[0]);
            cudaEventDestroy(f.ev);
          }
          std::lock_guard<std::mutex> lk(s->mu);
          for (Req *qp : f.reqs) {
            Req &q = *qp;
            s->in_use -= q.need;
            finish(s, q, now);
          }
        }
        s->cv.notify_all();
      }
    }
    if (idle) {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv.wait_for(lk, std::chrono::microseconds(20),
                     [&] { return !s->inbox.empty() || (s->stop && s->flights.empty() && s->pending.empty()); });
    }
  }
}

}  // namespace

extern "C" {

HSMA_API hsma_status_t hsma_server_create(size_t budget_bytes, int n_streams, unsigned int flags,
                                          hsma_server_t **out) {
  if (out == nullptr || budget_bytes == 0 || n_streams < 1 || n_streams > 64) return HSMA_ERR_INVALID_ARG;
  if ((flags & ~(HSMA_SERVER_FAKE_DEVICE | HSMA_SERVER_FP64_EMULATED)) != 0) return HSMA_ERR_INVALID_ARG;
  *out = nullptr;
  auto *s = new hsma_server();
  s->budget = budget_bytes;
  s->nstreams = n_streams;
  s->flags = flags;
  s->fake = (flags & HSMA_SERVER_FAKE_DEVICE) != 0;
  if (!s->fake) {
    cudaError_t e = cudaGetDevice(&s->device);
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof props);
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = s->device;
    if (e == cudaSuccess) e = cudaMemPoolCreate(&s->pool, &props);
    if (e == cudaSuccess) {
      uint64_t thr = budget_bytes;
      e = cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    for (int k = 0; k < n_streams && e == cudaSuccess; ++k) {
      cudaStream_t st;
      e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
      if (e == cudaSuccess) s->streams.push_back(st);
    }
    if (e != cudaSuccess) {
      for (auto st : s->streams) cudaStreamDestroy(st);
      if (s->pool) cudaMemPoolDestroy(s->pool);
      delete s;
      return hsma_from_cuda(e);
    }
  }
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return HSMA_OK;
}

HSMA_API hsma_status_t hsma_server_submit(hsma_server_t *s, const hsma_request_t *req, uint64_t *ticket) {
  if (s == nullptr || req == nullptr || ticket == nullptr) return HSMA_ERR_INVALID_ARG;
  const hsma_request_t &r = *req;
  if ((r.dtype != HSMA_R64 && r.dtype != HSMA_C128) || (r.diag != HSMA_NON_UNIT && r.diag != HSMA_UNIT))
    return HSMA_ERR_INVALID_ARG;
  if (r.m < 1 || r.n < 1 || r.m > INT32_MAX || r.n > INT32_MAX) return HSMA_ERR_INVALID_ARG;
  if (r.A_host != nullptr && (r.B_host == nullptr || r.lda < r.m || r.ldb < r.m)) return HSMA_ERR_INVALID_ARG;
  if (r.X_host != nullptr && r.ldx < r.m) return HSMA_ERR_INVALID_ARG;
  if (r.A_host == nullptr && r.gen_inst < -1) return HSMA_ERR_INVALID_ARG;
  if (r.kind < HSMA_REQ_TRSM || r.kind > HSMA_REQ_POTRS) return HSMA_ERR_INVALID_ARG;
  if (r.ipiv_host != nullptr && r.kind != HSMA_REQ_GETRS) return HSMA_ERR_INVALID_ARG;
  auto q = std::make_unique<Req>();
  q->r = r;
  q->arrival = Clock::now();
  q->need = request_bytes(r, s->flags);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return HSMA_ERR_BUSY;
    *ticket = s->all.size();
    s->inbox.push_back(q.get());
    s->all.push_back(std::move(q));
  }
  s->n_sub.fetch_add(1);
  s->cv.notify_all();
  return HSMA_OK;
}

HSMA_API hsma_status_t hsma_server_poll(hsma_server_t *s, uint64_t ticket, int *done, double *latency_s) {
  if (s == nullptr || done == nullptr) return HSMA_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  if (ticket >= s->all.size()) return HSMA_ERR_INVALID_ARG;
  Req &q = *s->all[ticket];
  *done = q.done.load();
  if (latency_s) *latency_s = *done ? q.latency : 0.0;
  return *done ? q.status : HSMA_OK;
}

HSMA_API hsma_status_t hsma_server_drain(hsma_server_t *s, double timeout_s) {
  if (s == nullptr) return HSMA_ERR_INVALID_ARG;
  const auto until = Clock::now() + std::chrono::microseconds((long long)(timeout_s * 1e6));
  std::unique_lock<std::mutex> lk(s->mu);
  while (s->n_done.load() < s->n_sub.load()) {
    if (timeout_s > 0 && Clock::now() >= until) return HSMA_ERR_TIMEOUT;
    s->cv.wait_for(lk, std::chrono::milliseconds(1));
  }
  return HSMA_OK;
}

HSMA_API hsma_status_t hsma_server_stats(hsma_server_t *s, hsma_server_stats_t *out) {
  if (s == nullptr || out == nullptr) return HSMA_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  out->submitted = s->n_sub.load();
  out->admitted = s->n_adm.load();
  out->completed = s->n_done.load();
  out->bytes_in_use = s->in_use;
  out->peak_bytes_in_use = s->peak;
  out->budget_bytes = s->budget;
  out->batched_launches = s->n_batched.load();
  out->blocked_launches = s->n_blocked.load();
  return HSMA_OK;
}

HSMA_API hsma_status_t hsma_server_destroy(hsma_server_t *s) {
  if (s == nullptr) return HSMA_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  if (!s->fake) {
    for (auto st : s->streams) {
      cudaStreamSynchronize(st);
      cudaStreamDestroy(st);
    }
    if (s->pool) cudaMemPoolDestroy(s->pool);
  }
  delete s;
  return HSMA_OK;
}

}  // extern "C"
