// Phase tracer (see trace.h): per-phase launch counts and device time.
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "trace.h"

namespace {

struct Pending {
  std::string phase;
  cudaEvent_t a, b;
};

struct Totals {
  double ms = 0.0;
  long long count = 0;
};

std::mutex g_mu;
std::atomic<int> g_enabled{-1};  // -1: not yet read from the environment
std::atomic<long long> g_launches{0};  // every kernel launched, traced or not
std::vector<Pending> g_open;  // indexed by slot
std::vector<int> g_free_slots;
std::vector<int> g_done;  // slots recorded, not yet folded into totals
std::map<std::string, Totals> g_totals;

bool enabled_locked() {
  if (g_enabled.load() < 0) {
    const char *e = std::getenv("HSMA_PHASE_TIMING");
    g_enabled.store((e != nullptr && e[0] == '1') ? 1 : 0);
  }
  return g_enabled.load() == 1;
}

// fold finished records into the totals (waits for their events)
void drain_locked() {
  for (int s : g_done) {
    Pending &p = g_open[s];
    float ms = 0.f;
    if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      Totals &t = g_totals[p.phase];
      t.ms += ms;
      t.count += 1;
    }
    g_free_slots.push_back(s);
  }
  g_done.clear();
}

}  // namespace

void hsma_count_launches(int kernels) { g_launches.fetch_add(kernels, std::memory_order_relaxed); }

HsmaTraceScope::HsmaTraceScope(const char *phase, cudaStream_t st, int kernels)
    : phase_(phase), st_(st), slot_(-1) {
  g_launches.fetch_add(kernels, std::memory_order_relaxed);
  if (g_enabled.load(std::memory_order_relaxed) == 0) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!enabled_locked()) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
  if (g_free_slots.empty()) {
    if (g_open.size() >= 65536) drain_locked();
    if (g_free_slots.empty()) {
      Pending p;
      if (cudaEventCreate(&p.a) != cudaSuccess) return;
      if (cudaEventCreate(&p.b) != cudaSuccess) {
        cudaEventDestroy(p.a);
        return;
      }
      g_open.push_back(p);
      g_free_slots.push_back((int)g_open.size() - 1);
    }
  }
  slot_ = g_free_slots.back();
  g_free_slots.pop_back();
  g_open[slot_].phase = phase;
  cudaEventRecord(g_open[slot_].a, st);
}

HsmaTraceScope::~HsmaTraceScope() {
  if (slot_ < 0) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEventRecord(g_open[slot_].b, st_);
  g_done.push_back(slot_);
}

extern "C" {

HSMA_API hsma_status_t hsma_trace_enable(int on) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_enabled.store(on ? 1 : 0);
  return HSMA_OK;
}

HSMA_API hsma_status_t hsma_trace_read(const char *phase, double *total_ms, long long *count) {
  if (phase == nullptr || total_ms == nullptr || count == nullptr) return HSMA_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  drain_locked();
  auto it = g_totals.find(phase);
  *total_ms = it == g_totals.end() ? 0.0 : it->second.ms;
  *count = it == g_totals.end() ? 0 : it->second.count;
  return HSMA_OK;
}

HSMA_API long long hsma_trace_launches(void) { return g_launches.load(); }

HSMA_API void hsma_trace_reset(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  drain_locked();
  g_totals.clear();
  g_launches.store(0);
}

}  // extern "C"
