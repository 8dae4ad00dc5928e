// Internal phase tracer: CUDA events around kernel launch sites, per named
// phase (off unless enabled through hsma_trace_enable or HSMA_PHASE_TIMING=1).
#pragma once
#include <cuda_runtime.h>

struct HsmaTraceScope {
  HsmaTraceScope(const char *phase, cudaStream_t st);
  ~HsmaTraceScope();
  const char *phase_;
  cudaStream_t st_;
  int slot_;
};
