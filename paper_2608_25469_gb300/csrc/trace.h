// Internal phase tracer: CUDA events around kernel launch sites, per named
// phase (off unless enabled through hsma_trace_enable or HSMA_PHASE_TIMING=1).
#pragma once
#include <cuda_runtime.h>

// `kernels`: the kernels the scope launches (0 for a scope around copies);
// the library's launch counter (hsma_trace_launches) adds them up.
struct HsmaTraceScope {
  HsmaTraceScope(const char *phase, cudaStream_t st, int kernels = 1);
  ~HsmaTraceScope();
  const char *phase_;
  cudaStream_t st_;
  int slot_;
};

// Kernel launches made outside any HsmaTraceScope, or beyond the count a
// scope was given.
void hsma_count_launches(int kernels);
