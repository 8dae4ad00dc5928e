#include "blocked.h"
hsma_status_t hsma_blocked_solve(int, int, const void *, int64_t, void *, int64_t, int64_t, int64_t, const double *,
                                 int, cudaStream_t) {
  return HSMA_ERR_UNSUPPORTED;
}
