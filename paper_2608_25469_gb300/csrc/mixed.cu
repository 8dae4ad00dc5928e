#include "mixed.h"
hsma_status_t hsma_mixed_r32(int, int, const float *, int64_t, float *, int64_t, int64_t, int64_t, double, int,
                             cudaStream_t) {
  return HSMA_ERR_UNSUPPORTED;
}
hsma_status_t hsma_mixed_ir(int, const hsma_opts_t *, const double *, int64_t, double *, int64_t, int64_t, int64_t,
                            double, int, cudaStream_t, hsma_info_t *) {
  return HSMA_ERR_UNSUPPORTED;
}
