// Tensor-core products (tcgen05 + TMA).  Not built yet: reports unavailable.
#include "tc.h"

namespace gsvdr {

bool tc_available(int) { return false; }
cudaError_t tc_gemm_gx(int, const float*, int64_t, int64_t, int64_t, const float*, int64_t, int, float*,
                       int64_t, double*, cudaStream_t) {
  return cudaErrorNotSupported;
}
int tc_gx_ctas(int64_t) { return 1; }
cudaError_t tc_gemm_gtq(int, const float*, int64_t, int64_t, int64_t, const float*, int64_t, int, float*,
                        int64_t, int*, int64_t, cudaStream_t) {
  return cudaErrorNotSupported;
}
int64_t tc_gtq_part_elems(int64_t, int64_t, int) { return 0; }

}  // namespace gsvdr
