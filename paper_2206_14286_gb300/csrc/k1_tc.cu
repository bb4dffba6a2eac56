// k1_tc.cu -- tensor-core PartialReduce (placeholder until the tcgen05 kernel lands).
#include "common.cuh"
#include "kernels.h"

namespace tpuknn {
cudaError_t launch_k1_tc(const K1Plan&, const void*, const float*, const float*, const void*,
                         const float*, Partials, cudaStream_t) {
  return cudaErrorNotSupported;
}
bool k1_tc_take_timeout() { return false; }
}  // namespace tpuknn
