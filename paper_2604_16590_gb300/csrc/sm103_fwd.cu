// sm103_fwd.cu -- placeholder until the tcgen05 forward lands.
#include "internal.cuh"

GATTN_DEFINE_STATUS(sm103_fwd)

namespace gattn {
cudaError_t launch_sm103_fwd(const Geom&, const __nv_bfloat16*, const __nv_bfloat16*, const __nv_bfloat16*, void*,
                             int, float*, float*, uint32_t, cudaStream_t) {
  return cudaErrorNotSupported;
}
}  // namespace gattn
