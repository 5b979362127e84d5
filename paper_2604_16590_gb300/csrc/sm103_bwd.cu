// sm103_bwd.cu -- placeholder until the tcgen05 backward lands.
#include "internal.cuh"

GATTN_DEFINE_STATUS(sm103_bwd)

namespace gattn {
cudaError_t launch_sm103_bwd(const Geom&, const __nv_bfloat16*, const __nv_bfloat16*, const __nv_bfloat16*,
                             const __nv_bfloat16*, const float*, const float*, void*, void*, void*, int, float*,
                             float*, float*, uint32_t, cudaStream_t) {
  return cudaErrorNotSupported;
}
}  // namespace gattn
