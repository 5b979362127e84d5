// sm103_host.cu -- host helpers of the tensor-core path: TMA tensor-map
// encoding (the driver entry point is resolved at run time, so the library
// does not link libcuda) and the SM count.
#include <mutex>

#include "internal.cuh"
#include "sm103_common.cuh"

namespace gattn {

namespace {
using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeFn encode_fn() {
  static EncodeFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeFn>(p);
  });
  return fn;
}
}  // namespace

bool make_tmap_5d(CUtensorMap* map, const void* base, int d, int X, int Y, int T, int BH, int bx, int by, int bt) {
  EncodeFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[5] = {(cuuint64_t)d, (cuuint64_t)X, (cuuint64_t)Y, (cuuint64_t)T, (cuuint64_t)BH};
  const cuuint64_t row = (cuuint64_t)d * 2;
  const cuuint64_t strides[4] = {row, row * X, row * X * Y, row * X * Y * T};
  const cuuint32_t box[5] = {64u, (cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bt, 1u};
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

int num_sms() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
  }
  return n;
}

}  // namespace gattn
