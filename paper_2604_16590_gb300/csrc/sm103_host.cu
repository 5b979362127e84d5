// sm103_host.cu -- host helpers of the tensor-core path: TMA tensor-map
// encoding (the driver entry point is resolved at run time, so the library
// does not link libcuda) and the choice of the 128-token block shape.
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

// Block shape (bt, by, bx), bt*by*bx = 128, each a power of two <= 256.  The
// attention work of a tile grows with the square of its block count, so the
// shape minimising sum_tiles NB_t^2 = prod_a sum_k ceil(e_a(k)/b_a)^2 (the sum
// factorises over dimensions) wins; ties go to the longest contiguous x run.
BlockShape choose_block_shape(const Geom& g) {
  BlockShape best{1, 1, 128};
  double best_cost = -1.0;
  for (int lt = 0; lt <= 7; ++lt)
    for (int ly = 0; ly + lt <= 7; ++ly) {
      const int lx = 7 - lt - ly;
      const int b[3] = {1 << lt, 1 << ly, 1 << lx};
      double cost = 1.0;
      for (int a = 0; a < 3; ++a) {
        double s = 0.0;
        for (int k = 0; k < g.n[a]; ++k) {
          int lo = k * g.c[a] - g.h[a], hi = (k + 1) * g.c[a] + g.h[a];
          lo = lo < 0 ? 0 : lo;
          hi = hi > g.G[a] ? g.G[a] : hi;
          const double nb = (double)((hi - lo + b[a] - 1) / b[a]);
          s += nb * nb;
        }
        cost *= s;
      }
      if (best_cost < 0 || cost < best_cost * (1 - 1e-12) || (cost <= best_cost * (1 + 1e-12) && b[2] > best.bx)) {
        best_cost = cost;
        best = BlockShape{b[0], b[1], b[2]};
      }
    }
  best.lt = __builtin_ctz(best.bt);
  best.ly = __builtin_ctz(best.by);
  best.lx = __builtin_ctz(best.bx);
  for (int a = 0; a < 3; ++a) {
    const int b = a == 0 ? best.bt : (a == 1 ? best.by : best.bx);
    best.nbmax[a] = (g.emax[a] + b - 1) / b;
  }
  return best;
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
