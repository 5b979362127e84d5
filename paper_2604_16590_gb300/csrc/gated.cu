// gated.cu -- noise-gated mixing of spatial self-attention and current <->
// temporal cross-attention (arXiv 2604.16590, Sec. III-B, the noise-gated
// attention paragraph): every STORM-DiT layer runs self-attention on the
// current state and cross-attention from the current state to the compressed
// temporal representation, and weights the two with a gate driven by the
// diffusion noise level (more temporal weight at high noise).  Both attentions
// are the tile-local GPA operator; this file holds the final per-head blend
//
//     out = g_h * self + (1 - g_h) * cross,
//
// one elementwise pass (HBM-bound: reads two tensors, writes one).
#include "internal.cuh"

namespace gattn {
namespace {

constexpr int kThreadsG = 256;

template <typename T>
struct Vec8;
template <>
struct Vec8<__nv_bfloat16> {
  static constexpr int kN = 8;  // elements per 16-byte vector
  __device__ __forceinline__ static void load(const void* p, float* f) {
    const uint4 u = *reinterpret_cast<const uint4*>(p);
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      f[2 * i] = __uint_as_float(w[i] << 16);
      f[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
    }
  }
  __device__ __forceinline__ static void store(void* p, const float* f) {
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const __nv_bfloat162 h = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);
      w[i] = *reinterpret_cast<const uint32_t*>(&h);
    }
    *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
  }
};
template <>
struct Vec8<float> {
  static constexpr int kN = 4;
  __device__ __forceinline__ static void load(const void* p, float* f) {
    const float4 u = *reinterpret_cast<const float4*>(p);
    f[0] = u.x;
    f[1] = u.y;
    f[2] = u.z;
    f[3] = u.w;
  }
  __device__ __forceinline__ static void store(void* p, const float* f) {
    *reinterpret_cast<float4*>(p) = make_float4(f[0], f[1], f[2], f[3]);
  }
};

// out (holding the self-attention result) <- g_h out + (1 - g_h) cross, one
// 16-byte vector per thread and iteration.
template <typename T>
__global__ void __launch_bounds__(kThreadsG) gated_mix_kernel(T* __restrict__ out, const T* __restrict__ cross,
                                                              const float* __restrict__ gate, int64_t per_head,
                                                              int nh, int64_t nvec) {
  constexpr int V = Vec8<T>::kN;
  for (int64_t i = (int64_t)blockIdx.x * kThreadsG + threadIdx.x; i < nvec; i += (int64_t)gridDim.x * kThreadsG) {
    const int64_t e = i * V;
    const int h = (int)((e / per_head) % nh);
    const float g = gate[h];
    float a[V], b[V];
    Vec8<T>::load(out + e, a);
    Vec8<T>::load(cross + e, b);
#pragma unroll
    for (int j = 0; j < V; ++j) a[j] = fmaf(g, a[j] - b[j], b[j]);
    Vec8<T>::store(out + e, a);
  }
}

}  // namespace

cudaError_t launch_gated_mix(const Geom& g, void* out, const void* cross, const float* gate, int out_dtype,
                             cudaStream_t st) {
  const int64_t per_head = (int64_t)g.N * g.d;
  const int64_t total = (int64_t)g.B * g.nh * per_head;
  const int V = out_dtype == GATTN_BF16 ? 8 : 4;
  const int64_t nvec = total / V;  // d is a multiple of 8
  int64_t blocks = (nvec + kThreadsG - 1) / kThreadsG;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (out_dtype == GATTN_BF16)
    gated_mix_kernel<__nv_bfloat16><<<(unsigned)blocks, kThreadsG, 0, st>>>(
        static_cast<__nv_bfloat16*>(out), static_cast<const __nv_bfloat16*>(cross), gate, per_head, g.nh, nvec);
  else
    gated_mix_kernel<float><<<(unsigned)blocks, kThreadsG, 0, st>>>(static_cast<float*>(out),
                                                                     static_cast<const float*>(cross), gate,
                                                                     per_head, g.nh, nvec);
  return cudaGetLastError();
}

}  // namespace gattn
