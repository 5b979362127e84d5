// dps.cu -- the elementwise parts of one diffusion-posterior-sampling step with
// the GPA denoiser (arXiv 2604.16590, Sec. III-A: reverse SDE, score
// decomposition, DPS likelihood score, Eq. denoise).  The step is
//
//     D      = GPA(z, z, z)                       (tile kernels + merge)
//     r      = H^T (H D - y)                      (dps_residual_kernel; H a token mask)
//     J^T r  = dq + dk + dv of GPA at (z, z, z)   (backward kernels with dOut = r)
//     S      = (D - z) / sigma^2 - lam J^T r      (prior + likelihood score)
//     z     <- z + delta S + sqrt(delta) eps,  delta = sigma^2 - sigma_next^2
//                                              (dps_update_kernel, Euler-Maruyama)
//
// Both kernels stream 16-byte vectors (HBM-bound).
#include "internal.cuh"

namespace gattn {
namespace {

constexpr int kThreadsD = 256;
constexpr int kMaxBlocks = 152 * 16;

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }

// r = mask[b, i] ? D - y : 0, in the attention's input dtype; four elements per thread.
template <typename InT>
__global__ void __launch_bounds__(kThreadsD) dps_residual_kernel(const float* __restrict__ D,
                                                                 const float* __restrict__ y,
                                                                 const uint8_t* __restrict__ mask,
                                                                 InT* __restrict__ r, int64_t N, int nh, int d,
                                                                 int64_t nvec) {
  for (int64_t i = (int64_t)blockIdx.x * kThreadsD + threadIdx.x; i < nvec; i += (int64_t)gridDim.x * kThreadsD) {
    const int64_t e = 4 * i;
    const int64_t tok = e / d;           // (b * nh + h) * N + t
    const int64_t t = tok % N;
    const int64_t b = tok / N / nh;
    const bool obs = mask[b * N + t] != 0;
    const float4 a = ld4(D + e), c = ld4(y + e);
    const float v[4] = {obs ? a.x - c.x : 0.f, obs ? a.y - c.y : 0.f, obs ? a.z - c.z : 0.f, obs ? a.w - c.w : 0.f};
    if constexpr (sizeof(InT) == 2) {
      const __nv_bfloat162 lo = __floats2bfloat162_rn(v[0], v[1]), hi = __floats2bfloat162_rn(v[2], v[3]);
      uint2 u;
      u.x = *reinterpret_cast<const uint32_t*>(&lo);
      u.y = *reinterpret_cast<const uint32_t*>(&hi);
      *reinterpret_cast<uint2*>(r + e) = u;
    } else {
      *reinterpret_cast<float4*>(r + e) = make_float4(v[0], v[1], v[2], v[3]);
    }
  }
}

// z <- z + delta ((D - z) / sigma^2 - lam (dq + dk + dv)) + sqrt(delta) eps; zb <- bf16(z).
__global__ void __launch_bounds__(kThreadsD) dps_update_kernel(float* __restrict__ z, __nv_bfloat16* __restrict__ zb,
                                                               const float* __restrict__ D,
                                                               const float* __restrict__ dq,
                                                               const float* __restrict__ dk,
                                                               const float* __restrict__ dv,
                                                               const float* __restrict__ eps, float inv_s2,
                                                               float lam, float delta, float sqrt_delta,
                                                               int64_t nvec) {
  for (int64_t i = (int64_t)blockIdx.x * kThreadsD + threadIdx.x; i < nvec; i += (int64_t)gridDim.x * kThreadsD) {
    const int64_t e = 4 * i;
    const float4 zz = ld4(z + e), dd = ld4(D + e), a = ld4(dq + e), b = ld4(dk + e), c = ld4(dv + e),
                 n = ld4(eps + e);
    const float zi[4] = {zz.x, zz.y, zz.z, zz.w}, di[4] = {dd.x, dd.y, dd.z, dd.w};
    const float gi[4] = {a.x + b.x + c.x, a.y + b.y + c.y, a.z + b.z + c.z, a.w + b.w + c.w};
    const float ni[4] = {n.x, n.y, n.z, n.w};
    float o[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float score = (di[j] - zi[j]) * inv_s2 - lam * gi[j];
      o[j] = fmaf(sqrt_delta, ni[j], fmaf(delta, score, zi[j]));
    }
    *reinterpret_cast<float4*>(z + e) = make_float4(o[0], o[1], o[2], o[3]);
    if (zb) {
      const __nv_bfloat162 lo = __floats2bfloat162_rn(o[0], o[1]), hi = __floats2bfloat162_rn(o[2], o[3]);
      uint2 u;
      u.x = *reinterpret_cast<const uint32_t*>(&lo);
      u.y = *reinterpret_cast<const uint32_t*>(&hi);
      *reinterpret_cast<uint2*>(zb + e) = u;
    }
  }
}

unsigned blocks_for(int64_t nvec) {
  int64_t b = (nvec + kThreadsD - 1) / kThreadsD;
  return (unsigned)(b < kMaxBlocks ? b : kMaxBlocks);
}

}  // namespace

cudaError_t launch_dps_residual(const Geom& g, const float* D, const float* y, const uint8_t* mask, void* r,
                                bool r_bf16, cudaStream_t st) {
  const int64_t nvec = (int64_t)g.B * g.nh * g.N * g.d / 4;
  if (r_bf16)
    dps_residual_kernel<__nv_bfloat16><<<blocks_for(nvec), kThreadsD, 0, st>>>(
        D, y, mask, static_cast<__nv_bfloat16*>(r), g.N, g.nh, g.d, nvec);
  else
    dps_residual_kernel<float><<<blocks_for(nvec), kThreadsD, 0, st>>>(D, y, mask, static_cast<float*>(r), g.N,
                                                                       g.nh, g.d, nvec);
  return cudaGetLastError();
}

cudaError_t launch_dps_update(const Geom& g, float* z, void* zb, const float* D, const float* dq, const float* dk,
                              const float* dv, const float* eps, float sigma, float sigma_next, float lam,
                              cudaStream_t st) {
  const int64_t nvec = (int64_t)g.B * g.nh * g.N * g.d / 4;
  const float delta = sigma * sigma - sigma_next * sigma_next;
  dps_update_kernel<<<blocks_for(nvec), kThreadsD, 0, st>>>(z, static_cast<__nv_bfloat16*>(zb), D, dq, dk, dv, eps,
                                                           1.f / (sigma * sigma), lam, delta, sqrtf(delta), nvec);
  return cudaGetLastError();
}

}  // namespace gattn
