// internal.cuh -- buffer layouts, device status word and launcher declarations
// shared by the translation units of libgattn.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "geom.cuh"

namespace gattn {

constexpr size_t kAlign = 256;
__host__ __device__ inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Saved state written by the forward, read by the backward.
//   lse2 : float[S]     log2-domain log-sum-exp of every (tile, row) slot
//   ot   : float[S * d] per-tile output O_t of rows covered by >1 tile
// S = B * nh * ntiles * per_tile (box-ordered slots, see geom.cuh).
struct SavedLayout {
  size_t S, lse_off, ot_off, bytes;
};
inline SavedLayout saved_layout(const Geom& g) {
  SavedLayout s;
  s.S = (size_t)g.B * g.nh * g.ntiles * g.per_tile;
  s.lse_off = 0;
  s.ot_off = align_up(s.S * sizeof(float));
  s.bytes = s.ot_off + align_up(s.S * g.d * sizeof(float));
  return s;
}

// Backward workspace.
//   lse2c : float[S]      -(log2-domain LSE - log2(w_t / sum w)) (folds the dO_t scaling into P), negated
//   dd    : float[S]      -D, D = dOut . O_t per slot, negated
//   dq_s, dk_s, dv_s : float[S * d]  per-tile gradients of multiply-covered rows
//   ext   : 16 B[S]       BF16 row (x0, x1, x2, y0, y1, y2, 0, 0) per slot: x0 + x1 + x2 = -lse' / (scale
//                          log2 e) and y0 + y1 + y2 = -D, each split into three BF16 terms; the BF16
//                          dK/dV kernels add both to S^T and dP^T with one extra K = 16 MMA step each
struct BwdLayout {
  size_t S, lse_off, dd_off, ext_off, dq_off, dk_off, dv_off, bytes;
};
inline BwdLayout bwd_layout(const Geom& g) {
  BwdLayout b;
  b.S = (size_t)g.B * g.nh * g.ntiles * g.per_tile;
  size_t vec = align_up(b.S * sizeof(float));
  size_t mat = align_up(b.S * g.d * sizeof(float));
  b.lse_off = 0;
  b.dd_off = vec;
  b.ext_off = 2 * vec;
  b.dq_off = 2 * vec + align_up(b.S * 16);
  b.dk_off = b.dq_off + mat;
  b.dv_off = b.dk_off + mat;
  b.bytes = b.dv_off + mat;
  return b;
}

// Device status codes (subset of gattn_status) set by kernels.
enum : uint32_t { kStatusOk = 0, kStatusTimeout = GATTN_ERR_TIMEOUT, kStatusBounds = GATTN_ERR_DEVICE_BOUNDS };

// One status word per translation unit; the ABI reads and clears all of them.
#define GATTN_DEFINE_STATUS(NAME)                                                       \
  static __device__ uint32_t g_status_word;                                             \
  static __device__ __forceinline__ void set_status(uint32_t code) {                    \
    atomicCAS(&g_status_word, 0u, code);                                                \
  }                                                                                     \
  namespace gattn {                                                                     \
  uint32_t fetch_status_##NAME() {                                                      \
    uint32_t v = 0, z = 0;                                                              \
    if (cudaMemcpyFromSymbol(&v, g_status_word, sizeof(v)) != cudaSuccess) return ~0u;  \
    if (v) cudaMemcpyToSymbol(g_status_word, &z, sizeof(z));                            \
    return v;                                                                           \
  }                                                                                     \
  }

uint32_t fetch_status_simt();
uint32_t fetch_status_merge();
uint32_t fetch_status_sm103_fwd();
uint32_t fetch_status_sm103_fwd64();
uint32_t fetch_status_sm103_bwd();
uint32_t fetch_status_sm103_bwd64();
uint32_t fetch_status_serve();
uint32_t fetch_status_compress();
uint32_t fetch_status_linear();

// ---- per-kernel device timing (gattn_profile_*); no-ops unless enabled
enum KernelId : int {
  kKFwdTiles = 0, kKMergeFwd, kKBwdPrep, kKBwdDkdv, kKBwdDq, kKMergeBwd, kKCompress, kKCompressCombine, kKGatedMix, kKDpsResidual, kKDpsUpdate, kKLinearSummary, kKLinearCombine,
  kKLinearQuery, kKLinearBwdQuery, kKLinearBwdCombine, kKLinearBwdKey, kKCount
};
void prof_begin(int kernel, cudaStream_t st);
void prof_end(int kernel, cudaStream_t st);

// Temporal compression (compress.cu): frames are split into `splits` ranges of
// `chunk` frames when the (b, h, 32-location block) units alone cannot fill the
// GPU; the partials then live in the caller's workspace:
//   acc [splits, B*nh, M, d] FP32, then (log2 max, sum) [splits, B*nh, M, 2] FP32.
struct CompressPlan {
  int splits, chunk, mblocks;
};
CompressPlan compress_plan(int B, int nh, int S, int M);
inline size_t compress_ws_bytes(int B, int nh, int S, int M, int d) {
  const CompressPlan p = compress_plan(B, nh, S, M);
  if (p.splits <= 1) return 0;
  return (size_t)p.splits * B * nh * M * (size_t)(d + 2) * sizeof(float);
}
cudaError_t launch_compress(const float* q, const void* k, const void* v, void* out, float* lse, float* ws, int B,
                            int nh, int S, int M, int d, bool in_bf16, bool out_bf16, float scale, cudaStream_t st);

// ---- launchers (return cudaGetLastError() of their launches)
cudaError_t launch_simt_fwd(const Geom& g, const float* q, const float* k, const float* v, void* out,
                            int out_dtype, float* lse2, float* ot, cudaStream_t st);
cudaError_t launch_simt_bwd(const Geom& g, const float* q, const float* k, const float* v,
                            const float* dout, const float* lse2c, const float* dd, void* dq, void* dk,
                            void* dv, int out_dtype, float* dq_s, float* dk_s, float* dv_s,
                            cudaStream_t st);
cudaError_t launch_merge_fwd(const Geom& g, const float* ot, void* out, int out_dtype, cudaStream_t st);
// factorised linear attention (linear.cu): split-N summary over chunks of
// 128-token tiles, fixed-order combine, query pass; BF16, d = 64.
struct LinearPlan {
  int ntiles, chunk_tiles, chunks, q_tiles_per_cta;
};
LinearPlan linear_plan(int B, int nh, int64_t N);
// Forward workspace: per-chunk FP32 partials of S and z, then the combined
// S^T as BF16 high and low parts ([BH, 64 (v), 64 (k)] each) and z (FP32
// [BH, 64]); the backward reads the last three.
struct LinearLayout {
  size_t part_S, part_z, sth, stl, z, bytes;
};
LinearLayout linear_layout(int B, int nh, int64_t N);
size_t linear_ws_bytes(int B, int nh, int64_t N);
cudaError_t launch_linear(const void* q, const void* k, const void* v, void* out, void* ws, int B, int nh, int64_t N,
                          cudaStream_t st);
// Backward workspace: per-chunk FP32 partials of the query-side gradient
// summary dS (64 x 64) and dz (64), then dS and dS^T as BF16 high and low
// parts and dz (FP32).
struct LinearBwdLayout {
  size_t part_dS, part_dz, dsh, dsl, dsth, dstl, dz, bytes;
};
LinearBwdLayout linear_bwd_layout(int B, int nh, int64_t N);
cudaError_t launch_linear_bwd(const void* q, const void* k, const void* v, const void* dout, const void* saved,
                              void* dq, void* dk, void* dv, void* ws, int B, int nh, int64_t N, cudaStream_t st);
// posterior-sampling step, elementwise parts (dps.cu)
cudaError_t launch_dps_residual(const Geom& g, const float* D, const float* y, const uint8_t* mask, void* r,
                                bool r_bf16, cudaStream_t st);
cudaError_t launch_dps_update(const Geom& g, float* z, void* zb, const float* D, const float* dq, const float* dk,
                              const float* dv, const float* eps, float sigma, float sigma_next, float lam,
                              cudaStream_t st);
// out <- gate[h] * out + (1 - gate[h]) * cross over [B, nh, N, d] (gated.cu)
cudaError_t launch_gated_mix(const Geom& g, void* out, const void* cross, const float* gate, int out_dtype,
                             cudaStream_t st);
cudaError_t launch_bwd_prep(const Geom& g, const void* out, int out_dtype, const void* dout,
                            int in_dtype, const float* lse2, const float* ot, float* lse2c, float* dd,
                            void* ext, cudaStream_t st);
cudaError_t launch_merge_bwd(const Geom& g, const float* dq_s, const float* dk_s, const float* dv_s,
                             void* dq, void* dk, void* dv, int out_dtype, cudaStream_t st);
cudaError_t launch_sm103_fwd(const Geom& g, const __nv_bfloat16* q, const __nv_bfloat16* k,
                             const __nv_bfloat16* v, void* out, int out_dtype, float* lse2, float* ot,
                             uint32_t flags, cudaStream_t st);
cudaError_t launch_sm103_fwd64(const Geom& g, const __nv_bfloat16* q, const __nv_bfloat16* k,
                               const __nv_bfloat16* v, void* out, int out_dtype, float* lse2, float* ot,
                               uint32_t flags, cudaStream_t st);
cudaError_t launch_sm103_bwd(const Geom& g, const __nv_bfloat16* q, const __nv_bfloat16* k,
                             const __nv_bfloat16* v, const __nv_bfloat16* dout, const float* lse2c,
                             const float* dd, const void* ext, void* dq, void* dk, void* dv, int out_dtype,
                             float* dq_s, float* dk_s, float* dv_s, uint32_t flags, cudaStream_t st);
cudaError_t launch_sm103_bwd64(const Geom& g, const __nv_bfloat16* q, const __nv_bfloat16* k,
                               const __nv_bfloat16* v, const __nv_bfloat16* dout, const float* lse2c,
                               const float* dd, const void* ext, void* dq, void* dk, void* dv, int out_dtype,
                               float* dq_s, float* dk_s, float* dv_s, cudaStream_t st);

// ---- ragged (multi-request) forward, used by the serving engine.
// One descriptor per active request, in device memory, sorted by item0: the
// request's token state z ([nh, N, d] BF16, Q = K = V = z), its geometry
// (B = 1) and TMA tensor map, its attention output and per-slot scratch.
struct alignas(128) ReqDesc {
  CUtensorMap tmap;      // over z, box of the geometry's block shape
  Geom g;
  __nv_bfloat16* z;      // state (read by the attention, updated by the step kernel)
  void* out;             // GPA(z) for rows covered by one tile (BF16)
  float* ot;             // per-slot FP32 outputs of multiply-covered rows
  int64_t tok0;          // first global (head, token) row of this request (step kernel)
  int item0;             // first global attention work item of this request
  int items;             // work items of the request (see the ragged launchers)
};
// counts[0] = number of requests, counts[1] = total attention work items,
// counts[2] = total (head, token) rows; read on the device so that one
// captured launch serves any active set.
// box_rows: the rows R of the box shape every request of the launch uses
// (items of a request with another shape are refused as bounds errors).
cudaError_t launch_sm103_fwd_ragged(const ReqDesc* reqs, const int64_t* counts, int d, int box_rows,
                                    cudaStream_t st);
// d = 64: the two-box kernel; its work items per (head, tile) are pairs of boxes
cudaError_t launch_sm103_fwd64_ragged(const ReqDesc* reqs, const int64_t* counts, int box_rows, cudaStream_t st);
int fwd64_ragged_items(const Geom& g);  // nh * ntiles * ceil(nbmax_tot / 2)
// warp_covers: the most tiles that cover a token, for the warp-per-32-rows
// form (at most kMaxCover); 0 selects one thread per 4 columns of a row
cudaError_t launch_serve_update(const ReqDesc* reqs, const int64_t* counts, int d, float c, int warp_covers,
                                cudaStream_t st);

// ---- small device helpers
#ifdef __CUDACC__
template <typename T>
__device__ __forceinline__ void store4(T* p, float4 v);
template <>
__device__ __forceinline__ void store4<float>(float* p, float4 v) {
  *reinterpret_cast<float4*>(p) = v;
}
template <>
__device__ __forceinline__ void store4<__nv_bfloat16>(__nv_bfloat16* p, float4 v) {
  __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y);
  __nv_bfloat162 b = __floats2bfloat162_rn(v.z, v.w);
  uint2 u;
  u.x = *reinterpret_cast<uint32_t*>(&a);
  u.y = *reinterpret_cast<uint32_t*>(&b);
  *reinterpret_cast<uint2*>(p) = u;
}
template <typename T>
__device__ __forceinline__ float4 load4(const T* p);
template <>
__device__ __forceinline__ float4 load4<float>(const float* p) {
  return __ldg(reinterpret_cast<const float4*>(p));
}
template <>
__device__ __forceinline__ float4 load4<__nv_bfloat16>(const __nv_bfloat16* p) {
  uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
  __nv_bfloat162 a = *reinterpret_cast<__nv_bfloat162*>(&u.x);
  __nv_bfloat162 b = *reinterpret_cast<__nv_bfloat162*>(&u.y);
  float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
  return make_float4(fa.x, fa.y, fb.x, fb.y);
}
#endif

}  // namespace gattn
