// compress.cu -- temporal compression of STORM-DiT (arXiv 2604.16590, Sec. III-B,
// the STORM-DiT architecture paragraph and Fig. 2(b)): the S history frames of
// every spatial location are folded into one token by cross-attention with a
// learned query per head,
//
//     out[b,h,m] = sum_t softmax_t(scale q_h . k[b,h,t,m]) v[b,h,t,m],
//
// the same primitive that aggregates the variable dimension (S = variables).
// Linear in S; every history token is read once: the pass is HBM-bound.
//
// Layout: k, v [B, nh, S, M, d] (location m contiguous within a frame), q [nh, d]
// FP32, out [B, nh, M, d], lse [B, nh, M] (natural log).
//
// Kernel design.  Eight lanes own one location (16-byte loads, the eight lanes
// of a group read 128 contiguous bytes per instruction, a warp four
// locations); a block of 256 threads streams 32 consecutive locations through
// a range of frames, four frames per step so that eight 16-byte loads per
// thread are in flight.  The score is a group dot product (three xor
// shuffles).  Softmax is online in the log2 domain with one rescale per
// four-frame step.  The S-long sums are compensated by blocking: an inner
// accumulator covers at most 256 frames and is folded into the outer one at
// each block boundary, so the rounding error grows with 256 + S/256 instead
// of S.  When (b, h, location-block) units alone cannot fill the GPU, the
// frames are split into ranges whose partial (max, sum, accumulator) go to
// the workspace; a second kernel merges them in fixed split order
// (deterministic, no atomics).
#include <math.h>

#include "internal.cuh"

namespace gattn {
namespace {

constexpr int kThreadsC = 256;
constexpr int kLocPerBlock = 32;   // 8 warps x 4 locations
constexpr int kInner = 256;        // frames per inner (compensated) accumulation block
constexpr int kTargetItems = 152 * 16;
constexpr float kLn2 = 0.6931471805599453f;
constexpr float kLog2e = 1.4426950408889634f;

__device__ __forceinline__ float ex2f(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ uint4 ld_stream(const void* p) {
  uint4 r;
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
               : "l"(p));
  return r;
}

// Elements of one 16-byte chunk as floats.
template <typename InT>
struct Chunk;
template <>
struct Chunk<__nv_bfloat16> {
  static constexpr int kE = 8;
  __device__ __forceinline__ static void to_float(const uint4& u, float* f) {
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      f[2 * i] = __uint_as_float(w[i] << 16);
      f[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
    }
  }
};
template <>
struct Chunk<float> {
  static constexpr int kE = 4;
  __device__ __forceinline__ static void to_float(const uint4& u, float* f) {
    f[0] = __uint_as_float(u.x);
    f[1] = __uint_as_float(u.y);
    f[2] = __uint_as_float(u.z);
    f[3] = __uint_as_float(u.w);
  }
};

template <typename T>
__device__ __forceinline__ void store_out(T* p, float x);
template <>
__device__ __forceinline__ void store_out<float>(float* p, float x) {
  *p = x;
}
template <>
__device__ __forceinline__ void store_out<__nv_bfloat16>(__nv_bfloat16* p, float x) {
  *p = __float2bfloat16_rn(x);
}

struct CArgs {
  const float* q;
  const void* k;
  const void* v;
  void* out;
  float* lse;
  float* ws_acc;  // [splits, B*nh, M, D] partial accumulators (splits > 1)
  float* ws_ml;   // [splits, B*nh, M, 2] partial (log2 max, sum)
  int BH, nh, S, M, splits, chunk, mblocks;
  float sl2;  // scale * log2(e)
};

// Element j of lane `sub` (chunk c, position i) is d-index c * 8 * CE + sub * CE + i:
// each load instruction of the eight lanes covers 128 contiguous bytes.
template <typename InT, typename OutT, int D>
__global__ void __launch_bounds__(kThreadsC) compress_kernel(const CArgs a) {
  using C = Chunk<InT>;
  constexpr int CE = C::kE;
  constexpr int NC = D / (8 * CE);  // 16-byte chunks per lane and frame
  constexpr int E = NC * CE;        // elements per lane
  constexpr int F = (NC <= 2) ? 4 : 2;  // frames per step
  static_assert(NC >= 1 && D % (8 * CE) == 0, "head dim");
  static_assert(kInner % F == 0, "inner block");

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int sub = lane & 7, grp = lane >> 3;
  const long long item = blockIdx.x;
  const int split = (int)(item % a.splits);
  const long long rest = item / a.splits;
  const int mb = (int)(rest % a.mblocks);
  const int bh = (int)(rest / a.mblocks);
  const int h = bh % a.nh;
  const int m_raw = mb * kLocPerBlock + warp * 4 + grp;
  const bool valid = m_raw < a.M;
  const int m = valid ? m_raw : a.M - 1;  // out-of-range groups stream a valid location and store nothing
  const int t0 = split * a.chunk;
  const int t1 = min(a.S, t0 + a.chunk);

  float qv[E];
#pragma unroll
  for (int c = 0; c < NC; ++c)
#pragma unroll
    for (int i = 0; i < CE; ++i) qv[c * CE + i] = a.q[(size_t)h * D + c * 8 * CE + sub * CE + i] * a.sl2;

  const size_t fstride = (size_t)a.M * D;  // elements between consecutive frames
  const InT* kp = static_cast<const InT*>(a.k) + ((size_t)bh * a.S * a.M + m) * D + sub * CE;
  const InT* vp = static_cast<const InT*>(a.v) + ((size_t)bh * a.S * a.M + m) * D + sub * CE;

  float mo = -INFINITY, lo = 0.f, acco[E];
  float mi = -INFINITY, li = 0.f, acci[E];
#pragma unroll
  for (int e = 0; e < E; ++e) acco[e] = acci[e] = 0.f;

  auto fold = [&]() {
    const float mn = fmaxf(mo, mi);
    const float fa = ex2f(mo - mn), fb = ex2f(mi - mn);
    lo = lo * fa + li * fb;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      acco[e] = acco[e] * fa + acci[e] * fb;
      acci[e] = 0.f;
    }
    mo = mn;
    mi = -INFINITY;
    li = 0.f;
  };

  int t = t0;
  int inner = 0;
  for (; t + F <= t1; t += F) {
    uint4 kr[F][NC], vr[F][NC];
#pragma unroll
    for (int f = 0; f < F; ++f)
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        kr[f][c] = ld_stream(kp + (size_t)(t + f) * fstride + c * 8 * CE);
        vr[f][c] = ld_stream(vp + (size_t)(t + f) * fstride + c * 8 * CE);
      }
    float s[F];
#pragma unroll
    for (int f = 0; f < F; ++f) {
      float acc = 0.f;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        float kf[CE];
        C::to_float(kr[f][c], kf);
#pragma unroll
        for (int i = 0; i < CE; ++i) acc = fmaf(qv[c * CE + i], kf[i], acc);
      }
      acc += __shfl_xor_sync(0xffffffffu, acc, 1);
      acc += __shfl_xor_sync(0xffffffffu, acc, 2);
      acc += __shfl_xor_sync(0xffffffffu, acc, 4);
      s[f] = acc;
    }
    float mx = mi;
#pragma unroll
    for (int f = 0; f < F; ++f) mx = fmaxf(mx, s[f]);
    const float al = ex2f(mi - mx);
    float p[F], psum = 0.f;
#pragma unroll
    for (int f = 0; f < F; ++f) {
      p[f] = ex2f(s[f] - mx);
      psum += p[f];
    }
    li = li * al + psum;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      float vf[F][CE];
#pragma unroll
      for (int f = 0; f < F; ++f) C::to_float(vr[f][c], vf[f]);
#pragma unroll
      for (int i = 0; i < CE; ++i) {
        float x = acci[c * CE + i] * al;
#pragma unroll
        for (int f = 0; f < F; ++f) x = fmaf(p[f], vf[f][i], x);
        acci[c * CE + i] = x;
      }
    }
    mi = mx;
    inner += F;
    if (inner == kInner) {
      fold();
      inner = 0;
    }
  }
  for (; t < t1; ++t) {  // ragged tail of the frame range
    uint4 kr[NC], vr[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      kr[c] = ld_stream(kp + (size_t)t * fstride + c * 8 * CE);
      vr[c] = ld_stream(vp + (size_t)t * fstride + c * 8 * CE);
    }
    float acc = 0.f;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      float kf[CE];
      C::to_float(kr[c], kf);
#pragma unroll
      for (int i = 0; i < CE; ++i) acc = fmaf(qv[c * CE + i], kf[i], acc);
    }
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    acc += __shfl_xor_sync(0xffffffffu, acc, 4);
    const float mx = fmaxf(mi, acc);
    const float al = ex2f(mi - mx), p = ex2f(acc - mx);
    li = li * al + p;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      float vf[CE];
      C::to_float(vr[c], vf);
#pragma unroll
      for (int i = 0; i < CE; ++i) acci[c * CE + i] = fmaf(p, vf[i], acci[c * CE + i] * al);
    }
    mi = mx;
  }
  if (t1 > t0) fold();
  if (!valid) return;

  const size_t loc = (size_t)bh * a.M + m;
  if (a.splits == 1) {
    const float inv = 1.f / lo;
    OutT* o = static_cast<OutT*>(a.out) + loc * D;
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
      for (int i = 0; i < CE; ++i) store_out<OutT>(o + c * 8 * CE + sub * CE + i, acco[c * CE + i] * inv);
    if (a.lse && sub == 0) a.lse[loc] = (mo + __log2f(lo)) * kLn2;
  } else {
    const size_t ploc = (size_t)split * a.BH * a.M + loc;
    float* w = a.ws_acc + ploc * D;
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
      for (int i = 0; i < CE; ++i) w[c * 8 * CE + sub * CE + i] = acco[c * CE + i];
    if (sub == 0) {
      a.ws_ml[2 * ploc] = mo;
      a.ws_ml[2 * ploc + 1] = lo;
    }
  }
}

// Merge of the per-split partials of every location, splits in ascending order.
template <typename OutT, int D>
__global__ void __launch_bounds__(kThreadsC) compress_combine_kernel(const CArgs a) {
  const long long gid = (long long)blockIdx.x * kThreadsC + threadIdx.x;
  const long long loc = gid / 8;
  const int sub = (int)(gid & 7);
  const long long nloc = (long long)a.BH * a.M;
  if (loc >= nloc) return;
  constexpr int E = D / 8;
  const size_t per_split = (size_t)a.BH * a.M;
  float mx = -INFINITY;
  for (int s = 0; s < a.splits; ++s) mx = fmaxf(mx, a.ws_ml[2 * (s * per_split + loc)]);
  float l = 0.f, acc[E];
#pragma unroll
  for (int e = 0; e < E; ++e) acc[e] = 0.f;
  for (int s = 0; s < a.splits; ++s) {
    const size_t p = s * per_split + loc;
    const float w = ex2f(a.ws_ml[2 * p] - mx);
    l += w * a.ws_ml[2 * p + 1];
    const float* src = a.ws_acc + p * D + sub * E;
#pragma unroll
    for (int e = 0; e < E; ++e) acc[e] = fmaf(w, src[e], acc[e]);
  }
  const float inv = 1.f / l;
  OutT* o = static_cast<OutT*>(a.out) + loc * D + sub * E;
#pragma unroll
  for (int e = 0; e < E; ++e) store_out<OutT>(o + e, acc[e] * inv);
  if (a.lse && sub == 0) a.lse[loc] = (mx + __log2f(l)) * kLn2;
}

template <typename InT, typename OutT, int D>
cudaError_t launch_t(const CArgs& a, cudaStream_t st) {
  const long long items = (long long)a.BH * a.mblocks * a.splits;
  prof_begin(kKCompress, st);
  compress_kernel<InT, OutT, D><<<(unsigned)items, kThreadsC, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  prof_end(kKCompress, st);
  if (e != cudaSuccess || a.splits == 1) return e;
  const long long threads = (long long)a.BH * a.M * 8;
  prof_begin(kKCompressCombine, st);
  compress_combine_kernel<OutT, D><<<(unsigned)((threads + kThreadsC - 1) / kThreadsC), kThreadsC, 0, st>>>(a);
  e = cudaGetLastError();
  prof_end(kKCompressCombine, st);
  return e;
}

template <typename InT, typename OutT>
cudaError_t launch_d(const CArgs& a, int d, cudaStream_t st) {
  switch (d) {
    case 32:
      if constexpr (sizeof(InT) == 4) return launch_t<InT, OutT, 32>(a, st);
      return cudaErrorInvalidValue;
    case 64:
      return launch_t<InT, OutT, 64>(a, st);
    case 128:
      return launch_t<InT, OutT, 128>(a, st);
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace

CompressPlan compress_plan(int B, int nh, int S, int M) {
  CompressPlan p;
  const long long mblocks = ((long long)M + kLocPerBlock - 1) / kLocPerBlock;
  const long long base = (long long)B * nh * mblocks;
  long long want = (kTargetItems + base - 1) / base;
  const long long cap = S / 64 > 1 ? S / 64 : 1;  // at least 64 frames per split
  if (want > cap) want = cap;
  if (want < 1) want = 1;
  long long chunk = ((long long)S + want - 1) / want;
  chunk = (chunk + 3) / 4 * 4;
  p.splits = (int)(((long long)S + chunk - 1) / chunk);
  p.chunk = (int)chunk;
  p.mblocks = (int)mblocks;
  return p;
}

cudaError_t launch_compress(const float* q, const void* k, const void* v, void* out, float* lse, float* ws, int B,
                            int nh, int S, int M, int d, bool in_bf16, bool out_bf16, float scale,
                            cudaStream_t st) {
  const CompressPlan p = compress_plan(B, nh, S, M);
  CArgs a;
  a.q = q;
  a.k = k;
  a.v = v;
  a.out = out;
  a.lse = lse;
  const size_t nloc = (size_t)B * nh * M;
  a.ws_acc = ws;
  a.ws_ml = ws ? ws + (size_t)p.splits * nloc * d : nullptr;
  a.BH = B * nh;
  a.nh = nh;
  a.S = S;
  a.M = M;
  a.splits = p.splits;
  a.chunk = p.chunk;
  a.mblocks = p.mblocks;
  a.sl2 = scale * kLog2e;
  if (in_bf16)
    return out_bf16 ? launch_d<__nv_bfloat16, __nv_bfloat16>(a, d, st) : launch_d<__nv_bfloat16, float>(a, d, st);
  return out_bf16 ? launch_d<float, __nv_bfloat16>(a, d, st) : launch_d<float, float>(a, d, st);
}

}  // namespace gattn
