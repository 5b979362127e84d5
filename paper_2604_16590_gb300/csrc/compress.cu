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
// Kernel design.  A work item is 32 consecutive locations of one (b, h) over a
// range of frames.  Per frame, the keys (and the values) of those locations are
// one contiguous slab; a producer warp streams the slabs of successive frames
// into a ring of shared-memory stages with bulk asynchronous copies (TMA,
// completion on an mbarrier), ~190 KB in flight per SM, so that the HBM stream
// never waits on the arithmetic.  Eight consumer warps read the stages: eight
// lanes own one location (16-byte shared loads, a warp reads 512 contiguous
// bytes per instruction), and release the stage with one arrival per warp.
// Persistent CTAs (two per SM) take the items in a fixed stride.  The score is
// a group dot product (three xor shuffles).  Softmax is online in the log2
// domain with one rescale per stage.  The S-long sums are compensated by blocking: an inner
// accumulator covers at most 256 frames and is folded into the outer one at
// each block boundary, so the rounding error grows with 256 + S/256 instead
// of S.  When (b, h, location-block) units alone cannot fill the GPU, the
// frames are split into ranges whose partial (max, sum, accumulator) go to
// the workspace; a second kernel merges them in fixed split order
// (deterministic, no atomics).
#include <math.h>

#include "internal.cuh"
#include "sm103_ptx.cuh"

GATTN_DEFINE_STATUS(compress)

namespace gattn {
namespace {

constexpr int kThreadsC = 256;
constexpr int kLocPerBlock = 32;   // 8 warps x 4 locations
constexpr int kInner = 256;        // frames per inner (compensated) accumulation block
constexpr int kPersistentCtas = 152 * 2;  // two CTAs per SM
constexpr int kTargetItems = 152 * 32;
constexpr float kLn2 = 0.6931471805599453f;
constexpr float kLog2e = 1.4426950408889634f;

__device__ __forceinline__ float ex2f(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
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

__device__ void set_status_c(uint32_t c) { set_status(c); }

// Ring geometry per (input type, head dim): a slab is the 32 locations of one
// frame of one tensor; a stage holds FR frames of keys and values.
template <typename InT, int D>
struct Ring {
  static constexpr int kSlab = kLocPerBlock * D * (int)sizeof(InT);
  static constexpr int kFR = kSlab >= 8192 ? 1 : 8192 / kSlab;
  static constexpr int kStage = kFR * 2 * kSlab;
  static constexpr int kStages = 98304 / kStage;
  static constexpr int kBars = kStages * kStage;  // barrier block offset
  static constexpr int kSmem = kBars + 2 * kStages * 8 + 16;
};
constexpr int kConsumerWarps = 8;
constexpr int kThreadsT = 32 * (kConsumerWarps + 1);

// Element j of lane `sub` (chunk c, position i) is d-index c * 8 * CE + sub * CE + i:
// each 16-byte load of the eight lanes of a group covers 128 contiguous bytes.
template <typename InT, typename OutT, int D>
__global__ void __launch_bounds__(kThreadsT, 2) compress_kernel(const CArgs a) {
  using C = Chunk<InT>;
  using R = Ring<InT, D>;
  constexpr int CE = C::kE;
  constexpr int NC = D / (8 * CE);  // 16-byte chunks per lane and frame
  constexpr int E = NC * CE;        // elements per lane
  constexpr int FR = R::kFR;
  static_assert(NC >= 1 && D % (8 * CE) == 0, "head dim");
  static_assert(kInner % FR == 0, "inner block");

  extern __shared__ __align__(128) uint8_t smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + R::kBars);
  uint64_t* empty = full + R::kStages;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + R::kStages);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    for (int i = 0; i < R::kStages; ++i) {
      sm103::mbar_init(full + i, 1);
      sm103::mbar_init(empty + i, kConsumerWarps);
    }
    *abort_flag = 0;
    sm103::fence_mbar_init();
  }
  __syncthreads();
  const long long n_items = (long long)a.BH * a.mblocks * a.splits;
  const size_t fstride = (size_t)a.M * D;  // elements between consecutive frames

  if (warp == kConsumerWarps) {
    // ------------------------------------------------------------ producer
    if (lane != 0) return;
    uint32_t G = 0, armed = 0, par = 0;
    bool ok = true;
    for (long long item = blockIdx.x; item < n_items && ok; item += gridDim.x) {
      const int split = (int)(item % a.splits);
      const long long rest = item / a.splits;
      const int mb = (int)(rest % a.mblocks);
      const int bh = (int)(rest / a.mblocks);
      const int m0 = mb * kLocPerBlock;
      const int nval = min(kLocPerBlock, a.M - m0);
      const uint32_t slab = (uint32_t)(nval * D * (int)sizeof(InT));
      const int t0 = split * a.chunk, t1 = min(a.S, t0 + a.chunk);
      const InT* kb = static_cast<const InT*>(a.k) + ((size_t)bh * a.S * a.M + m0) * D;
      const InT* vb = static_cast<const InT*>(a.v) + ((size_t)bh * a.S * a.M + m0) * D;
      for (int t = t0; t < t1; t += FR, ++G) {
        const uint32_t st = G % R::kStages, n = G / R::kStages;
        if (!(ok = sm103::mbar_wait<set_status_c>(empty + st, (n & 1) ^ 1, abort_flag))) break;
        const int nf = min(FR, t1 - t);
        sm103::mbar_arrive_expect_tx(full + st, 2u * nf * slab);
        armed |= 1u << st;
        par = (par & ~(1u << st)) | ((n & 1) << st);
        uint8_t* dst = smem + st * R::kStage;
        for (int f = 0; f < nf; ++f) {
          sm103::bulk_load(dst + (2 * f) * R::kSlab, kb + (size_t)(t + f) * fstride, slab, full + st);
          sm103::bulk_load(dst + (2 * f + 1) * R::kSlab, vb + (size_t)(t + f) * fstride, slab, full + st);
        }
      }
    }
    if (!ok) {  // let every copy this thread issued land before the CTA exits
      for (int s = 0; s < R::kStages; ++s)
        if (armed & (1u << s)) sm103::mbar_wait<set_status_c>(full + s, (par >> s) & 1, abort_flag, false);
    }
    return;
  }

  // -------------------------------------------------------------- consumers
  const int sub = lane & 7, grp = lane >> 3;
  const int lm = warp * 4 + grp;  // location within the block
  uint32_t G = 0;
  bool ok = true;
  for (long long item = blockIdx.x; item < n_items && ok; item += gridDim.x) {
    const int split = (int)(item % a.splits);
    const long long rest = item / a.splits;
    const int mb = (int)(rest % a.mblocks);
    const int bh = (int)(rest / a.mblocks);
    const int h = bh % a.nh;
    const int m = mb * kLocPerBlock + lm;
    const bool valid = m < a.M;
    const int t0 = split * a.chunk, t1 = min(a.S, t0 + a.chunk);

    float qv[E];
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
      for (int i = 0; i < CE; ++i) qv[c * CE + i] = a.q[(size_t)h * D + c * 8 * CE + sub * CE + i] * a.sl2;

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

    int inner = 0;
    for (int t = t0; t < t1; t += FR, ++G) {
      const uint32_t st = G % R::kStages;
      if (!(ok = sm103::mbar_wait<set_status_c>(full + st, (G / R::kStages) & 1, abort_flag))) break;
      const int nf = min(FR, t1 - t);
      const uint8_t* src = smem + st * R::kStage + lm * D * (int)sizeof(InT) + sub * 16;
      float s[FR];
      uint4 vr[FR][NC];
#pragma unroll
      for (int f = 0; f < FR; ++f) {
        float acc = 0.f;
        if (f < nf) {
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            const uint4 kr = *reinterpret_cast<const uint4*>(src + (2 * f) * R::kSlab + c * 128);
            vr[f][c] = *reinterpret_cast<const uint4*>(src + (2 * f + 1) * R::kSlab + c * 128);
            float kf[CE];
            C::to_float(kr, kf);
#pragma unroll
            for (int i = 0; i < CE; ++i) acc = fmaf(qv[c * CE + i], kf[i], acc);
          }
        }
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        acc += __shfl_xor_sync(0xffffffffu, acc, 2);
        acc += __shfl_xor_sync(0xffffffffu, acc, 4);
        s[f] = f < nf ? acc : -INFINITY;
      }
      __syncwarp();
      if (lane == 0) sm103::mbar_arrive(empty + st);
      float mx = mi;
#pragma unroll
      for (int f = 0; f < FR; ++f) mx = fmaxf(mx, s[f]);
      const float al = ex2f(mi - mx);
      float p[FR], psum = 0.f;
#pragma unroll
      for (int f = 0; f < FR; ++f) {
        p[f] = f < nf ? ex2f(s[f] - mx) : 0.f;
        psum += p[f];
      }
      li = li * al + psum;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        float vf[FR][CE];
#pragma unroll
        for (int f = 0; f < FR; ++f) {
          if (f < nf)
            C::to_float(vr[f][c], vf[f]);
          else
#pragma unroll
            for (int i = 0; i < CE; ++i) vf[f][i] = 0.f;
        }
#pragma unroll
        for (int i = 0; i < CE; ++i) {
          float x = acci[c * CE + i] * al;
#pragma unroll
          for (int f = 0; f < FR; ++f) x = fmaf(p[f], vf[f][i], x);
          acci[c * CE + i] = x;
        }
      }
      mi = mx;
      inner += FR;
      if (inner >= kInner) {
        fold();
        inner = 0;
      }
    }
    if (!ok) break;
    fold();
    if (!valid) continue;

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
  using R = Ring<InT, D>;
  const long long items = (long long)a.BH * a.mblocks * a.splits;
  auto kern = compress_kernel<InT, OutT, D>;
  static bool attr = false;  // per instantiation
  if (!attr) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, R::kSmem) != cudaSuccess)
      return cudaErrorInvalidValue;
    attr = true;
  }
  const long long grid = items < kPersistentCtas ? items : kPersistentCtas;
  prof_begin(kKCompress, st);
  kern<<<(unsigned)grid, kThreadsT, R::kSmem, st>>>(a);
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
