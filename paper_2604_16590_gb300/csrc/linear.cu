// linear.cu -- factorised (kernelised) linear attention with phi = elu + 1:
//
//     S = sum_n phi(k_n) v_n^T (d x d),  z = sum_n phi(k_n),
//     out_i = phi(q_i)^T S / (phi(q_i)^T z).
//
// Not an operator of the paper (whose global attention is the tiled GPA): the
// textbook linear-complexity global attention with a fixed-size per-head
// summary and normaliser.  The feature map is the one of Katharopoulos et al.
// (2020).  BF16 inputs, d = 64.
//
// Three kernels, all HBM-bound:
//   la_summary_kernel  split-N summary: each CTA streams a chunk of 128-token
//                      K and V tiles (TMA, 128-byte swizzle) through a ring of
//                      shared-memory stages; four warps apply phi to the K tile
//                      in place (BF16, rows past N zeroed) and accumulate z in
//                      FP32; one thread issues S += phi(K)^T V on tcgen05
//                      (M = N = 64, both operands MN-major, K = 128 tokens)
//                      with the accumulator in TMEM; the CTA writes its FP32
//                      partial S and z.
//   la_combine_kernel  per (b, h), the chunk partials summed in fixed order
//                      with Kahan compensation; S^T split into BF16 high and
//                      low parts (S = hi + lo to ~2^-17) for the query pass.
//   la_query_kernel    per 128-token query tile: phi(Q) in place, the
//                      denominator phi(q) . z per row in FP32, O = phi(Q) S on
//                      tcgen05 (two MMAs: hi and lo parts of S), out = O / den.
#include <math.h>

#include "internal.cuh"
#include "sm103_common.cuh"
#include "sm103_ptx.cuh"

GATTN_DEFINE_STATUS(linear)

namespace gattn {
namespace {
using namespace sm103;

constexpr int kD = 64;
constexpr int kTile = 128;                 // tokens per tile
constexpr int kTileBytes = kTile * kD * 2;  // 16 KB, one TMA box
constexpr int kStagesS = 3;                 // summary ring: K + V per stage
constexpr int kThreadsL = 192;              // producer, issuer, 4 math warps
constexpr int kQStages = 2;

__device__ void set_status_l(uint32_t c) { set_status(c); }
#define LWAIT(bar, par) mbar_wait<set_status_l>((bar), (par), abort_flag)

__device__ __forceinline__ float phi_f(float x) { return x > 0.f ? x + 1.f : ex2(x * 1.4426950408889634f); }

// phi of the eight BF16 values of one 16-byte chunk, in place; the rounded
// values are also returned as floats.
__device__ __forceinline__ uint4 phi_chunk(uint4 u, bool valid, float (&f)[8]) {
  uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float a = valid ? phi_f(__uint_as_float(w[i] << 16)) : 0.f;
    const float b = valid ? phi_f(__uint_as_float(w[i] & 0xffff0000u)) : 0.f;
    w[i] = pack_bf16(a, b);
    f[2 * i] = __uint_as_float(w[i] << 16);
    f[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
  }
  return make_uint4(w[0], w[1], w[2], w[3]);
}

// 5-D tiled store shared -> global (bulk group); rows past the tensor's end are
// not written.
__device__ __forceinline__ void tma_store_5d(const CUtensorMap* m, const void* src, int c0, int c1, int c2, int c3,
                                             int c4) {
  asm volatile("cp.async.bulk.tensor.5d.global.shared::cta.bulk_group [%0, {%2, %3, %4, %5, %6}], [%1];" ::"l"(
                   reinterpret_cast<uint64_t>(m)),
               "r"(smem_u32(src)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// byte offset of 16-byte chunk c of row r in a 128-byte-swizzled tile
__device__ __forceinline__ uint32_t swz(int r, int c) { return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4)); }

struct SumArgs {
  int N, BH, ntiles, chunk_tiles;
  float* ws_S;  // [chunks, BH, 64, 64]
  float* ws_z;  // [chunks, BH, 64]
};

__global__ void __launch_bounds__(kThreadsL) la_summary_kernel(const __grid_constant__ CUtensorMap tk,
                                                               const __grid_constant__ CUtensorMap tv,
                                                               const SumArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStagesS * 2 * kTileBytes);
  uint64_t* kready = full + kStagesS;
  uint64_t* empty = kready + kStagesS;
  uint64_t* done = empty + kStagesS;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int chunk = blockIdx.x, bh = blockIdx.y;
  const int t0 = chunk * a.chunk_tiles, t1 = min(a.ntiles, t0 + a.chunk_tiles);
  if (threadIdx.x == 0) {
    for (int i = 0; i < kStagesS; ++i) {
      mbar_init(full + i, 1);
      mbar_init(kready + i, 4);
      mbar_init(empty + i, 1);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    fence_mbar_init();
    prefetch_tmap(&tk);
    prefetch_tmap(&tv);
  }
  if (warp == 1) {
    tmem_alloc(tslot, 64);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    if (lane == 0) {  // ------------------------------------------------ TMA producer
      uint32_t armed = 0, par = 0;
      bool ok = true;
      for (int t = t0, G = 0; t < t1; ++t, ++G) {
        const int st = G % kStagesS, n = G / kStagesS;
        if (!(ok = LWAIT(empty + st, (n & 1) ^ 1))) break;
        mbar_arrive_expect_tx(full + st, 2 * kTileBytes);
        armed |= 1u << st;
        par = (par & ~(1u << st)) | ((n & 1) << st);
        uint8_t* dst = smem + st * 2 * kTileBytes;
        tma_load_5d(dst, &tk, full + st, 0, t * kTile, 0, 0, bh);
        tma_load_5d(dst + kTileBytes, &tv, full + st, 0, t * kTile, 0, 0, bh);
      }
      if (!ok)
        for (int s = 0; s < kStagesS; ++s)
          if (armed & (1u << s)) mbar_wait<set_status_l>(full + s, (par >> s) & 1, abort_flag, false);
    }
  } else if (warp == 1) {
    if (lane == 0) {  // ------------------------------------------------ MMA issuer
      // S[64 x 64] += phi(K)^T V: A = phi(K) tile MN-major (M = d contiguous),
      // B = V tile MN-major (N = d contiguous); a K = 16 step is 16 token rows.
      constexpr uint32_t idS = idesc_bf16(64, 64, 1) | (1u << 15);  // A MN-major
      bool ok = true;
      for (int t = t0, G = 0; t < t1; ++t, ++G) {
        const int st = G % kStagesS, n = G / kStagesS;
        if (!(ok = LWAIT(kready + st, n & 1))) break;
        tc_fence_after();
        const uint32_t base = smem_u32(smem + st * 2 * kTileBytes);
        const uint64_t dA = sw128_desc(base, 16384, 1024), dB = sw128_desc(base + kTileBytes, 16384, 1024);
#pragma unroll
        for (int ks = 0; ks < kTile / 16; ++ks)
          umma_bf16(tmem, dmove(dA, ks * 2048), dmove(dB, ks * 2048), idS, (G > 0 || ks > 0) ? 1u : 0u);
        umma_commit(empty + st);
      }
      umma_commit(done);
      if (!ok) *abort_flag = 1;
    }
  } else {
    // ------------------------------------------------------------------ phi warps + epilogue
    const int quad = warp & 3;
    const int r = quad * 32 + lane;  // tile row (token) of this thread
    float zacc[kD];
#pragma unroll
    for (int i = 0; i < kD; ++i) zacc[i] = 0.f;
    bool ok = true;
    for (int t = t0, G = 0; t < t1; ++t, ++G) {
      const int st = G % kStagesS, n = G / kStagesS;
      if (!(ok = LWAIT(full + st, n & 1))) break;
      uint8_t* kt = smem + st * 2 * kTileBytes;
      const bool valid = t * kTile + r < a.N;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        uint4* p = reinterpret_cast<uint4*>(kt + swz(r, c));
        float f[8];
        *p = phi_chunk(*p, valid, f);
#pragma unroll
        for (int e = 0; e < 8; ++e) zacc[c * 8 + e] += f[e];
      }
      fence_proxy_async_smem();  // the tensor core reads what these threads wrote
      __syncwarp();
      if (lane == 0) mbar_arrive(kready + st);
    }
    // epilogue: S partial from TMEM (M = 64: rows 16q .. 16q+15 in lanes 0..15
    // of lane quadrant q), z partial reduced over the 128 rows in fixed order
    const bool got = ok && LWAIT(done, 0);
    tc_fence_after();
    uint32_t s0[32], s1[32];
    const uint32_t tq = tmem + ((uint32_t)(quad * 32) << 16);
    tmem_ld32(tq, s0);
    tmem_ld32(tq + 32, s1);
    tmem_wait_ld(s0);
    tmem_wait_ld(s1);
    const size_t part = (size_t)chunk * a.BH + bh;
    if (got && lane < 16) {
      float* dst = a.ws_S + (part * kD + quad * 16 + lane) * kD;
#pragma unroll
      for (int j = 0; j < 32; j += 4) {
        *reinterpret_cast<float4*>(dst + j) = make_float4(__uint_as_float(s0[j]), __uint_as_float(s0[j + 1]),
                                                          __uint_as_float(s0[j + 2]), __uint_as_float(s0[j + 3]));
        *reinterpret_cast<float4*>(dst + 32 + j) = make_float4(
            __uint_as_float(s1[j]), __uint_as_float(s1[j + 1]), __uint_as_float(s1[j + 2]), __uint_as_float(s1[j + 3]));
      }
    }
    // all stages are idle once `done` completed: reuse them for the z rows
    float* zbuf = reinterpret_cast<float*>(smem);
    if (got) {
#pragma unroll
      for (int i = 0; i < kD; ++i) zbuf[r * kD + i] = zacc[i];
    }
    asm volatile("bar.sync 1, 128;" ::: "memory");  // the four math warps only
    const int tid = threadIdx.x - 64;
    if (got && tid < kD) {
      float s = 0.f;
      for (int i = 0; i < kTile; ++i) s += zbuf[i * kD + tid];
      a.ws_z[part * kD + tid] = s;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 64);
  }
}

struct CombArgs {
  int BH, chunks;
  const float* ws_S;
  const float* ws_z;
  __nv_bfloat16* sth;  // [BH, 64 (v), 64 (k)] high part of S^T
  __nv_bfloat16* stl;  // low part
  float* zt;           // [BH, 64]
};

// grid (BH, ceil((64 * 64 + 64) / 256)): one summary entry per thread
__global__ void __launch_bounds__(256) la_combine_kernel(const CombArgs a) {
  const int bh = blockIdx.x;
  for (int e = blockIdx.y * 256 + threadIdx.x; e < kD * kD + kD; e += 256 * gridDim.y) {
    const bool is_z = e >= kD * kD;
    float sum = 0.f, comp = 0.f;  // Kahan
    for (int c = 0; c < a.chunks; ++c) {
      const size_t part = (size_t)c * a.BH + bh;
      const float x = is_z ? a.ws_z[part * kD + (e - kD * kD)] : a.ws_S[part * kD * kD + e];
      const float y = x - comp;
      const float t = sum + y;
      comp = (t - sum) - y;
      sum = t;
    }
    if (is_z) {
      a.zt[(size_t)bh * kD + (e - kD * kD)] = sum;
    } else {
      const int k = e / kD, v = e % kD;  // S[k][v] -> S^T[v][k]
      const __nv_bfloat16 hi = __float2bfloat16_rn(sum);
      const __nv_bfloat16 lo = __float2bfloat16_rn(sum - __bfloat162float(hi));
      a.sth[((size_t)bh * kD + v) * kD + k] = hi;
      a.stl[((size_t)bh * kD + v) * kD + k] = lo;
    }
  }
}

struct QArgs {
  int N, BH, ntiles, tiles_per_cta;
  const __nv_bfloat16* sth;
  const __nv_bfloat16* stl;
  const float* zt;
};

constexpr int kThreadsQ = 224;  // producer, issuer, 4 math warps, storer

__global__ void __launch_bounds__(kThreadsQ, 3) la_query_kernel(const __grid_constant__ CUtensorMap tq,
                                                             const __grid_constant__ CUtensorMap to, const QArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sHi = smem;                       // S^T high part, 64 rows x 128 B, swizzled
  uint8_t* sLo = smem + 8192;                // low part
  uint8_t* qst = smem + 16384;               // Q stages
  uint8_t* ost = qst + kQStages * kTileBytes;  // output staging tile (swizzled, TMA store)
  float* zs = reinterpret_cast<float*>(ost + kTileBytes);
  uint64_t* qfull = reinterpret_cast<uint64_t*>(zs + kD);
  uint64_t* aready = qfull + kQStages;
  uint64_t* qempty = aready + kQStages;
  uint64_t* ofull = qempty + kQStages;  // [2]: O double-buffered in TMEM
  uint64_t* ofree = ofull + 2;          // [2]
  uint64_t* sready = ofree + 2;
  uint64_t* staged = sready + 1;
  uint64_t* sfree = staged + 1;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sfree + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int bh = blockIdx.y;
  const int t0 = blockIdx.x * a.tiles_per_cta, t1 = min(a.ntiles, t0 + a.tiles_per_cta);
  if (threadIdx.x == 0) {
    for (int i = 0; i < kQStages; ++i) {
      mbar_init(qfull + i, 1);
      mbar_init(aready + i, 4);
      mbar_init(qempty + i, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(ofull + b, 1);
      mbar_init(ofree + b, 4);
    }
    mbar_init(sready, 4);
    mbar_init(staged, 4);
    mbar_init(sfree, 1);
    *abort_flag = 0;
    fence_mbar_init();
    prefetch_tmap(&tq);
    prefetch_tmap(&to);
  }
  if (warp == 1) {
    tmem_alloc(tslot, 128);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    if (lane == 0) {  // ------------------------------------------------ TMA producer
      uint32_t armed = 0, par = 0;
      bool ok = true;
      for (int t = t0, G = 0; t < t1; ++t, ++G) {
        const int st = G % kQStages, n = G / kQStages;
        if (!(ok = LWAIT(qempty + st, (n & 1) ^ 1))) break;
        mbar_arrive_expect_tx(qfull + st, kTileBytes);
        armed |= 1u << st;
        par = (par & ~(1u << st)) | ((n & 1) << st);
        tma_load_5d(qst + st * kTileBytes, &tq, qfull + st, 0, t * kTile, 0, 0, bh);
      }
      if (!ok)
        for (int s = 0; s < kQStages; ++s)
          if (armed & (1u << s)) mbar_wait<set_status_l>(qfull + s, (par >> s) & 1, abort_flag, false);
    }
  } else if (warp == 1) {
    if (lane == 0) {  // ------------------------------------------------ MMA issuer
      // O[128 x 64] = phi(Q) S: A = phi(Q) tile K-major, B = S^T rows (K-major),
      // the high and the low BF16 parts of S accumulated in turn.
      constexpr uint32_t idO = idesc_bf16(128, 64, 0);
      const uint64_t dHi = sw128_desc(smem_u32(sHi), 16, 1024), dLo = sw128_desc(smem_u32(sLo), 16, 1024);
      bool ok = LWAIT(sready, 0);
      for (int t = t0, G = 0; t < t1 && ok; ++t, ++G) {
        const int st = G % kQStages, n = G / kQStages;
        const int b = G & 1;
        if (!(ok = LWAIT(aready + st, n & 1))) break;
        if (G >= 2 && !(ok = LWAIT(ofree + b, ((G >> 1) - 1) & 1))) break;
        tc_fence_after();
        const uint64_t dA = sw128_desc(smem_u32(qst + st * kTileBytes), 16, 1024);
        const uint32_t tO = tmem + 64 * b;
#pragma unroll
        for (int ks = 0; ks < kD / 16; ++ks) umma_bf16(tO, dmove(dA, ks * 32), dmove(dHi, ks * 32), idO, ks > 0);
#pragma unroll
        for (int ks = 0; ks < kD / 16; ++ks) umma_bf16(tO, dmove(dA, ks * 32), dmove(dLo, ks * 32), idO, 1u);
        umma_commit(qempty + st);
        umma_commit(ofull + b);
      }
      if (!ok) *abort_flag = 1;
    }
  } else if (warp == 6) {
    if (lane == 0) {  // ------------------------------------------------ output store
      bool ok = true;
      for (int t = t0, G = 0; t < t1; ++t, ++G) {
        if (!(ok = LWAIT(staged, G & 1))) break;
        fence_proxy_async_smem();
        tma_store_5d(&to, ost, 0, t * kTile, 0, 0, bh);
        bulk_commit();
        bulk_wait_read();  // the staging tile may be rewritten once the store has read it
        mbar_arrive(sfree);
      }
      bulk_wait_all();
      if (!ok) *abort_flag = 1;
    }
  } else {
    // ------------------------------------------------------------------ phi, denominator, epilogue
    const int quad = warp & 3;
    const int r = quad * 32 + lane;  // tile row = TMEM lane
    const int tid = threadIdx.x - 64;
    // S^T parts into swizzled shared memory, z alongside
    for (int i = tid; i < 2 * 64 * 8; i += 128) {
      const int m = i >> 9, row = (i >> 3) & 63, c = i & 7;
      const __nv_bfloat16* src = (m ? a.stl : a.sth) + ((size_t)bh * kD + row) * kD + c * 8;
      *reinterpret_cast<uint4*>((m ? sLo : sHi) + swz(row, c)) = *reinterpret_cast<const uint4*>(src);
    }
    if (tid < kD) zs[tid] = a.zt[(size_t)bh * kD + tid];
    fence_proxy_async_smem();
    asm volatile("bar.sync 1, 128;" ::: "memory");  // z visible to all four math warps
    __syncwarp();
    if (lane == 0) mbar_arrive(sready);
    // phi of tile G + 1 runs while the tensor core computes tile G
    auto phi_tile = [&](int G, float& den) -> bool {
      const int st = G % kQStages, n = G / kQStages;
      if (!LWAIT(qfull + st, n & 1)) return false;
      uint8_t* qt = qst + st * kTileBytes;
      den = 0.f;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        uint4* p = reinterpret_cast<uint4*>(qt + swz(r, c));
        float f[8];
        *p = phi_chunk(*p, true, f);
#pragma unroll
        for (int e = 0; e < 8; ++e) den = fmaf(f[e], zs[c * 8 + e], den);
      }
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(aready + st);
      return true;
    };
    const int count = t1 - t0;
    float den_cur = 0.f, den_next = 0.f;
    bool ok = count <= 0 || phi_tile(0, den_cur);
    for (int G = 0; G < count && ok; ++G) {
      if (G + 1 < count && !(ok = phi_tile(G + 1, den_next))) break;
      const int b = G & 1;
      if (!(ok = LWAIT(ofull + b, (G >> 1) & 1))) break;
      tc_fence_after();
      uint32_t o0[32], o1[32];
      const uint32_t tl = tmem + ((uint32_t)(quad * 32) << 16) + 64 * b;
      tmem_ld32(tl, o0);
      tmem_ld32(tl + 32, o1);
      tmem_wait_ld(o0);
      tmem_wait_ld(o1);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(ofree + b);
      // row r of the output tile into the staging buffer once the previous store read it
      if (G > 0 && !(ok = LWAIT(sfree, (G - 1) & 1))) break;
      const float inv = 1.f / den_cur;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const uint32_t* o = c < 4 ? o0 + 8 * c : o1 + 8 * (c - 4);
        *reinterpret_cast<uint4*>(ost + swz(r, c)) =
            make_uint4(pack_bf16(__uint_as_float(o[0]) * inv, __uint_as_float(o[1]) * inv),
                       pack_bf16(__uint_as_float(o[2]) * inv, __uint_as_float(o[3]) * inv),
                       pack_bf16(__uint_as_float(o[4]) * inv, __uint_as_float(o[5]) * inv),
                       pack_bf16(__uint_as_float(o[6]) * inv, __uint_as_float(o[7]) * inv));
      }
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(staged);
      den_cur = den_next;
    }
    (void)ok;
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 128);
  }
}

constexpr int kSumSmem = kStagesS * 2 * kTileBytes + 1024 + 256;
constexpr int kQSmem = 16384 + (kQStages + 1) * kTileBytes + 1024 + 512;

}  // namespace

LinearPlan linear_plan(int B, int nh, int64_t N) {
  LinearPlan p;
  p.ntiles = (int)((N + kTile - 1) / kTile);
  const int64_t units = (int64_t)p.ntiles * B * nh;
  int64_t ct = (units + 304 * 4 - 1) / (304 * 4);
  if (ct < 1) ct = 1;
  p.chunk_tiles = (int)ct;
  p.chunks = (int)((p.ntiles + ct - 1) / ct);
  p.q_tiles_per_cta = 16;
  return p;
}

size_t linear_ws_bytes(int B, int nh, int64_t N) {
  const LinearPlan p = linear_plan(B, nh, N);
  const size_t BH = (size_t)B * nh;
  return align_up((size_t)p.chunks * BH * kD * kD * 4) + align_up((size_t)p.chunks * BH * kD * 4) +
         2 * align_up(BH * kD * kD * 2) + align_up(BH * kD * 4);
}

cudaError_t launch_linear(const void* q, const void* k, const void* v, void* out, void* ws, int B, int nh, int64_t N,
                          cudaStream_t st) {
  const LinearPlan p = linear_plan(B, nh, N);
  const int BH = B * nh;
  char* w = static_cast<char*>(ws);
  SumArgs sa;
  sa.N = (int)N;
  sa.BH = BH;
  sa.ntiles = p.ntiles;
  sa.chunk_tiles = p.chunk_tiles;
  sa.ws_S = reinterpret_cast<float*>(w);
  w += align_up((size_t)p.chunks * BH * kD * kD * 4);
  sa.ws_z = reinterpret_cast<float*>(w);
  w += align_up((size_t)p.chunks * BH * kD * 4);
  CombArgs ca;
  ca.BH = BH;
  ca.chunks = p.chunks;
  ca.ws_S = sa.ws_S;
  ca.ws_z = sa.ws_z;
  ca.sth = reinterpret_cast<__nv_bfloat16*>(w);
  w += align_up((size_t)BH * kD * kD * 2);
  ca.stl = reinterpret_cast<__nv_bfloat16*>(w);
  w += align_up((size_t)BH * kD * kD * 2);
  ca.zt = reinterpret_cast<float*>(w);
  QArgs qa;
  qa.N = (int)N;
  qa.BH = BH;
  qa.ntiles = p.ntiles;
  qa.tiles_per_cta = p.q_tiles_per_cta;
  qa.sth = ca.sth;
  qa.stl = ca.stl;
  qa.zt = ca.zt;

  CUtensorMap mq, mk, mv, mo;
  if (!make_tmap_5d(&mq, q, kD, (int)N, 1, 1, BH, kTile, 1, 1) || !make_tmap_5d(&mo, out, kD, (int)N, 1, 1, BH, kTile, 1, 1) ||
      !make_tmap_5d(&mk, k, kD, (int)N, 1, 1, BH, kTile, 1, 1) || !make_tmap_5d(&mv, v, kD, (int)N, 1, 1, BH, kTile, 1, 1))
    return cudaErrorInvalidValue;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(la_summary_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSumSmem) != cudaSuccess ||
        cudaFuncSetAttribute(la_query_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kQSmem) != cudaSuccess)
      return cudaErrorInvalidValue;
    attr = true;
  }
  prof_begin(kKLinearSummary, st);
  la_summary_kernel<<<dim3(p.chunks, BH), kThreadsL, kSumSmem, st>>>(mk, mv, sa);
  cudaError_t e = cudaGetLastError();
  prof_end(kKLinearSummary, st);
  if (e != cudaSuccess) return e;
  prof_begin(kKLinearCombine, st);
  la_combine_kernel<<<dim3(BH, (kD * kD + kD + 255) / 256), 256, 0, st>>>(ca);
  e = cudaGetLastError();
  prof_end(kKLinearCombine, st);
  if (e != cudaSuccess) return e;
  prof_begin(kKLinearQuery, st);
  la_query_kernel<<<dim3((p.ntiles + p.q_tiles_per_cta - 1) / p.q_tiles_per_cta, BH), kThreadsQ, kQSmem, st>>>(mq, mo,
                                                                                                             qa);
  e = cudaGetLastError();
  prof_end(kKLinearQuery, st);
  return e;
}

}  // namespace gattn
