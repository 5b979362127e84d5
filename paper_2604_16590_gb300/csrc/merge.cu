// merge.cu -- the Hann-weighted overlap average of STORM-GPA (arXiv 2604.16590,
// Sec. III-C "average denoised outputs in overlapping halos" + Hanning window)
// and its backward counterparts.  Shared by the BF16 and FP32 forms.
//
// The tile kernels write rows covered by a single tile straight into the
// output tensor and park the FP32 per-tile value of every multiply-covered row
// in a (tile, row) slot.  These kernels finish the multiply-covered tokens by
// visiting their covering tiles in ascending tile order (fixed order, no
// atomics: bitwise reproducible run to run).
#include "internal.cuh"
#include "merge_common.cuh"

GATTN_DEFINE_STATUS(merge)

namespace gattn {
namespace {

constexpr int kThreads = 256;

// Token position and, per dimension, the covering tile range and the clipped
// extended box origin/extents needed to find the token's row in each tile.
struct Cover {
  int p[3];
  int k0[3], k1[3];
};

__device__ __forceinline__ bool cover_of(const Geom& g, int64_t i, Cover& c) {
  token_pos(g, i, c.p);
  bool multi = false;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    cover_dim(g, a, c.p[a], c.k0[a], c.k1[a]);
    multi = multi || (c.k1[a] > c.k0[a]);
  }
  return multi;
}

// slot of grid position p in tile (k[0], k[1], k[2]) of batch*head bh
__device__ __forceinline__ int64_t slot_in_tile(const Geom& g, int bh, const int p[3], const int k[3]) {
  int e[3], l[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    int lo = k[a] * g.c[a] - g.h[a];
    int hi = (k[a] + 1) * g.c[a] + g.h[a];
    lo = lo < 0 ? 0 : lo;
    hi = hi > g.G[a] ? g.G[a] : hi;
    e[a] = hi - lo;
    l[a] = p[a] - lo;
  }
  const int tile = (k[0] * g.n[1] + k[1]) * g.n[2] + k[2];
  return slot_of(g, bh, tile, e, l);
}

// One thread per (batch*head, token, float4 of d).
template <typename OutT>
__global__ void __launch_bounds__(kThreads) merge_fwd_kernel(Geom g, const float* __restrict__ ot,
                                                             OutT* __restrict__ out) {
  const int F4 = g.d / 4;
  const int64_t total = (int64_t)g.B * g.nh * g.N * F4;
  for (int64_t idx = (int64_t)blockIdx.x * kThreads + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * kThreads) {
    const int f = (int)(idx % F4);
    const int64_t bi = idx / F4;
    const int bh = (int)(bi / g.N);
    const int64_t i = bi % g.N;
    Cover c;
    if (!cover_of(g, i, c)) continue;  // single-cover: written by the tile kernel
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    float wsum = 0.f;
    int k[3];
    for (k[0] = c.k0[0]; k[0] <= c.k1[0]; ++k[0])
      for (k[1] = c.k0[1]; k[1] <= c.k1[1]; ++k[1])
        for (k[2] = c.k0[2]; k[2] <= c.k1[2]; ++k[2]) {
          float w = tile_weight(g, c.p, k);
          float4 o = __ldg(reinterpret_cast<const float4*>(ot + slot_in_tile(g, bh, c.p, k) * g.d) + f);
          acc.x = fmaf(w, o.x, acc.x);
          acc.y = fmaf(w, o.y, acc.y);
          acc.z = fmaf(w, o.z, acc.z);
          acc.w = fmaf(w, o.w, acc.w);
          wsum += w;
        }
    const float inv = 1.f / wsum;
    store4<OutT>(out + bi * g.d + 4 * f, make_float4(acc.x * inv, acc.y * inv, acc.z * inv, acc.w * inv));
  }
}

// The same merge, one warp per 32 consecutive tokens.  Each lane lists its
// token's covering slots and weights (token_covers) and writes them into one
// of two shared-memory row lists (parity_offset): half-warp h reads the rows
// of the tokens of lanes h, h + 2, ... in turn, lane f of the half holding
// 16 bytes f of every row (contiguous 256-byte runs at d = 64; U = 2 more
// 16-byte units at d = 128).  The halves take their lists R rows at a time,
// all R loads issued before the weighted sums: how many rows are in flight no
// longer depends on how many tiles cover each token, and the kernel is bound
// by how many are.  Each token's rows come in ascending tile order and are
// summed in that order.
template <typename OutT, int MAXC, int U>
__global__ void __launch_bounds__(kThreads, 2)
    merge_fwd_warp_kernel(Geom g, const float* __restrict__ ot, OutT* __restrict__ out) {
  constexpr int R = (MAXC <= 4 ? 16 : 8) / U;  // 64 or 32 registers of rows in flight per lane, no spills
  constexpr int W = kThreads / 32;
  __shared__ float win[kWinMax];
  __shared__ RowRef rows[W][2][16 * MAXC];
  __shared__ float tinv[W][32];
  const WinTable tbl = build_win_table(g, win);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int f0 = lane & 15;
  const int64_t total = (int64_t)g.B * g.nh * g.N;
  const int F4 = g.d / 4;  // 8, 16 or 32
  const int64_t stride = (int64_t)gridDim.x * W * 32;
  const RowRef* list = rows[wid][lane >> 4];
  for (int64_t base = ((int64_t)blockIdx.x * W + wid) * 32; base < total; base += stride) {
    const int64_t idx = base + lane;
    int64_t slot[MAXC];
    float w[MAXC];
    int n = 0;
    float wsum = 0.f;
    if (idx < total) {
      n = token_covers(g, tbl, (int)(idx / g.N), idx % g.N, slot, w);
      if (n > MAXC) {  // the host chose MAXC from the largest cover count
        set_status(kStatusBounds);
        n = 0;
      }
#pragma unroll
      for (int c = 0; c < MAXC; ++c)
        if (c < n) wsum += w[c];
    }
    int len;
    RowRef* mine = rows[wid][lane & 1] + parity_offset(n, lane, len);
#pragma unroll
    for (int c = 0; c < MAXC; ++c)
      if (c < n) {
        RowRef e;
        e.p = ot + slot[c] * g.d;
        e.w = w[c];
        e.flags = lane | (c == n - 1 ? kRowLast : 0);
        mine[c] = e;
      }
    tinv[wid][lane] = 1.f / wsum;  // read only for tokens with rows
    __syncwarp();
    const int lmax = max(len, __shfl_xor_sync(0xffffffffu, len, 16));
    float4 acc[U];
#pragma unroll
    for (int u = 0; u < U; ++u) acc[u] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 1
    for (int e0 = 0; e0 < lmax; e0 += R) {
      const int nv = len - e0;  // rows of this half's list from e0 on
      float4 o[R][U];
#pragma unroll
      for (int j = 0; j < R; ++j)
        if (j < nv) {
          const float4* p = reinterpret_cast<const float4*>(row_addr(list + e0 + j));
#pragma unroll
          for (int u = 0; u < U; ++u)
            if (f0 + 16 * u < F4) o[j][u] = __ldg(p + f0 + 16 * u);
        }
#pragma unroll
      for (int j = 0; j < R; ++j) {
        if (j >= nv) break;
        float wr;
        int fl;
        row_weight_flags(list + e0 + j, wr, fl);
#pragma unroll
        for (int u = 0; u < U; ++u)
          acc[u] = make_float4(fmaf(wr, o[j][u].x, acc[u].x), fmaf(wr, o[j][u].y, acc[u].y),
                               fmaf(wr, o[j][u].z, acc[u].z), fmaf(wr, o[j][u].w, acc[u].w));
        if (fl & kRowLast) {
          const int owner = fl & 31;
          const float inv = tinv[wid][owner];
          OutT* dst = out + (base + owner) * g.d;
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int f = f0 + 16 * u;
            if (f < F4) store4<OutT>(dst + 4 * f, make_float4(acc[u].x * inv, acc[u].y * inv, acc[u].z * inv, acc[u].w * inv));
            acc[u] = make_float4(0.f, 0.f, 0.f, 0.f);
          }
        }
      }
    }
    __syncwarp();  // the lists are rewritten for the next 32 tokens
  }
}

// Input gradients of multiply-covered tokens, organised like
// merge_fwd_warp_kernel: each lane lists its token's covering slots in one of
// two shared-memory lists, and each half-warp reads the dQ, dK and dV rows of
// its list R slots at a time, all loads first, summing each token's per-tile
// gradients in ascending tile order.
template <typename OutT, int MAXC, int U>
__global__ void __launch_bounds__(kThreads, 2) merge_bwd_warp_kernel(Geom g, const float* __restrict__ dq_s,
                                                                  const float* __restrict__ dk_s,
                                                                  const float* __restrict__ dv_s, OutT* __restrict__ dq,
                                                                  OutT* __restrict__ dk, OutT* __restrict__ dv) {
  constexpr int R = 4 / U;
  constexpr int W = kThreads / 32;
  __shared__ float win[kWinMax];
  __shared__ RowRef rows[W][2][16 * MAXC];
  const WinTable tbl = build_win_table(g, win);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int f0 = lane & 15;
  const int64_t total = (int64_t)g.B * g.nh * g.N;
  const int F4 = g.d / 4;
  const int64_t stride = (int64_t)gridDim.x * W * 32;
  const RowRef* list = rows[wid][lane >> 4];
  for (int64_t base = ((int64_t)blockIdx.x * W + wid) * 32; base < total; base += stride) {
    const int64_t idx = base + lane;
    int64_t slot[MAXC];
    float w[MAXC];
    int n = 0;
    if (idx < total) {
      n = token_covers(g, tbl, (int)(idx / g.N), idx % g.N, slot, w);
      if (n > MAXC) {  // the host chose MAXC from the largest cover count
        set_status(kStatusBounds);
        n = 0;
      }
    }
    int len;
    RowRef* mine = rows[wid][lane & 1] + parity_offset(n, lane, len);
#pragma unroll
    for (int c = 0; c < MAXC; ++c)
      if (c < n) {
        RowRef e;
        e.p = reinterpret_cast<const void*>(slot[c] * g.d);  // element offset of the slot's rows
        e.w = 0.f;
        e.flags = lane | (c == n - 1 ? kRowLast : 0);
        mine[c] = e;
      }
    __syncwarp();
    const int lmax = max(len, __shfl_xor_sync(0xffffffffu, len, 16));
    float4 a[U], b[U], e[U];
#pragma unroll
    for (int u = 0; u < U; ++u) a[u] = b[u] = e[u] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 1
    for (int e0 = 0; e0 < lmax; e0 += R) {
      const int nv = len - e0;  // rows of this half's list from e0 on
      float4 x[R][U], y[R][U], z[R][U];
#pragma unroll
      for (int j = 0; j < R; ++j)
        if (j < nv) {
          const int64_t off = (int64_t)row_addr(list + e0 + j);
#pragma unroll
          for (int u = 0; u < U; ++u)
            if (f0 + 16 * u < F4) {
              x[j][u] = __ldg(reinterpret_cast<const float4*>(dq_s + off) + f0 + 16 * u);
              y[j][u] = __ldg(reinterpret_cast<const float4*>(dk_s + off) + f0 + 16 * u);
              z[j][u] = __ldg(reinterpret_cast<const float4*>(dv_s + off) + f0 + 16 * u);
            }
        }
#pragma unroll
      for (int j = 0; j < R; ++j) {
        if (j >= nv) break;
        float wr;
        int fl;
        row_weight_flags(list + e0 + j, wr, fl);
#pragma unroll
        for (int u = 0; u < U; ++u) {
          a[u].x += x[j][u].x; a[u].y += x[j][u].y; a[u].z += x[j][u].z; a[u].w += x[j][u].w;
          b[u].x += y[j][u].x; b[u].y += y[j][u].y; b[u].z += y[j][u].z; b[u].w += y[j][u].w;
          e[u].x += z[j][u].x; e[u].y += z[j][u].y; e[u].z += z[j][u].z; e[u].w += z[j][u].w;
        }
        if (fl & kRowLast) {
          const int64_t o0 = (base + (fl & 31)) * g.d;
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int f = f0 + 16 * u;
            if (f < F4) {
              store4<OutT>(dq + o0 + 4 * f, a[u]);
              store4<OutT>(dk + o0 + 4 * f, b[u]);
              store4<OutT>(dv + o0 + 4 * f, e[u]);
            }
            a[u] = b[u] = e[u] = make_float4(0.f, 0.f, 0.f, 0.f);
          }
        }
      }
    }
    __syncwarp();  // the lists are rewritten for the next 32 tokens
  }
}

// x as the sum of three BF16 terms (each the rounding of what the previous ones
// leave), exact to about 2^-24 |x|.
__device__ __forceinline__ void split3(float x, __nv_bfloat16& a, __nv_bfloat16& b, __nv_bfloat16& c) {
  a = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(a);
  b = __float2bfloat16_rn(r1);
  c = __float2bfloat16_rn(r1 - __bfloat162float(b));
}

// One 16-byte B-operand row (K = 8 BF16 values) of the BF16 dK/dV kernels:
// (x0, x1, x2, y0, y1, y2, 0, 0) with x0+x1+x2 = x and y0+y1+y2 = y.  With an
// A operand of ones in K-columns 0..2 (resp. 3..5) one extra MMA step adds x
// (resp. y) to every element of the row's S^T (resp. dP^T) column.
__device__ __forceinline__ uint4 stat_row(float x, float y) {
  __nv_bfloat16 v[8];
  split3(x, v[0], v[1], v[2]);
  split3(y, v[3], v[4], v[5]);
  v[6] = v[7] = __float2bfloat16_rn(0.f);
  uint4 r;
  uint32_t* w = reinterpret_cast<uint32_t*>(&r);
  for (int i = 0; i < 4; ++i)
    w[i] = (uint32_t)__bfloat16_as_ushort(v[2 * i]) | ((uint32_t)__bfloat16_as_ushort(v[2 * i + 1]) << 16);
  return r;
}

// Per (batch*head, tile, row) slot: fold the merge weight c = w_t / sum w into
// the log-sum-exp (lse' = lse2 - log2 c, so exp2(s - lse') = c P) and form
// D = dOut . O_t.  O_t is the output itself for single-cover rows, else the
// FP32 per-tile value saved by the forward.  Both are stored negated
// (-lse', -D) so that the backward kernels form exp2(s log2e + (-lse')) and
// dP + (-D) with single fused/packed instructions; with `ext` the slot's
// statistics row (stat_row) is written too.  Slots of a box that fall outside
// the tile get -lse' = -inf and -D = 0, so the tensor-core backward can run
// whole boxes without masking queries.  One thread per slot: consecutive slots
// of a box are consecutive tokens of a row, so a warp's 16-byte loads of its
// rows cover contiguous memory, and the geometry and merge weights are
// computed lane-parallel.
template <typename T>
__device__ __forceinline__ void load8(const T* p, float (&v)[8]);
template <>
__device__ __forceinline__ void load8<float>(const float* p, float (&v)[8]) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(p)), b = __ldg(reinterpret_cast<const float4*>(p) + 1);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}
template <>
__device__ __forceinline__ void load8<__nv_bfloat16>(const __nv_bfloat16* p, float (&v)[8]) {
  const uint4 u = __ldg(reinterpret_cast<const uint4*>(p));
  const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w[i]));
    v[2 * i] = f.x;
    v[2 * i + 1] = f.y;
  }
}

template <typename OutT, typename InT>
__global__ void __launch_bounds__(kThreads) bwd_prep_kernel(Geom g, const OutT* __restrict__ out,
                                                            const InT* __restrict__ dout,
                                                            const float* __restrict__ lse2,
                                                            const float* __restrict__ ot,
                                                            float* __restrict__ lse2c, float* __restrict__ dd,
                                                            uint4* __restrict__ ext) {
  __shared__ float win[kWinMax];
  const WinTable tbl = build_win_table(g, win);
  const int64_t S = (int64_t)g.B * g.nh * g.ntiles * g.per_tile;
  for (int64_t slot = (int64_t)blockIdx.x * kThreads + threadIdx.x; slot < S; slot += (int64_t)gridDim.x * kThreads) {
    const int64_t ut = slot / g.per_tile;
    const int within = (int)(slot - ut * g.per_tile);
    const int tile = (int)(ut % g.ntiles);
    const int bh = (int)(ut / g.ntiles);
    TileBox tb;
    tile_box(g, tile, tb);
    int lr[3];
    if (!slot_local(g, tb.e, within >> 7, within & 127, lr) || (within >> 7) >= g.nbmax_tot) {
      // padding slot of a box that sticks out of the tile: probability 0
      lse2c[slot] = -INFINITY;
      dd[slot] = 0.f;
      // finite (the extension MMA multiplies it by the other statistic's zero weights)
      if (ext) ext[slot] = stat_row(-1e30f, 0.f);
      continue;
    }
    const int64_t tok = grid_token(g, tb, lr);
    int p[3];
    token_pos(g, tok, p);
    const bool single = single_cover(g, p);
    const InT* a = dout + ((int64_t)bh * g.N + tok) * g.d;
    float part = 0.f;
    if (single) {
      const OutT* o = out + ((int64_t)bh * g.N + tok) * g.d;
      for (int c = 0; c < g.d; c += 8) {
        float x[8], y[8];
        load8<InT>(a + c, x);
        load8<OutT>(o + c, y);
#pragma unroll
        for (int e = 0; e < 8; ++e) part = fmaf(x[e], y[e], part);
      }
    } else {
      const float* o = ot + slot * g.d;
      for (int c = 0; c < g.d; c += 8) {
        float x[8], y[8];
        load8<InT>(a + c, x);
        load8<float>(o + c, y);
#pragma unroll
        for (int e = 0; e < 8; ++e) part = fmaf(x[e], y[e], part);
      }
    }
    float lc = lse2[slot];
    if (!single) {
      // c = w_t / sum over covering tiles of w
      Cover c;
      cover_of(g, tok, c);
      int kt[3];
      kt[0] = tile / (g.n[1] * g.n[2]);
      kt[1] = (tile / g.n[2]) % g.n[1];
      kt[2] = tile % g.n[2];
      float wt = table_weight(g, tbl, p, kt), ws = 0.f;
      int k[3];
      for (k[0] = c.k0[0]; k[0] <= c.k1[0]; ++k[0])
        for (k[1] = c.k0[1]; k[1] <= c.k1[1]; ++k[1])
          for (k[2] = c.k0[2]; k[2] <= c.k1[2]; ++k[2]) ws += table_weight(g, tbl, p, k);
      lc -= log2f(wt / ws);
    }
    lse2c[slot] = -lc;
    dd[slot] = -part;
    if (ext) ext[slot] = stat_row(-lc / g.scale_log2, -part);
  }
}

// Input gradients of multiply-covered tokens: ascending-tile sums of the
// per-tile FP32 gradients.
template <typename OutT>
__global__ void __launch_bounds__(kThreads) merge_bwd_kernel(Geom g, const float* __restrict__ dq_s,
                                                             const float* __restrict__ dk_s,
                                                             const float* __restrict__ dv_s, OutT* __restrict__ dq,
                                                             OutT* __restrict__ dk, OutT* __restrict__ dv) {
  const int F4 = g.d / 4;
  const int64_t total = (int64_t)g.B * g.nh * g.N * F4;
  for (int64_t idx = (int64_t)blockIdx.x * kThreads + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * kThreads) {
    const int f = (int)(idx % F4);
    const int64_t bi = idx / F4;
    const int bh = (int)(bi / g.N);
    const int64_t i = bi % g.N;
    Cover c;
    if (!cover_of(g, i, c)) continue;
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a, e = a;
    int k[3];
    for (k[0] = c.k0[0]; k[0] <= c.k1[0]; ++k[0])
      for (k[1] = c.k0[1]; k[1] <= c.k1[1]; ++k[1])
        for (k[2] = c.k0[2]; k[2] <= c.k1[2]; ++k[2]) {
          const int64_t off = slot_in_tile(g, bh, c.p, k) * g.d;
          float4 x = __ldg(reinterpret_cast<const float4*>(dq_s + off) + f);
          float4 y = __ldg(reinterpret_cast<const float4*>(dk_s + off) + f);
          float4 z = __ldg(reinterpret_cast<const float4*>(dv_s + off) + f);
          a.x += x.x; a.y += x.y; a.z += x.z; a.w += x.w;
          b.x += y.x; b.y += y.y; b.z += y.z; b.w += y.w;
          e.x += z.x; e.y += z.y; e.z += z.z; e.w += z.w;
        }
    store4<OutT>(dq + bi * g.d + 4 * f, a);
    store4<OutT>(dk + bi * g.d + 4 * f, b);
    store4<OutT>(dv + bi * g.d + 4 * f, e);
  }
}

inline unsigned grid_for(int64_t total) {
  int64_t blocks = (total + kThreads - 1) / kThreads;
  const int64_t cap = 152LL * 16 * 8;  // grid-stride beyond this
  return (unsigned)(blocks < cap ? (blocks > 0 ? blocks : 1) : cap);
}

}  // namespace

// grid of the warp-per-32-tokens kernels
inline unsigned grid_warp(int64_t tokens) {
  const int64_t blocks = (tokens + kThreads - 1) / kThreads;
  const int64_t cap = 152LL * 8;
  return (unsigned)(blocks < cap ? (blocks > 0 ? blocks : 1) : cap);
}

cudaError_t launch_merge_fwd(const Geom& g, const float* ot, void* out, int out_dtype, cudaStream_t st) {
  const int mc = max_covers(g);
  if (mc <= kMaxCover) {
    const unsigned grid = grid_warp((int64_t)g.B * g.nh * g.N);
    using bf = __nv_bfloat16;
    const bool b16 = out_dtype == GATTN_BF16, wide = g.d > 64;
    if (mc <= 2) {
      if (b16)
        wide ? merge_fwd_warp_kernel<bf, 2, 2><<<grid, kThreads, 0, st>>>(g, ot, static_cast<bf*>(out))
             : merge_fwd_warp_kernel<bf, 2, 1><<<grid, kThreads, 0, st>>>(g, ot, static_cast<bf*>(out));
      else
        wide ? merge_fwd_warp_kernel<float, 2, 2><<<grid, kThreads, 0, st>>>(g, ot, static_cast<float*>(out))
             : merge_fwd_warp_kernel<float, 2, 1><<<grid, kThreads, 0, st>>>(g, ot, static_cast<float*>(out));
    } else if (mc <= 4) {
      if (b16)
        wide ? merge_fwd_warp_kernel<bf, 4, 2><<<grid, kThreads, 0, st>>>(g, ot, static_cast<bf*>(out))
             : merge_fwd_warp_kernel<bf, 4, 1><<<grid, kThreads, 0, st>>>(g, ot, static_cast<bf*>(out));
      else
        wide ? merge_fwd_warp_kernel<float, 4, 2><<<grid, kThreads, 0, st>>>(g, ot, static_cast<float*>(out))
             : merge_fwd_warp_kernel<float, 4, 1><<<grid, kThreads, 0, st>>>(g, ot, static_cast<float*>(out));
    } else {
      if (b16)
        wide ? merge_fwd_warp_kernel<bf, kMaxCover, 2><<<grid, kThreads, 0, st>>>(g, ot, static_cast<bf*>(out))
             : merge_fwd_warp_kernel<bf, kMaxCover, 1><<<grid, kThreads, 0, st>>>(g, ot, static_cast<bf*>(out));
      else
        wide ? merge_fwd_warp_kernel<float, kMaxCover, 2><<<grid, kThreads, 0, st>>>(g, ot, static_cast<float*>(out))
             : merge_fwd_warp_kernel<float, kMaxCover, 1><<<grid, kThreads, 0, st>>>(g, ot, static_cast<float*>(out));
    }
    return cudaGetLastError();
  }
  const int64_t total = (int64_t)g.B * g.nh * g.N * (g.d / 4);
  if (out_dtype == GATTN_BF16)
    merge_fwd_kernel<__nv_bfloat16><<<grid_for(total), kThreads, 0, st>>>(g, ot, static_cast<__nv_bfloat16*>(out));
  else
    merge_fwd_kernel<float><<<grid_for(total), kThreads, 0, st>>>(g, ot, static_cast<float*>(out));
  return cudaGetLastError();
}

cudaError_t launch_bwd_prep(const Geom& g, const void* out, int out_dtype, const void* dout, int in_dtype,
                            const float* lse2, const float* ot, float* lse2c, float* dd, void* ext_,
                            cudaStream_t st) {
  uint4* ext = static_cast<uint4*>(ext_);
  const int64_t total = (int64_t)g.B * g.nh * g.ntiles * g.per_tile;  // one thread per slot
  const unsigned grid = grid_for(total);
  using bf = __nv_bfloat16;
  if (out_dtype == GATTN_BF16 && in_dtype == GATTN_BF16)
    bwd_prep_kernel<bf, bf><<<grid, kThreads, 0, st>>>(g, (const bf*)out, (const bf*)dout, lse2, ot, lse2c, dd, ext);
  else if (out_dtype == GATTN_BF16)
    bwd_prep_kernel<bf, float><<<grid, kThreads, 0, st>>>(g, (const bf*)out, (const float*)dout, lse2, ot, lse2c, dd, ext);
  else if (in_dtype == GATTN_BF16)
    bwd_prep_kernel<float, bf><<<grid, kThreads, 0, st>>>(g, (const float*)out, (const bf*)dout, lse2, ot, lse2c, dd, ext);
  else
    bwd_prep_kernel<float, float><<<grid, kThreads, 0, st>>>(g, (const float*)out, (const float*)dout, lse2, ot, lse2c, dd, ext);
  return cudaGetLastError();
}

cudaError_t launch_merge_bwd(const Geom& g, const float* dq_s, const float* dk_s, const float* dv_s, void* dq,
                             void* dk, void* dv, int out_dtype, cudaStream_t st) {
  using bf = __nv_bfloat16;
  const int mc = max_covers(g);
  if (mc <= kMaxCover) {
    const unsigned grid = grid_warp((int64_t)g.B * g.nh * g.N);
    const bool b16 = out_dtype == GATTN_BF16, wide = g.d > 64;
#define GATTN_MERGE_BWD(MC)                                                                                      \
  if (b16)                                                                                                       \
    wide ? merge_bwd_warp_kernel<bf, MC, 2><<<grid, kThreads, 0, st>>>(g, dq_s, dk_s, dv_s, (bf*)dq, (bf*)dk, (bf*)dv) \
         : merge_bwd_warp_kernel<bf, MC, 1><<<grid, kThreads, 0, st>>>(g, dq_s, dk_s, dv_s, (bf*)dq, (bf*)dk, (bf*)dv); \
  else                                                                                                           \
    wide ? merge_bwd_warp_kernel<float, MC, 2><<<grid, kThreads, 0, st>>>(g, dq_s, dk_s, dv_s, (float*)dq, (float*)dk, \
                                                                          (float*)dv)                            \
         : merge_bwd_warp_kernel<float, MC, 1><<<grid, kThreads, 0, st>>>(g, dq_s, dk_s, dv_s, (float*)dq, (float*)dk, \
                                                                          (float*)dv);
    if (mc <= 2) {
      GATTN_MERGE_BWD(2)
    } else if (mc <= 4) {
      GATTN_MERGE_BWD(4)
    } else {
      GATTN_MERGE_BWD(kMaxCover)
    }
#undef GATTN_MERGE_BWD
    return cudaGetLastError();
  }
  const int64_t total = (int64_t)g.B * g.nh * g.N * (g.d / 4);
  if (out_dtype == GATTN_BF16)
    merge_bwd_kernel<bf><<<grid_for(total), kThreads, 0, st>>>(g, dq_s, dk_s, dv_s, (bf*)dq, (bf*)dk, (bf*)dv);
  else
    merge_bwd_kernel<float><<<grid_for(total), kThreads, 0, st>>>(g, dq_s, dk_s, dv_s, (float*)dq, (float*)dk, (float*)dv);
  return cudaGetLastError();
}

}  // namespace gattn
