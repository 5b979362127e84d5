// merge_common.cuh -- per-token cover lists for the Hann-weighted overlap
// average of STORM-GPA (arXiv 2604.16590, Sec. III-C: outputs of overlapping
// extended tiles are averaged with Hanning weights).
//
// Window weights come from a per-dimension table of sin^2(pi (n + 1/2) / M)
// built in shared memory once per CTA (the same half-sample Hann as
// window_dim in geom.cuh), so a token's weights cost three table reads per
// covering tile.  A token's covering tiles (at most kMaxCover, which the host
// checks with max_covers) are listed with their slot and weight by the lane
// that owns the token, into per-warp shared-memory lists (RowRef); groups of
// lanes (half- or quarter-warps) then read the listed rows as contiguous
// runs, several rows at a time with all their loads in flight.
#pragma once

#include "internal.cuh"

namespace gattn {

constexpr int kMaxCover = 8;    // covering tiles a lane lists for its token
constexpr int kWinMax = 2048;   // table entries (sum of c_a + 2 h_a) kept in shared memory

// One row in a lane group's list of rows to read (the flattened merge loops):
// the row's address (or, in the gradient merge, its slot's element offset),
// its weight and flags (bits 0-4: the lane that owns the row's token;
// kRowLast: the token's last covering row; kRowBf16: a BF16 row, else FP32;
// kRowState: the token's state row, read, updated and written back).
struct alignas(16) RowRef {
  const void* p;
  float w;
  int flags;
};
constexpr int kRowLast = 32, kRowBf16 = 64, kRowState = 128;

// Most tiles covering one token (product over dimensions of the per-dimension
// maximum); the cover pattern repeats with period c, edges only lower it.
inline int max_covers(const Geom& g) {
  int m = 1;
  for (int a = 0; a < 3; ++a) {
    int best = 1;
    const int lim = g.G[a] < 3 * g.c[a] + 2 * g.h[a] ? g.G[a] : 3 * g.c[a] + 2 * g.h[a];
    for (int p = 0; p < lim; ++p) {
      int k0, k1;
      cover_dim(g, a, p, k0, k1);
      best = k1 - k0 + 1 > best ? k1 - k0 + 1 : best;
    }
    m *= best;
  }
  return m;
}

#ifdef __CUDACC__
struct WinTable {
  float* w;   // shared memory: dimension a's entries at off[a]
  int off[3];
  bool direct;  // table too large: evaluate the window directly
};

// Every thread of the CTA calls it (it ends with __syncthreads).
__device__ __forceinline__ WinTable build_win_table(const Geom& g, float* smem) {
  WinTable t;
  t.w = smem;
  int M[3], tot = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    M[a] = g.c[a] + 2 * g.h[a];
    t.off[a] = tot;
    tot += M[a];
  }
  t.direct = tot > kWinMax;
  if (!t.direct)
    for (int e = threadIdx.x; e < tot; e += blockDim.x) {
      const int a = e < t.off[1] ? 0 : e < t.off[2] ? 1 : 2;
      const int n = e - t.off[a];
      float v = 1.f;
      if (g.window != GATTN_WINDOW_FLAT && g.tiled[a]) {
        const float s = sinpif(((float)n + 0.5f) / (float)M[a]);
        v = s * s;
      }
      smem[e] = v;
    }
  __syncthreads();
  return t;
}

// w_t(p) of the tile with per-dimension indices k[3]
__device__ __forceinline__ float table_weight(const Geom& g, const WinTable& t, const int p[3], const int k[3]) {
  if (t.direct) return tile_weight(g, p, k);
  float w = 1.f;
#pragma unroll
  for (int a = 0; a < 3; ++a) w *= t.w[t.off[a] + p[a] - (k[a] * g.c[a] - g.h[a])];
  return w;
}

// Reads of a list entry's address, and of its weight and flags.  They are
// volatile so that the compiler does not merge a second read of an entry with
// the first (that would keep every entry's fields live across the row loads).
__device__ __forceinline__ uint64_t row_addr(const RowRef* e) {
  uint64_t v;
  asm volatile("ld.shared.b64 %0, [%1];" : "=l"(v) : "r"((uint32_t)__cvta_generic_to_shared(e)) : "memory");
  return v;
}
__device__ __forceinline__ void row_weight_flags(const RowRef* e, float& w, int& flags) {
  uint32_t a, b;
  asm volatile("ld.shared.v2.b32 {%0, %1}, [%2];"
               : "=r"(a), "=r"(b)
               : "r"((uint32_t)__cvta_generic_to_shared(e) + 8)
               : "memory");
  w = __uint_as_float(a);
  flags = (int)b;
}

// The rows of the 32 tokens of a warp are read from two lists, one per
// half-warp: half h reads the rows of the tokens of lanes h, h + 2, ..., h + 30
// in that order.  Returns where this lane's n rows start in its parity's list
// and sets len to the length of the list that this lane's half reads.
__device__ __forceinline__ int parity_offset(int n, int lane, int& len) {
  int x = n;  // inclusive sum over the lanes of this lane's parity
#pragma unroll
  for (int s = 2; s < 32; s <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, s);
    if (lane >= s) x += y;
  }
  len = __shfl_sync(0xffffffffu, x, 30 + (lane >> 4));
  return x - n;
}

// The same with four lists, one per quarter-warp: quarter q reads the rows
// of the tokens of lanes q, q + 4, ..., q + 28.  Returns where this lane's n
// rows start in its list and sets len to the length of the list that this
// lane's quarter reads.
__device__ __forceinline__ int group_offset(int n, int lane, int& len) {
  int x = n;  // inclusive sum over the lanes of this lane's residue mod 4
#pragma unroll
  for (int s = 4; s < 32; s <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, s);
    if (lane >= s) x += y;
  }
  len = __shfl_sync(0xffffffffu, x, 28 + (lane >> 3));
  return x - n;
}

// Covering tiles of token i of batch*head bh in ascending tile order: their
// slots and weights (the first NC of them).  Returns the count (0 for a token
// covered by one tile).
template <int NC>
__device__ __forceinline__ int token_covers(const Geom& g, const WinTable& t, int bh, int64_t i, int64_t (&slot)[NC],
                                            float (&w)[NC]) {
  int p[3], k0[3], k1[3];
  token_pos(g, i, p);
  bool multi = false;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    cover_dim(g, a, p[a], k0[a], k1[a]);
    multi = multi || k1[a] > k0[a];
  }
  if (!multi) return 0;
  int n = 0;
  int k[3];
  for (k[0] = k0[0]; k[0] <= k1[0]; ++k[0])
    for (k[1] = k0[1]; k[1] <= k1[1]; ++k[1])
      for (k[2] = k0[2]; k[2] <= k1[2]; ++k[2]) {
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
#pragma unroll
        for (int c = 0; c < NC; ++c)
          if (c == n) {
            slot[c] = slot_of(g, bh, tile, e, l);
            w[c] = table_weight(g, t, p, k);
          }
        ++n;
      }
  return n;
}
#endif

}  // namespace gattn
