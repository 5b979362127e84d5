// geom.cuh -- tile geometry of STORM-GPA shared by every kernel of the library
// (arXiv 2604.16590, Sec. III-C: tiles, halos, Hann-weighted overlap average).
//
// Grid (T, Y, X) = G[0..2]; core c[a], halo h[a]; n[a] = ceil(G[a]/c[a]) tiles
// per dimension; tile index = (k_t * n_y + k_y) * n_x + k_x (so ascending tile
// index is the fixed merge order).  Extended interval of tile k along a:
// [max(k c - h, 0), min((k+1) c + h, G)).  Rows of an extended tile are
// numbered r = (lt * e_y + ly) * e_x + lx over its clipped extents e[3].
// Every extended tile is also covered by 3-D boxes of bt x by x bx = R <= 128
// tokens (the box shape is chosen per problem on the host); one box is one
// 128-row MMA block whose rows R..127 are padding.  Box j of a tile with
// nb[3] boxes per dimension has origin ((j / (nb_y nb_x)) bt,
// ((j / nb_x) % nb_y) by, (j % nb_x) bx) in tile-local coordinates and its row
// rho < R sits at box offset (rho / (by bx), (rho / bx) % by, rho % bx).
// Per-(tile, row) state (log-sum-exp, per-tile outputs, softmax statistics,
// per-tile gradients) lives at slot
//     ((bh * ntiles + tile) * per_tile + j * 128 + rho),  per_tile = nbmax * 128,
// so the rows of one box are contiguous -- the order the tensor-core kernels
// process them in.
#pragma once

#include <stdint.h>

#include "gattn.h"

#ifndef __CUDACC__
#define __host__
#define __device__
#define __forceinline__ inline
#endif

namespace gattn {

struct Geom {
  int32_t B, nh, d;
  int32_t G[3];     // T, Y, X
  int32_t c[3];     // core
  int32_t h[3];     // halo
  int32_t n[3];     // tiles per dimension
  int32_t emax[3];  // largest clipped extended extent per dimension
  int32_t tiled[3]; // 0: dimension has one tile and no halo (window factor 1)
  int32_t ntiles;
  int32_t Lmax;
  int32_t window;   // gattn_window
  int32_t bt, by, bx;   // box shape, R = bt * by * bx <= 128 tokens
  int32_t R;            // rows of a box that hold tokens
  uint32_t mdx, mdxy;   // ceil(2^16 / bx), ceil(2^16 / (bx by)): exact quotients of rho < 128
  int32_t nbmax[3];     // most boxes any tile needs per dimension
  int32_t nbmax_tot;    // nbmax[0] * nbmax[1] * nbmax[2]
  int32_t per_tile;     // slots per tile = nbmax_tot * 128
  int64_t N;
  float scale;      // softmax scale s
  float scale_log2; // s * log2(e)
};

__host__ __device__ __forceinline__ int floordiv(int a, int b) {
  int q = a / b;
  return (a % b != 0 && ((a < 0) != (b < 0))) ? q - 1 : q;
}

struct TileBox {
  int lo[3];
  int e[3];
  int L;
};

__host__ __device__ __forceinline__ void tile_box(const Geom& g, int tile, TileBox& tb) {
  int k[3];
  k[2] = tile % g.n[2];
  k[1] = (tile / g.n[2]) % g.n[1];
  k[0] = tile / (g.n[2] * g.n[1]);
  tb.L = 1;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    int lo = k[a] * g.c[a] - g.h[a];
    int hi = (k[a] + 1) * g.c[a] + g.h[a];
    lo = lo < 0 ? 0 : lo;
    hi = hi > g.G[a] ? g.G[a] : hi;
    tb.lo[a] = lo;
    tb.e[a] = hi - lo;
    tb.L *= tb.e[a];
  }
}

// grid token index of row r of the extended tile
__host__ __device__ __forceinline__ int64_t tile_token(const Geom& g, const TileBox& tb, int r) {
  int lx = r % tb.e[2];
  int rr = r / tb.e[2];
  int ly = rr % tb.e[1];
  int lt = rr / tb.e[1];
  return ((int64_t)(tb.lo[0] + lt) * g.G[1] + (tb.lo[1] + ly)) * g.G[2] + (tb.lo[2] + lx);
}

__host__ __device__ __forceinline__ void token_pos(const Geom& g, int64_t i, int p[3]) {
  p[2] = (int)(i % g.G[2]);
  int64_t r = i / g.G[2];
  p[1] = (int)(r % g.G[1]);
  p[0] = (int)(r / g.G[1]);
}

// tiles along dimension a that cover grid position p: [k0, k1]
__host__ __device__ __forceinline__ void cover_dim(const Geom& g, int a, int p, int& k0, int& k1) {
  k0 = floordiv(p - g.h[a], g.c[a]);
  k1 = floordiv(p + g.h[a], g.c[a]);
  k0 = k0 < 0 ? 0 : k0;
  k1 = k1 > g.n[a] - 1 ? g.n[a] - 1 : k1;
}

// true if exactly one tile covers grid position p
__host__ __device__ __forceinline__ bool single_cover(const Geom& g, const int p[3]) {
  bool one = true;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    int k0, k1;
    cover_dim(g, a, p[a], k0, k1);
    one = one && (k0 == k1);
  }
  return one;
}

// tile-local coordinates of row r (row-major over the clipped extents)
__host__ __device__ __forceinline__ void tile_local(const TileBox& tb, int r, int l[3]) {
  l[2] = r % tb.e[2];
  const int rr = r / tb.e[2];
  l[1] = rr % tb.e[1];
  l[0] = rr / tb.e[1];
}

// offset (t, y, x) of row rho (0 <= rho < 128) inside a box; the quotients
// are multiply-shifts, exact for rho < 128 and box extents <= 128
__host__ __device__ __forceinline__ void box_offset(const Geom& g, int rho, int o[3]) {
  const int rt = (int)(((uint32_t)rho * g.mdxy) >> 16);
  const int rem = rho - rt * g.by * g.bx;
  const int ry = (int)(((uint32_t)rem * g.mdx) >> 16);
  o[0] = rt;
  o[1] = ry;
  o[2] = rem - ry * g.bx;
}

// slot of the token at tile-local coordinates l[3] of a tile with extents e[3]
__host__ __device__ __forceinline__ int64_t slot_of(const Geom& g, int bh, int tile, const int e[3], const int l[3]) {
  const int nby = (e[1] + g.by - 1) / g.by;
  const int nbx = (e[2] + g.bx - 1) / g.bx;
  const int qt = l[0] / g.bt, qy = l[1] / g.by, qx = l[2] / g.bx;
  const int j = (qt * nby + qy) * nbx + qx;
  const int rho = ((l[0] - qt * g.bt) * g.by + (l[1] - qy * g.by)) * g.bx + (l[2] - qx * g.bx);
  return ((int64_t)bh * g.ntiles + tile) * g.per_tile + (int64_t)j * 128 + rho;
}

// inverse of slot_of within one tile: tile-local coordinates of row rho of
// box j of a tile with extents e[3]; false if that row is padding (rho >= R)
// or lies outside the tile
__host__ __device__ __forceinline__ bool slot_local(const Geom& g, const int e[3], int j, int rho, int l[3]) {
  if (rho >= g.R) return false;
  const int nby = (e[1] + g.by - 1) / g.by;
  const int nbx = (e[2] + g.bx - 1) / g.bx;
  const int jx = j % nbx, jr = j / nbx;
  const int jy = jr % nby, jt = jr / nby;
  int o[3];
  box_offset(g, rho, o);
  l[0] = jt * g.bt + o[0];
  l[1] = jy * g.by + o[1];
  l[2] = jx * g.bx + o[2];
  return l[0] < e[0] && l[1] < e[1] && l[2] < e[2];
}

__host__ __device__ __forceinline__ int64_t grid_token(const Geom& g, const TileBox& tb, const int l[3]) {
  return ((int64_t)(tb.lo[0] + l[0]) * g.G[1] + (tb.lo[1] + l[1])) * g.G[2] + (tb.lo[2] + l[2]);
}

#ifdef __CUDACC__
// Window factor of tile index k along dimension a at grid position p:
// sin^2(pi (n + 1/2) / M), n = p - (k c - h), M = c + 2h (half-sample Hann).
__device__ __forceinline__ float window_dim(const Geom& g, int a, int p, int k) {
  if (g.window == GATTN_WINDOW_FLAT || !g.tiled[a]) return 1.0f;
  int n = p - (k * g.c[a] - g.h[a]);
  int M = g.c[a] + 2 * g.h[a];
  float s = sinpif(((float)n + 0.5f) / (float)M);
  return s * s;
}

// w_t(p) for the tile with per-dimension indices k[3]
__device__ __forceinline__ float tile_weight(const Geom& g, const int p[3], const int k[3]) {
  return window_dim(g, 0, p[0], k[0]) * window_dim(g, 1, p[1], k[1]) * window_dim(g, 2, p[2], k[2]);
}
#endif

// Host-side construction (including the box shape); false on an invalid descriptor.
bool make_geom(const gattn_desc* desc, Geom* g);
// Replace the box shape of a constructed geometry by b (bt, by, bx), R <= 128
// (every shape is valid, only the padding differs); false if b is not a box
// shape or the slot count overflows.
bool apply_box(Geom* g, const int b[3]);

}  // namespace gattn
