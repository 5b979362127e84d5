// sm103_common.cuh -- 128-token block decomposition of extended tiles used by
// the tcgen05 kernels.
//
// An extended tile (clipped extents e[3] along t, y, x) is covered by 3-D
// boxes of bt x by x bx = 128 tokens (powers of two, chosen with the geometry).  One box is one TMA load
// of a [bt, by, bx, 64] sub-tensor of the 5-D view (d, X, Y, T, B*nh) of a
// [B, nh, N, d] tensor, i.e. one 128-row MMA operand block (d = 128 takes two
// loads, one per 64-column half).  Row rho of a block sits at box offset
// (rho >> (ly + lx), (rho >> lx) & (by - 1), rho & (bx - 1)).  Boxes may stick
// out of the tile (rows outside it are masked: keys get probability 0,
// queries are not written) and out of the grid (TMA fills zeros).
#pragma once

#include "sm103_ptx.cuh"

namespace gattn {

int num_sms();

struct TileBlocks {
  TileBox tb;
  int nb[3];
  int NB;
};

__device__ __forceinline__ void tile_blocks(const Geom& g, int tile, TileBlocks& t) {
  tile_box(g, tile, t.tb);
  t.nb[0] = (t.tb.e[0] + g.bt - 1) >> g.lt;
  t.nb[1] = (t.tb.e[1] + g.by - 1) >> g.ly;
  t.nb[2] = (t.tb.e[2] + g.bx - 1) >> g.lx;
  t.NB = t.nb[0] * t.nb[1] * t.nb[2];
}

// tile-local origin of block j
__device__ __forceinline__ void block_origin(const Geom& g, const TileBlocks& t, int j, int o[3]) {
  const int jx = j % t.nb[2];
  const int jr = j / t.nb[2];
  const int jy = jr % t.nb[1];
  const int jt = jr / t.nb[1];
  o[0] = jt << g.lt;
  o[1] = jy << g.ly;
  o[2] = jx << g.lx;
}

// all 128 rows of the block lie inside the tile
__device__ __forceinline__ bool block_full(const Geom& g, const TileBlocks& t, const int o[3]) {
  return o[0] + g.bt <= t.tb.e[0] && o[1] + g.by <= t.tb.e[1] && o[2] + g.bx <= t.tb.e[2];
}

// tile-local coordinates of row rho of a block with origin o
__device__ __forceinline__ void block_row(const Geom& g, const int o[3], int rho, int l[3]) {
  l[0] = o[0] + (rho >> (g.ly + g.lx));
  l[1] = o[1] + ((rho >> g.lx) & (g.by - 1));
  l[2] = o[2] + (rho & (g.bx - 1));
}

__device__ __forceinline__ bool inside(const TileBlocks& t, const int l[3]) {
  return l[0] < t.tb.e[0] && l[1] < t.tb.e[1] && l[2] < t.tb.e[2];
}

// first slot of tile `tile` of batch*head bh (block j, row rho at + j*128 + rho)
__device__ __forceinline__ int64_t tile_slot0(const Geom& g, int bh, int tile) {
  return ((int64_t)bh * g.ntiles + tile) * g.per_tile;
}

}  // namespace gattn
