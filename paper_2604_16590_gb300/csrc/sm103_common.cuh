// sm103_common.cuh -- 128-token block decomposition of extended tiles used by
// the tcgen05 kernels.
//
// An extended tile (clipped extents e[3] along t, y, x) is covered by 3-D
// boxes of bt x by x bx = 128 tokens (powers of two).  One box is one TMA load
// of a [bt, by, bx, 64] sub-tensor of the 5-D view (d, X, Y, T, B*nh) of a
// [B, nh, N, d] tensor, i.e. one 128-row MMA operand block (d = 128 takes two
// loads, one per 64-column half).  Row rho of a block sits at box offset
// (rho >> (ly + lx), (rho >> lx) & (by - 1), rho & (bx - 1)).  Boxes may stick
// out of the tile (rows outside it are masked: keys get probability 0,
// queries are not written) and out of the grid (TMA fills zeros).
#pragma once

#include "sm103_ptx.cuh"

namespace gattn {

struct BlockShape {
  int bt, by, bx;     // box extents, product 128
  int lt, ly, lx;     // their log2
  int nbmax[3];       // most boxes any tile needs per dimension
};

BlockShape choose_block_shape(const Geom& g);
int num_sms();

struct TileBlocks {
  TileBox tb;
  int nb[3];
  int NB;
};

__device__ __forceinline__ void tile_blocks(const Geom& g, const BlockShape& bs, int tile, TileBlocks& t) {
  tile_box(g, tile, t.tb);
  t.nb[0] = (t.tb.e[0] + bs.bt - 1) >> bs.lt;
  t.nb[1] = (t.tb.e[1] + bs.by - 1) >> bs.ly;
  t.nb[2] = (t.tb.e[2] + bs.bx - 1) >> bs.lx;
  t.NB = t.nb[0] * t.nb[1] * t.nb[2];
}

// tile-local origin of block j
__device__ __forceinline__ void block_origin(const TileBlocks& t, const BlockShape& bs, int j, int o[3]) {
  const int jx = j % t.nb[2];
  const int jr = j / t.nb[2];
  const int jy = jr % t.nb[1];
  const int jt = jr / t.nb[1];
  o[0] = jt << bs.lt;
  o[1] = jy << bs.ly;
  o[2] = jx << bs.lx;
}

// all 128 rows of the block lie inside the tile
__device__ __forceinline__ bool block_full(const TileBlocks& t, const BlockShape& bs, const int o[3]) {
  return o[0] + bs.bt <= t.tb.e[0] && o[1] + bs.by <= t.tb.e[1] && o[2] + bs.bx <= t.tb.e[2];
}

// tile-local coordinates of row rho of a block with origin o
__device__ __forceinline__ void block_row(const BlockShape& bs, const int o[3], int rho, int l[3]) {
  l[0] = o[0] + (rho >> (bs.ly + bs.lx));
  l[1] = o[1] + ((rho >> bs.lx) & (bs.by - 1));
  l[2] = o[2] + (rho & (bs.bx - 1));
}

__device__ __forceinline__ bool inside(const TileBlocks& t, const int l[3]) {
  return l[0] < t.tb.e[0] && l[1] < t.tb.e[1] && l[2] < t.tb.e[2];
}

}  // namespace gattn
