// sm103_common.cuh -- 128-token block decomposition of extended tiles used by
// the tcgen05 kernels.
//
// An extended tile (clipped extents e[3] along t, y, x) is covered by 3-D
// boxes of bt x by x bx = R <= 128 tokens (chosen with the geometry).  One box
// is one TMA load of a [bt, by, bx, 64] sub-tensor of the 5-D view
// (d, X, Y, T, B*nh) of a [B, nh, N, d] tensor into the first R rows of a
// 128-row MMA operand block (d = 128 takes two loads, one per 64-column half);
// rows R..127 are never loaded and are zeroed once when a kernel starts.  Row
// rho < R of a block sits at box offset (rho / (by bx), (rho / bx) % by,
// rho % bx).  Boxes may stick out of the tile (rows outside it are masked:
// keys get probability 0, queries are not written) and out of the grid (TMA
// fills zeros).
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
  t.nb[0] = (t.tb.e[0] + g.bt - 1) / g.bt;
  t.nb[1] = (t.tb.e[1] + g.by - 1) / g.by;
  t.nb[2] = (t.tb.e[2] + g.bx - 1) / g.bx;
  t.NB = t.nb[0] * t.nb[1] * t.nb[2];
}

// tile-local origin of block j
__device__ __forceinline__ void block_origin(const Geom& g, const TileBlocks& t, int j, int o[3]) {
  const int jx = j % t.nb[2];
  const int jr = j / t.nb[2];
  const int jy = jr % t.nb[1];
  const int jt = jr / t.nb[1];
  o[0] = jt * g.bt;
  o[1] = jy * g.by;
  o[2] = jx * g.bx;
}

// all 128 rows of the block hold tokens of the tile (no padding row, none
// outside the tile)
__device__ __forceinline__ bool block_full(const Geom& g, const TileBlocks& t, const int o[3]) {
  return g.R == 128 && o[0] + g.bt <= t.tb.e[0] && o[1] + g.by <= t.tb.e[1] && o[2] + g.bx <= t.tb.e[2];
}

// tile-local coordinates of row rho of a block with origin o; a padding row
// (rho >= R) gets a coordinate outside every tile
__device__ __forceinline__ void block_row(const Geom& g, const int o[3], int rho, int l[3]) {
  int b[3];
  box_offset(g, rho, b);
  l[0] = rho < g.R ? o[0] + b[0] : (1 << 30);
  l[1] = o[1] + b[1];
  l[2] = o[2] + b[2];
}

// every block of the tile holds 128 rows of the tile (no padding anywhere)
__device__ __forceinline__ bool tile_all_full(const Geom& g, const TileBlocks& t) {
  return g.R == 128 && t.tb.e[0] % g.bt == 0 && t.tb.e[1] % g.by == 0 && t.tb.e[2] % g.bx == 0;
}

// Walks the blocks of a tile in index order with counters instead of
// divisions; full() says whether the current block is full (block_full).
struct BlockWalk {
  int jt = 0, jy = 0, jx = 0;
  __device__ __forceinline__ bool full(const Geom& g, const TileBlocks& t) const {
    const int o[3] = {jt * g.bt, jy * g.by, jx * g.bx};
    return block_full(g, t, o);
  }
  __device__ __forceinline__ void next(const TileBlocks& t) {
    if (++jx == t.nb[2]) {
      jx = 0;
      if (++jy == t.nb[1]) {
        jy = 0;
        ++jt;
      }
    }
  }
};

__device__ __forceinline__ bool inside(const TileBlocks& t, const int l[3]) {
  return l[0] < t.tb.e[0] && l[1] < t.tb.e[1] && l[2] < t.tb.e[2];
}

// Zero rows R..127 of n consecutive 16 KB operand blocks starting at `base`
// (128-row, 128-byte rows): TMA loads only the first R rows of a block, and
// the padding rows meet zero probabilities or gradients in the MMAs, where a
// stale NaN would survive the multiplication by zero.  All threads of the CTA
// call it before the first __syncthreads; it ends with the proxy fence that
// makes the writes visible to the tensor cores.
__device__ __forceinline__ void zero_pad_rows(uint8_t* base, int n, int R) {
  if (R >= 128) return;
  const int per = (128 - R) * 8;  // 16-byte units per block
  for (int u = threadIdx.x; u < n * per; u += blockDim.x) {
    const int b = u / per, r = u - b * per;
    *reinterpret_cast<uint4*>(base + (size_t)b * 16384 + R * 128 + r * 16) = make_uint4(0u, 0u, 0u, 0u);
  }
  sm103::fence_proxy_async_smem();
}

// first slot of tile `tile` of batch*head bh (block j, row rho at + j*128 + rho)
__device__ __forceinline__ int64_t tile_slot0(const Geom& g, int bh, int tile) {
  return ((int64_t)bh * g.ntiles + tile) * g.per_tile;
}

}  // namespace gattn
