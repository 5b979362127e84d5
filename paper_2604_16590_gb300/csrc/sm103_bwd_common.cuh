// sm103_bwd_common.cuh -- pieces shared by the tensor-core backward kernels
// (sm103_bwd64.cu: d = 64; sm103_bwd.cu: d = 128).  Each including translation unit gets its own
// copy (anonymous namespace) and defines its own status word and WAIT().
#pragma once
#include "internal.cuh"
#include "sm103_common.cuh"

namespace gattn {
namespace {
using namespace sm103;

struct BwdArgs {
  Geom g;
  const float* lse2c;
  const float* dd;
  const uint4* ext;  // dK/dV kernels: per-slot B-operand rows of the statistics (see bwd_prep)
  void* dq;
  void* dk;
  void* dv;
  float* dq_s;
  float* dk_s;
  float* dv_s;
  int items;  // B*nh * ntiles * nbmax_tot
};

__device__ __forceinline__ void decode_item(const Geom& g, int w, int& bh, int& tile, int& blk) {
  blk = w % g.nbmax_tot;
  const int r = w / g.nbmax_tot;
  tile = r % g.ntiles;
  bh = r / g.ntiles;
}

// byte offset of K-step ks (16 elements) in a 128-byte-swizzled K-major operand
__device__ __forceinline__ uint32_t kmaj_off(int ks) { return (ks >> 2) * 16384 + (ks & 3) * 32; }

// Warp roles of both backward kernels: warp 0 TMA producer, warp 1 TMEM
// allocator + issuer of the score products, warp kIssuerA issuer of the
// gradient products, warps kMath0.. elementwise math + epilogue (four per TMEM
// lane quadrant, each taking 32 of a row's 128 score columns).
constexpr int kMathW = 16;
constexpr int kMath0 = 3;
constexpr int kIssuerA = 2;
constexpr int kThreadsB = 32 * (kMath0 + kMathW);

// Stores N FP32 values of this thread's row (already in registers), scaled
// by `mul`: to `out` (OutT) if the row is covered by one tile, else to the
// FP32 slot `scr`, nothing if the row lies outside the tile.
template <int N, typename OutT>
__device__ __forceinline__ void row_store(const uint32_t (&r)[N], float mul, bool valid, bool single, OutT* out,
                                          float* scr) {
  if (!valid) return;
#pragma unroll
  for (int e = 0; e < N; e += 4) {
    const float4 v = make_float4(__uint_as_float(r[e]) * mul, __uint_as_float(r[e + 1]) * mul,
                                 __uint_as_float(r[e + 2]) * mul, __uint_as_float(r[e + 3]) * mul);
    if (single)
      store4<OutT>(out + e, v);
    else
      store4<float>(scr + e, v);
  }
}

// dK/dV: P'^T of 32 columns of this thread's key row (S'^T already carries the
// statistics): FP32 in place of the scores, and as BF16 pairs.
__device__ __forceinline__ void kv_p(uint32_t (&s)[32], uint64_t s2, uint32_t (&pp)[16]) {
#pragma unroll
  for (int c = 0; c < 32; c += 2) {
    float a0, a1;
    f2unpack(fmul2(u2pack(s[c], s[c + 1]), s2), a0, a1);
    const float p0 = ex2(a0), p1 = ex2(a1);
    s[c] = __float_as_uint(p0);
    s[c + 1] = __float_as_uint(p1);
    pp[c >> 1] = pack_bf16(p0, p1);
  }
}
// dK/dV: dS^T = P'^T dP'^T (dP'^T already carries -D) as BF16 pairs
__device__ __forceinline__ void kv_ds(const uint32_t (&p)[32], const uint32_t (&dp)[32], uint32_t (&pd)[16]) {
#pragma unroll
  for (int c = 0; c < 32; c += 2) {
    float e0, e1;
    f2unpack(fmul2(u2pack(p[c], p[c + 1]), u2pack(dp[c], dp[c + 1])), e0, e1);
    pd[c >> 1] = pack_bf16(e0, e1);
  }
}

// dQ: P' = exp2(s S log2e - lse') of 32 columns of this thread's query row,
// FP32 in place of the scores
__device__ __forceinline__ void q_p(uint32_t (&s)[32], float sl2, float nL) {
  const uint64_t s2 = f2pack(sl2, sl2), nl2 = f2pack(nL, nL);
#pragma unroll
  for (int c = 0; c < 32; c += 2) {
    float a0, a1;
    f2unpack(ffma2(u2pack(s[c], s[c + 1]), s2, nl2), a0, a1);
    s[c] = __float_as_uint(ex2(a0));
    s[c + 1] = __float_as_uint(ex2(a1));
  }
}
// dQ: dS = P' (dP - D) as BF16 pairs
__device__ __forceinline__ void q_ds(const uint32_t (&p)[32], const uint32_t (&dp)[32], float nD, uint32_t (&pk)[16]) {
  const uint64_t nd2 = f2pack(nD, nD);
#pragma unroll
  for (int c = 0; c < 32; c += 2) {
    float e0, e1;
    f2unpack(fmul2(u2pack(p[c], p[c + 1]), fadd2(u2pack(dp[c], dp[c + 1]), nd2)), e0, e1);
    pk[c >> 1] = pack_bf16(e0, e1);
  }
}

// Constant A operands of the extension steps, K-major without swizzle: 128
// rows x 16 B (K-columns 0..7) followed by 2 KB of zeros (K-columns 8..15).
// `n` blocks of 4 KB from `base`: block 0 has ones in K 0..2 (dK/dV: adds x of
// the statistics row) or in K 0 (dQ: adds the key bias), block 1 ones in K
// 3..5 (dK/dV: adds y).  Then `nz` further 4 KB B-operand blocks at `zb`
// whose zero halves are cleared (their first 2 KB is loaded per box).
__device__ __forceinline__ void init_ext_operands(uint8_t* base, int n, bool stats, uint8_t* zb, int nz) {
  for (int r = threadIdx.x; r < n * 256 + nz * 128; r += blockDim.x) {
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    uint8_t* dst;
    if (r < n * 256) {
      const int blk = r >> 8, rr = r & 255;
      if (rr < 128) {
        if (!stats)
          v = make_uint4(0x00003F80u, 0u, 0u, 0u);                                      // (1, 0, ..., 0)
        else
          v = blk == 0 ? make_uint4(0x3F803F80u, 0x00003F80u, 0u, 0u)                   // (1, 1, 1, 0, 0, 0, 0, 0)
                       : make_uint4(0u, 0x3F800000u, 0x3F803F80u, 0u);                  // (0, 0, 0, 1, 1, 1, 0, 0)
      }
      dst = base + blk * 4096 + rr * 16;
    } else {
      const int q = r - n * 256;
      dst = zb + (q >> 7) * 4096 + 2048 + (q & 127) * 16;
    }
    *reinterpret_cast<uint4*>(dst) = v;
  }
}

}  // namespace
}  // namespace gattn
