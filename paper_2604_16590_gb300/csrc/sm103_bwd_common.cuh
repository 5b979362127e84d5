// sm103_bwd_common.cuh -- pieces shared by the tensor-core backward kernels
// (sm103_bwd.cu: general head size, shared-memory operands; sm103_bwd64.cu:
// d = 64 with TMEM operands).  Each including translation unit gets its own
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
  const uint4* ext;  // d = 64 kernels: per-slot B-operand rows of the statistics (see bwd_prep)
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

// Epilogue of one D-wide FP32 TMEM row (this thread's lane), scaled by `mul`:
// to `out` (OutT) if the row is covered by one tile, else to the FP32 slot
// `scr`; nothing if the row lies outside the tile.  The TMEM loads are
// warp-synchronous (.sync.aligned), so every lane executes them and only the
// global stores depend on the lane's row.
template <int NCOLS, typename OutT>
__device__ __forceinline__ void tmem_row_epilogue(uint32_t taddr, float mul, bool valid, bool single, OutT* out,
                                                  float* scr) {
  uint32_t r[32];
#pragma unroll
  for (int c = 0; c < NCOLS / 32; ++c) {
    tmem_ld32(taddr + c * 32, r);
    tmem_wait_ld(r);
    if (valid) {
#pragma unroll
      for (int e = 0; e < 32; e += 4) {
        const float4 v = make_float4(__uint_as_float(r[e]) * mul, __uint_as_float(r[e + 1]) * mul,
                                     __uint_as_float(r[e + 2]) * mul, __uint_as_float(r[e + 3]) * mul);
        if (single)
          store4<OutT>(out + c * 32 + e, v);
        else
          store4<float>(scr + c * 32 + e, v);
      }
    }
  }
}

// Write 32 BF16 values (16 packed words) as half of one 128-byte row (16-byte
// units 4*ch .. 4*ch+3) of a 128B-swizzled K-major operand buffer.
__device__ __forceinline__ void store_row32(uint32_t buf, int row, int ch, const uint32_t (&pk)[16]) {
#pragma unroll
  for (int u = 0; u < 4; ++u)
    st_shared_v4(buf + row * 128 + (((ch * 4 + u) ^ (row & 7)) << 4), pk[4 * u], pk[4 * u + 1], pk[4 * u + 2],
                 pk[4 * u + 3]);
}

// Math warps: kMathWarps warps, two per TMEM lane quadrant; the two warps of a
// quadrant share its 32 rows and split each row's columns in half.
constexpr int kMathWarps = 8;
constexpr int kThreads = 64 + 32 * kMathWarps;

template <bool MASK>
__device__ __forceinline__ void dq_half(const uint32_t (&s)[32], const uint32_t (&dp)[32], uint32_t mbits, float sl2,
                                        float nL, float nD, uint32_t (&pk)[16]) {
  const uint64_t s2 = f2pack(sl2, sl2), nl2 = f2pack(nL, nL), nd2 = f2pack(nD, nD);
#pragma unroll
  for (int c = 0; c < 32; c += 2) {
    float a0, a1;
    f2unpack(ffma2(u2pack(s[c], s[c + 1]), s2, nl2), a0, a1);
    float p0 = ex2(a0), p1 = ex2(a1);
    if (MASK) {
      p0 = (mbits >> c) & 1u ? p0 : 0.f;
      p1 = (mbits >> (c + 1)) & 1u ? p1 : 0.f;
    }
    float e0, e1;
    f2unpack(fmul2(f2pack(p0, p1), fadd2(u2pack(dp[c], dp[c + 1]), nd2)), e0, e1);
    pk[c >> 1] = pack_bf16(e0, e1);
  }
}

// TMEM column of K-step ks (16 BF16 values = 8 packed columns) of a row whose
// packed values were written as two 16-column halves of 32 columns each
__device__ __forceinline__ uint32_t pair_col(int ks) { return ks < 2 ? ks * 8 : 32 + (ks - 2) * 8; }

}  // namespace
}  // namespace gattn
