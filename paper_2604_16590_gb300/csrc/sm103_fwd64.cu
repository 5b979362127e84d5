// sm103_fwd64.cu -- BF16 tensor-core forward of STORM-GPA tile attention for
// head size d = 64 on GB300 (sm_103a): two query boxes per work item in
// ping-pong.
//
// Per extended tile t (arXiv 2604.16590, Sec. III-C) and pair of 128-query
// boxes (A, B) of the tile, the CTA streams the tile's 128-key boxes once for
// both query boxes (flash-style online softmax, the FlashAttention of
// Sec. III-D Level 5):
//   S_x  = Q_x K_j^T                    tcgen05, A = Q_x from TMEM, B = K_j (smem)
//   m_x  = max(m_x, rowmax(s S_x))      log2 domain, lazily moved (threshold 8)
//   P_x  = exp2(s S_x log2e - m_x)      BF16 pairs written over S_x's first 64 columns
//   O_x += P_x V_j                      tcgen05, A = P_x from TMEM, B = V_j (MN-major)
// While the softmax warps of one box work on its scores, the tensor core runs
// the other box's products: each box's chain (S, softmax, P V) is serial --
// S_x(j+1) overwrites the P_x that P V_x(j) reads -- and two chains in flight
// keep the tensor pipe and the MUFU units busy at the same time.  K and V are
// loaded once for both boxes.  The epilogue writes O / l for rows covered by
// one tile straight to the output and parks multiply-covered rows (FP32) for
// the deterministic Hann merge, and stores the row log-sum-exp.
//
// Warp roles (352 threads, one CTA per SM, persistent over work items
// (batch*head, tile, box pair)):
//   warp 0        TMA producer (Q_A, Q_B once per item; K_j, V_j through a ring)
//   warp 1        TMEM allocator + issuer of the S products
//   warp 2        issuer of the P V products (a thread's mbarrier waits stall
//                 until its own issued MMAs drain, so the two product streams
//                 come from two threads)
//   warps 3..6    softmax + epilogue of box A, warps 7..10 of box B: one warp
//                 per TMEM lane quadrant, one thread per query row owning all
//                 128 key columns (no cross-warp reduction)
// TMEM (448 columns): S_x at 128 x (P_x over its first 64), O_x at 256 + 64 x,
// Q_x at 384 + 32 x.
#include "internal.cuh"
#include "sm103_common.cuh"

GATTN_DEFINE_STATUS(sm103_fwd64)

namespace gattn {
namespace {
using namespace sm103;

__device__ void set_status_f64(uint32_t c) { set_status(c); }
#define WAIT(bar, par) mbar_wait<set_status_f64>((bar), (par), abort_flag)

constexpr int kD = 64;
constexpr int kBox = 128 * kD * 2;  // one 128-token box of one operand, BF16, 16 KB
constexpr int kStages = 4;          // K/V ring depth
constexpr int kSoft0 = 3;           // first softmax warp
constexpr int kThreadsF = 32 * (kSoft0 + 8);
constexpr float kRescaleLog2 = 8.f;

struct Cfg {
  static constexpr int kQ = 0;  // Q_A at kQ, Q_B at kQ + kBox
  static constexpr int kK = 2 * kBox;
  static constexpr int kV = kK + kStages * kBox;
  static constexpr int kBar = kV + kStages * kBox;
  // q_full, q_empty, k_full[S], k_empty[S], v_full[S], v_empty[S],
  // per box: qt_full, s_full, p_full, pv_done, o_empty; drain[2], never
  static constexpr int kNumBars = 2 + 4 * kStages + 2 * 5 + 3;
  static constexpr int kMisc = kBar + kNumBars * 8;
  static constexpr int kSmem = kMisc + 16 + 1024;
};
__device__ __forceinline__ uint32_t col_s(int x) { return 128u * x; }
__device__ __forceinline__ uint32_t col_o(int x) { return 256u + 64u * x; }
__device__ __forceinline__ uint32_t col_q(int x) { return 384u + 32u * x; }

struct Fwd64Args {
  Geom g;
  void* out;
  float* lse2;
  float* ot;
  int items;  // B*nh * ntiles * box pairs
  int npairs;
  uint32_t flags;
};

__device__ __forceinline__ void decode_pair(const Fwd64Args& a, int w, int& bh, int& tile, int& pair) {
  pair = w % a.npairs;
  const int r = w / a.npairs;
  tile = r % a.g.ntiles;
  bh = r / a.g.ntiles;
}

// running max of 32 scores into 4 partial maxima (3-input max)
template <bool MASK>
__device__ __forceinline__ void chunk_max(const uint32_t (&r)[32], uint32_t mbits, float (&mx)[4]) {
#pragma unroll
  for (int i = 0; i < 32; i += 2) {
    float x0 = __uint_as_float(r[i]), x1 = __uint_as_float(r[i + 1]);
    if (MASK) {
      x0 = (mbits >> i) & 1u ? x0 : -INFINITY;
      x1 = (mbits >> (i + 1)) & 1u ? x1 : -INFINITY;
    }
    mx[(i >> 1) & 3] = fmax3(mx[(i >> 1) & 3], x0, x1);
  }
}

// exp2 of 32 scores -> 16 BF16 pairs, row sum in packed FP32 pairs
template <bool MASK>
__device__ __forceinline__ void exp_chunk(const uint32_t (&r)[32], uint32_t mbits, uint64_t s2, uint64_t nm2,
                                          uint64_t (&acc)[4], uint32_t (&pk)[16]) {
#pragma unroll
  for (int i = 0; i < 32; i += 2) {
    float a0, a1;
    f2unpack(ffma2(u2pack(r[i], r[i + 1]), s2, nm2), a0, a1);
    float p0 = ex2(a0), p1 = ex2(a1);
    if (MASK) {
      p0 = (mbits >> i) & 1u ? p0 : 0.f;
      p1 = (mbits >> (i + 1)) & 1u ? p1 : 0.f;
    }
    acc[(i >> 1) & 3] = fadd2(acc[(i >> 1) & 3], f2pack(p0, p1));
    pk[i >> 1] = pack_bf16(p0, p1);
  }
}

// One key box of the online softmax for this thread's query row: row max over
// the 128 scores, lazy move of the reference max (rescaling O in TMEM -- the
// previous P V of this box is complete, because these scores were computed
// after it), then exp2 of the scores written as BF16 pairs over the scores'
// first 64 columns (chunk c of 32 scores -> columns [16c, 16c+16), which only
// ever covers scores already read).
template <bool MASK>
__device__ __forceinline__ void softmax_box(float& m, float& l, uint32_t tS, uint32_t tO, const uint32_t (&km)[4],
                                            float sl2, bool first) {
  float mx[4] = {-INFINITY, -INFINITY, -INFINITY, -INFINITY};
  {
    uint32_t r0[32], r1[32];
#pragma unroll
    for (int c = 0; c < 4; c += 2) {
      tmem_ld32(tS + 32 * c, r0);
      tmem_ld32(tS + 32 * c + 32, r1);
      tmem_wait_ld(r0);
      tmem_wait_ld(r1);
      chunk_max<MASK>(r0, km[c], mx);
      chunk_max<MASK>(r1, km[c + 1], mx);
    }
  }
  const float mblk = fmaxf(fmaxf(mx[0], mx[1]), fmaxf(mx[2], mx[3])) * sl2;
  if (first) {
    m = mblk;
  } else {
    const bool grow = mblk > m + kRescaleLog2;
    if (__any_sync(0xffffffffu, grow)) {
      const float f = grow ? ex2(m - mblk) : 1.f;
      const uint64_t f2 = f2pack(f, f);
      uint32_t r[32];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        tmem_ld32(tO + 32 * c, r);
        tmem_wait_ld(r);
#pragma unroll
        for (int i = 0; i < 32; i += 2) {
          float x, y;
          f2unpack(fmul2(u2pack(r[i], r[i + 1]), f2), x, y);
          r[i] = __float_as_uint(x);
          r[i + 1] = __float_as_uint(y);
        }
        tmem_st32(tO + 32 * c, r);
      }
      tmem_wait_st();
      l *= f;
      if (grow) m = mblk;
    }
  }
  const uint64_t s2 = f2pack(sl2, sl2), nm2 = f2pack(-m, -m);
  uint64_t acc[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) acc[i] = f2pack(0.f, 0.f);
#pragma unroll 1
  for (int c = 0; c < 4; ++c) {
    uint32_t r[32], pk[16];
    tmem_ld32(tS + 32 * c, r);
    const uint32_t mb = c == 0 ? km[0] : c == 1 ? km[1] : c == 2 ? km[2] : km[3];
    tmem_wait_ld(r);
    exp_chunk<MASK>(r, mb, s2, nm2, acc, pk);
    tmem_st16(tS + 16 * c, pk);
  }
  float lsum = 0.f;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float x, y;
    f2unpack(acc[i], x, y);
    lsum += x + y;
  }
  l += lsum;
  tmem_wait_st();
}

template <typename OutT>
__global__ void __launch_bounds__(kThreadsF, 1)
    fwd64_kernel(const __grid_constant__ CUtensorMap tq, const __grid_constant__ CUtensorMap tk,
                 const __grid_constant__ CUtensorMap tv, const Fwd64Args a) {
  using C = Cfg;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::kBar);
  uint64_t* q_full = bars;
  uint64_t* q_empty = bars + 1;
  uint64_t* k_full = bars + 2;
  uint64_t* k_empty = k_full + kStages;
  uint64_t* v_full = k_empty + kStages;
  uint64_t* v_empty = v_full + kStages;
  uint64_t* boxbar = v_empty + kStages;  // [x * 5 + i]
  auto qt_full = [&](int x) { return boxbar + 5 * x; };
  auto s_full = [&](int x) { return boxbar + 5 * x + 1; };
  auto p_full = [&](int x) { return boxbar + 5 * x + 2; };
  auto pv_done = [&](int x) { return boxbar + 5 * x + 3; };
  auto o_empty = [&](int x) { return boxbar + 5 * x + 4; };
  uint64_t* drain = boxbar + 10;  // [2]
  uint64_t* never = drain + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + C::kMisc);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + C::kMisc + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    mbar_init(q_full, 1);
    mbar_init(q_empty, 8);
    for (int s = 0; s < kStages; ++s) {
      mbar_init(k_full + s, 1);
      mbar_init(k_empty + s, 1);
      mbar_init(v_full + s, 1);
      mbar_init(v_empty + s, 1);
    }
    for (int x = 0; x < 2; ++x) {
      mbar_init(qt_full(x), 4);
      mbar_init(s_full(x), 1);
      mbar_init(p_full(x), 4);
      mbar_init(pv_done(x), 1);
      mbar_init(o_empty(x), 4);
    }
    mbar_init(drain, 1);
    mbar_init(drain + 1, 1);
    mbar_init(never, 1);
    *abort_flag = 0;
    fence_mbar_init();
    prefetch_tmap(&tq);
    prefetch_tmap(&tk);
    prefetch_tmap(&tv);
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const Geom& g = a.g;

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      uint32_t G = 0, W = 0;
      uint32_t q_arm = 0, q_par = 0, k_arm = 0, k_par = 0, v_arm = 0, v_par = 0;
      bool ok = true;
      for (int w = blockIdx.x; w < a.items && ok; w += gridDim.x) {
        int bh, tile, pair;
        decode_pair(a, w, bh, tile, pair);
        TileBlocks tbk;
        tile_blocks(g, tile, tbk);
        const int qa = 2 * pair;
        if (qa >= tbk.NB) continue;
        const int nact = qa + 1 < tbk.NB ? 2 : 1;
        if (!(ok = WAIT(q_empty, (W & 1) ^ 1))) break;
        mbar_arrive_expect_tx(q_full, nact * kBox);
        q_arm = 1;
        q_par = W & 1;
        for (int x = 0; x < nact; ++x) {
          int o[3];
          block_origin(g, tbk, qa + x, o);
          tma_load_5d(smem + C::kQ + x * kBox, &tq, q_full, 0, tbk.tb.lo[2] + o[2], tbk.tb.lo[1] + o[1],
                      tbk.tb.lo[0] + o[0], bh);
        }
        int jt = 0, jy = 0, jx = 0;
        for (int j = 0; j < tbk.NB; ++j, ++G) {
          const uint32_t st = G % kStages, n = G / kStages;
          const int c1 = tbk.tb.lo[2] + (jx << g.lx), c2 = tbk.tb.lo[1] + (jy << g.ly), c3 = tbk.tb.lo[0] + (jt << g.lt);
          if (++jx == tbk.nb[2]) {
            jx = 0;
            if (++jy == tbk.nb[1]) {
              jy = 0;
              ++jt;
            }
          }
          if (!(ok = WAIT(k_empty + st, (n & 1) ^ 1))) break;
          mbar_arrive_expect_tx(k_full + st, kBox);
          k_arm |= 1u << st;
          k_par = (k_par & ~(1u << st)) | ((n & 1) << st);
          tma_load_5d(smem + C::kK + st * kBox, &tk, k_full + st, 0, c1, c2, c3, bh);
          if (!(ok = WAIT(v_empty + st, (n & 1) ^ 1))) break;
          mbar_arrive_expect_tx(v_full + st, kBox);
          v_arm |= 1u << st;
          v_par = (v_par & ~(1u << st)) | ((n & 1) << st);
          tma_load_5d(smem + C::kV + st * kBox, &tv, v_full + st, 0, c1, c2, c3, bh);
        }
        ++W;
      }
      if (!ok) {
        // let every load this thread issued land before the CTA exits
        if (q_arm) mbar_wait<set_status_f64>(q_full, q_par, abort_flag, false);
        for (int s = 0; s < kStages; ++s) {
          if (k_arm & (1u << s)) mbar_wait<set_status_f64>(k_full + s, (k_par >> s) & 1, abort_flag, false);
          if (v_arm & (1u << s)) mbar_wait<set_status_f64>(v_full + s, (v_par >> s) & 1, abort_flag, false);
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ issuer of S_x = Q_x K^T
    if (lane == 0) {
      constexpr uint32_t idS = idesc_bf16(128, 128, 0);
      const uint64_t dK0 = sw128_desc(smem_u32(smem + C::kK), 16, 1024);
      uint32_t G = 0, GX[2] = {0, 0}, WX[2] = {0, 0};
      bool ok = true;
      if (a.flags & GATTN_FLAG_TEST_STALL)  // failure-detection hook: a wait that cannot complete
        ok = mbar_wait<set_status_f64>(never, 0, abort_flag, true, 20000000ull);
      for (int w = blockIdx.x; w < a.items && ok; w += gridDim.x) {
        int bh, tile, pair;
        decode_pair(a, w, bh, tile, pair);
        TileBlocks tbk;
        tile_blocks(g, tile, tbk);
        const int qa = 2 * pair;
        if (qa >= tbk.NB) continue;
        const int nact = qa + 1 < tbk.NB ? 2 : 1;
#pragma unroll
        for (int x = 0; x < 2; ++x)  // Q_x in TMEM
          if (x < nact && ok) ok = WAIT(qt_full(x), WX[x] & 1);
        for (int j = 0; j < tbk.NB && ok; ++j, ++G) {
          const uint32_t st = G % kStages;
          if (!(ok = WAIT(k_full + st, (G / kStages) & 1))) break;
          const uint64_t dk = dmove(dK0, st * kBox);
#pragma unroll
          for (int x = 0; x < 2; ++x) {
            if (x >= nact) break;
            // S_x overwrites P_x: the previous P V of box x must be complete
            if (GX[x] > 0 && !(ok = WAIT(pv_done(x), (GX[x] - 1) & 1))) break;
            tc_fence_after();
#pragma unroll
            for (int ks = 0; ks < kD / 16; ++ks)
              umma_bf16_ts(tmem + col_s(x), tmem + col_q(x) + ks * 8, dmove(dk, ks * 32), idS, ks > 0);
            umma_commit(s_full(x));
            ++GX[x];
          }
          if (!ok) break;
          umma_commit(k_empty + st);
        }
#pragma unroll
        for (int x = 0; x < 2; ++x)
          if (x < nact) ++WX[x];
      }
      umma_commit(drain);
      mbar_wait<set_status_f64>(drain, 0, abort_flag, false);
    }
  } else if (warp == 2) {
    // ------------------------------------------------------------ issuer of O_x += P_x V
    if (lane == 0) {
      constexpr uint32_t idO = idesc_bf16(128, kD, 1);
      const uint64_t dV0 = sw128_desc(smem_u32(smem + C::kV), 16384, 1024);  // MN-major (K = keys)
      uint32_t G = 0, GX[2] = {0, 0}, WX[2] = {0, 0};
      bool ok = true;
      for (int w = blockIdx.x; w < a.items && ok; w += gridDim.x) {
        int bh, tile, pair;
        decode_pair(a, w, bh, tile, pair);
        TileBlocks tbk;
        tile_blocks(g, tile, tbk);
        const int qa = 2 * pair;
        if (qa >= tbk.NB) continue;
        const int nact = qa + 1 < tbk.NB ? 2 : 1;
        for (int j = 0; j < tbk.NB && ok; ++j, ++G) {
          const uint32_t st = G % kStages;
          if (!(ok = WAIT(v_full + st, (G / kStages) & 1))) break;
          const uint64_t dv = dmove(dV0, st * kBox);
#pragma unroll
          for (int x = 0; x < 2; ++x) {
            if (x >= nact) break;
            if (!(ok = WAIT(p_full(x), GX[x] & 1))) break;
            if (j == 0 && !(ok = WAIT(o_empty(x), (WX[x] & 1) ^ 1))) break;
            tc_fence_after();
#pragma unroll
            for (int ks = 0; ks < 8; ++ks)
              umma_bf16_ts(tmem + col_o(x), tmem + col_s(x) + ks * 8, dmove(dv, ks * 2048), idO,
                           (j > 0 || ks > 0) ? 1u : 0u);
            umma_commit(pv_done(x));
            ++GX[x];
          }
          if (!ok) break;
          umma_commit(v_empty + st);
        }
#pragma unroll
        for (int x = 0; x < 2; ++x)
          if (x < nact) ++WX[x];
      }
      umma_commit(drain + 1);
      mbar_wait<set_status_f64>(drain + 1, 0, abort_flag, false);
    }
  } else {
    // ------------------------------------------------------------ softmax + epilogue of box x
    const int x = (warp - kSoft0) >> 2;
    const int quad = warp & 3;
    const int row = quad * 32 + lane;  // TMEM lane = query row of the box
    const uint32_t tl = tmem + ((uint32_t)(quad * 32) << 16);
    const uint32_t tS = tl + col_s(x), tO = tl + col_o(x);
    const float sl2 = g.scale_log2;
    uint32_t GX = 0, W = 0;
    bool ok = true;
    for (int w = blockIdx.x; w < a.items && ok; w += gridDim.x) {
      int bh, tile, pair;
      decode_pair(a, w, bh, tile, pair);
      TileBlocks tbk;
      tile_blocks(g, tile, tbk);
      const int qa = 2 * pair;
      if (qa >= tbk.NB) continue;
      const bool active = qa + x < tbk.NB;
      // the query boxes: shared memory (TMA) -> TMEM (A operand of S = Q K^T);
      // both groups take part in the Q handshake of every item
      if (!(ok = WAIT(q_full, W & 1))) break;
      ++W;
      if (active) {
        uint32_t qr[32];
        ld_swizzled_row<8>(smem_u32(smem + C::kQ + x * kBox), row, 0, qr);
        tmem_st32(tl + col_q(x), qr);
        tmem_wait_st();
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(q_empty);
        if (active) mbar_arrive(qt_full(x));
      }
      if (!active) continue;
      const int qb = qa + x;
      int qo[3], ql[3];
      block_origin(g, tbk, qb, qo);
      block_row(g, qo, row, ql);
      const bool qvalid = inside(tbk, ql);
      float m = -INFINITY, l = 0.f;
      int jt = 0, jy = 0, jx = 0;
      for (int j = 0; j < tbk.NB; ++j, ++GX) {
        const int ko[3] = {jt << g.lt, jy << g.ly, jx << g.lx};
        if (++jx == tbk.nb[2]) {
          jx = 0;
          if (++jy == tbk.nb[1]) {
            jy = 0;
            ++jt;
          }
        }
        uint32_t km[4] = {~0u, ~0u, ~0u, ~0u};
        const bool full = block_full(g, tbk, ko);
        if (!full) {
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            int kl[3];
            block_row(g, ko, c * 32 + lane, kl);
            km[c] = __ballot_sync(0xffffffffu, inside(tbk, kl));
          }
        }
        if (!(ok = WAIT(s_full(x), GX & 1))) break;
        tc_fence_after();
        if (full)
          softmax_box<false>(m, l, tS, tO, km, sl2, j == 0);
        else
          softmax_box<true>(m, l, tS, tO, km, sl2, j == 0);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(p_full(x));
      }
      if (!ok) break;
      // ---- epilogue: wait for the last P V, O / l
      if (!(ok = WAIT(pv_done(x), (GX - 1) & 1))) break;
      tc_fence_after();
      const float inv = 1.f / l;
      const int64_t slot = tile_slot0(g, bh, tile) + qb * 128 + row;
      if (qvalid && a.lse2) a.lse2[slot] = m + __log2f(l);
      const int p[3] = {tbk.tb.lo[0] + ql[0], tbk.tb.lo[1] + ql[1], tbk.tb.lo[2] + ql[2]};
      const int64_t tok = qvalid ? ((int64_t)p[0] * g.G[1] + p[1]) * g.G[2] + p[2] : 0;
      const bool single = qvalid && single_cover(g, p);
      OutT* dst_out = static_cast<OutT*>(a.out) + ((int64_t)bh * g.N + tok) * kD;
      float* dst_scr = a.ot + slot * kD;
      uint32_t r[32];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        tmem_ld32(tO + c * 32, r);
        tmem_wait_ld(r);
        if (qvalid) {
#pragma unroll
          for (int e = 0; e < 32; e += 4) {
            const float4 v4 = make_float4(__uint_as_float(r[e]) * inv, __uint_as_float(r[e + 1]) * inv,
                                          __uint_as_float(r[e + 2]) * inv, __uint_as_float(r[e + 3]) * inv);
            if (single)
              store4<OutT>(dst_out + c * 32 + e, v4);
            else
              store4<float>(dst_scr + c * 32 + e, v4);
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(o_empty(x));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

template <typename OutT>
cudaError_t run_fwd64(const Geom& g, const __nv_bfloat16* q, const __nv_bfloat16* k, const __nv_bfloat16* v,
                      void* out, float* lse2, float* ot, uint32_t flags, cudaStream_t st) {
  Fwd64Args a;
  a.g = g;
  a.out = out;
  a.lse2 = lse2;
  a.ot = ot;
  a.flags = flags;
  a.npairs = (g.nbmax_tot + 1) / 2;
  const int64_t items = (int64_t)g.B * g.nh * g.ntiles * a.npairs;
  if (items >= (1LL << 31)) return cudaErrorNotSupported;
  a.items = (int)items;
  const int BH = g.B * g.nh;
  CUtensorMap mq, mk, mv;
  if (!make_tmap_5d(&mq, q, kD, g.G[2], g.G[1], g.G[0], BH, g.bx, g.by, g.bt) ||
      !make_tmap_5d(&mk, k, kD, g.G[2], g.G[1], g.G[0], BH, g.bx, g.by, g.bt) ||
      !make_tmap_5d(&mv, v, kD, g.G[2], g.G[1], g.G[0], BH, g.bx, g.by, g.bt))
    return cudaErrorInvalidValue;
  auto kern = fwd64_kernel<OutT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::kSmem);
  if (e != cudaSuccess) return e;
  const int grid = (int)(a.items < num_sms() ? a.items : num_sms());
  kern<<<grid, kThreadsF, Cfg::kSmem, st>>>(mq, mk, mv, a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sm103_fwd64(const Geom& g, const __nv_bfloat16* q, const __nv_bfloat16* k, const __nv_bfloat16* v,
                               void* out, int out_dtype, float* lse2, float* ot, uint32_t flags, cudaStream_t st) {
  if (g.d != kD) return cudaErrorNotSupported;
  if (out_dtype == GATTN_BF16) return run_fwd64<__nv_bfloat16>(g, q, k, v, out, lse2, ot, flags, st);
  return run_fwd64<float>(g, q, k, v, out, lse2, ot, flags, st);
}

}  // namespace gattn
