// sm103_bwd.cu -- BF16 tensor-core backward of STORM-GPA tile attention for
// head size d = 128 on GB300 (sm_103a); d = 64 runs sm103_bwd64.cu.  Two
// deterministic kernels (no atomics), every product over whole 128-token
// boxes (M = N = 128):
//
//   dK/dV kernel, one work item per (batch*head, tile, 128-key box kb):
//     for every 128-query box i of the tile:
//       S'^T  = K Q_i^T  + 1 x_i^T,  x = -lse' / (scale log2 e)      8 + 1 K-steps
//       dP'^T = V dO_i^T + 1 y_i^T,  y = -D                          8 + 1 K-steps
//       P'^T = exp2(scale log2e S'^T),  dS^T = P'^T * dP'^T          math warps, BF16 pairs -> TMEM
//       dV += P'^T dO_i,  dK += dS^T Q_i                             A from TMEM, FP32 in TMEM
//   dQ kernel, one work item per (batch*head, tile, 128-query box qb):
//     for every 128-key box j of the tile:
//       S = Q K_j^T (+ 1 b_j^T, b = -1e30 on keys outside the tile),  dP = dO V_j^T
//       dS = P' (dP - D),  dQ += dS K_j                              A from TMEM, FP32 in TMEM
//
// TMEM at d = 128: the two accumulators of the dK/dV kernel take 256 of the
// 512 columns and its two score matrices the other 256, so the packed P'^T
// and dS^T are written over the FP32 scores they come from (each math warp
// packs the 32 columns it read into the first 16 of them).  The next box's
// S'^T therefore waits for this box's dV product, the reader of P'^T, and its
// dP'^T for the dK product; with one issuing thread per product pair those
// waits overlap the other pair's MMAs.  The dQ kernel copies the item's Q and
// dOut into TMEM (S 0, dP 128, dQ 256, Q 384, dOut 448) and packs its dS over
// the dP it comes from.
//
// Shared memory (one operand box = 32 KB, two 64-element halves of 128-byte
// rows): the dK/dV kernel holds the item's K and V and a two-stage ring of
// (Q, dO, statistics rows); the dQ kernel stages the item's Q and dO (for the
// copy into TMEM) and has a two-stage ring of (K, V, key-bias row).  A work item streams every box of its tile,
// so one K, V (resp. Q, dO) buffer per item costs one load wait per item.
//
// The merge weight of the Hann-weighted overlap average (arXiv 2604.16590,
// Sec. III-C) enters through lse' = lse - log2(w_t / sum w), which makes P'
// the probabilities of the per-tile gradient dO_t = (w_t / sum w) dOut, and
// D = dOut . O_t.  The statistics of a query slot enter the dK/dV scores as
// one extra K = 16 MMA step against a constant A operand of ones (the prep
// pass writes each slot's -lse' / (scale log2 e) and -D as sums of three BF16
// terms).  Rows covered by one tile are written straight to dQ/dK/dV;
// multiply-covered rows go to FP32 per-tile slots that the merge kernel sums
// in fixed tile order.
//
// Warp roles: warp 0 TMA producer, warp 1 TMEM allocator + issuer of the
// score products, warp 2 issuer of the gradient products, warps 3..18
// elementwise math + epilogue: one TMEM lane = one box row, four warps per
// lane quadrant, each taking 32 of the row's 128 score columns.  Two issuing
// threads, because a thread's mbarrier wait is held until the tcgen05.mma it
// issued before it have drained from the tensor pipe.
#include "sm103_bwd_common.cuh"

GATTN_DEFINE_STATUS(sm103_bwd)

namespace gattn {
namespace {
using namespace sm103;

__device__ void set_status_bwd(uint32_t c) { set_status(c); }
#define WAIT(bar, par) mbar_wait<set_status_bwd>((bar), (par), abort_flag)

constexpr int kD = 128;
constexpr int kBox = 128 * kD * 2;  // one 128-token box of one operand, BF16, 32 KB

// TMEM column of K-step ks (16 BF16 values = 8 packed columns) of an operand
// that warp c4 packed into the first 16 of its 32 columns [32 c4, 32 c4 + 32)
__device__ __forceinline__ uint32_t inplace_col(int ks) { return 32 * (ks >> 1) + 8 * (ks & 1); }

// =============================================================== dK / dV
struct Kv128 {
  static constexpr int kStages = 2;  // (Q, dOut, statistics rows) ring
  static constexpr int kK = 0;
  static constexpr int kV = kBox;
  static constexpr int kQ = 2 * kBox;  // stage s: Q at kQ + s*2*kBox, dOut after it
  // A: ones in K 0..2 at kOnes, ones in K 3..5 at kOnes + 4096; B, stage s at
  // kExt + s*4096: the box's 128 statistics rows, each block followed by 2 KB of zeros
  static constexpr int kOnes = kQ + kStages * 2 * kBox;
  static constexpr int kExt = kOnes + 2 * 4096;
  static constexpr int kBar = kExt + kStages * 4096;
  // kv_full, kv_empty, qd_full[S], qd_empty[S], s_full[2], p_full[2], p_empty[2],
  // acc_full, acc_empty, drain[2]   ([0]: the S'^T / P'^T / dV chain, [1]: dP'^T / dS^T / dK)
  static constexpr int kNumBars = 2 + 2 * kStages + 6 + 4;
  static constexpr int kMisc = kBar + kNumBars * 8;
  static constexpr int kSmem = kMisc + 16 + 1024;
  // TMEM: S'^T (then P'^T packed) 0, dP'^T (then dS^T packed) 128, dV 256, dK 384
  static constexpr uint32_t kColST = 0, kColDP = 128, kColDV = 256, kColDK = 384;
};

template <typename OutT>
__global__ void __launch_bounds__(kThreadsB, 1)
    dkdv128_kernel(const __grid_constant__ CUtensorMap tq, const __grid_constant__ CUtensorMap tk,
                   const __grid_constant__ CUtensorMap tv, const __grid_constant__ CUtensorMap tdo,
                   const BwdArgs a) {
  using C = Kv128;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::kBar);
  uint64_t* kv_full = bars;
  uint64_t* kv_empty = bars + 1;
  uint64_t* qd_full = bars + 2;
  uint64_t* qd_empty = qd_full + C::kStages;
  uint64_t* s_full = qd_empty + C::kStages;  // [2]: S'^T, dP'^T computed
  uint64_t* p_full = s_full + 2;             // [2]: P'^T, dS^T packed in place
  uint64_t* p_empty = p_full + 2;            // [2]: dV, dK products of the box done
  uint64_t* acc_full = p_empty + 2;
  uint64_t* acc_empty = acc_full + 1;
  uint64_t* drain = acc_empty + 1;  // [2]: one per issuing thread
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + C::kMisc);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + C::kMisc + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  init_ext_operands(smem + C::kOnes, 2, true, smem + C::kExt, C::kStages);
  zero_pad_rows(smem, (2 + 2 * C::kStages) * 2, a.g.R);  // K, V and the Q / dOut ring (16 KB halves)
  fence_proxy_async_smem();
  if (threadIdx.x == 0) {
    mbar_init(kv_full, 1);
    mbar_init(kv_empty, 1);
    for (int s = 0; s < C::kStages; ++s) {
      mbar_init(qd_full + s, 1);
      mbar_init(qd_empty + s, 1);
    }
    for (int c = 0; c < 2; ++c) {
      mbar_init(s_full + c, 1);
      mbar_init(p_full + c, kMathW);
      mbar_init(p_empty + c, 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, kMathW);
    mbar_init(drain, 1);
    mbar_init(drain + 1, 1);
    *abort_flag = 0;
    fence_mbar_init();
    prefetch_tmap(&tq);
    prefetch_tmap(&tk);
    prefetch_tmap(&tv);
    prefetch_tmap(&tdo);
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
      uint32_t kv_arm = 0, kv_par = 0, qd_arm = 0, qd_par = 0;
      bool ok = true;
      for (int w = blockIdx.x; w < a.items && ok; w += gridDim.x) {
        int bh, tile, kb;
        decode_item(g, w, bh, tile, kb);
        TileBlocks tbk;
        tile_blocks(g, tile, tbk);
        if (kb >= tbk.NB) continue;
        int o[3];
        block_origin(g, tbk, kb, o);
        if (!(ok = WAIT(kv_empty, (W & 1) ^ 1))) break;
        mbar_arrive_expect_tx(kv_full, 4 * g.R * 128);
        kv_arm = 1;
        kv_par = W & 1;
        for (int h = 0; h < 2; ++h) {
          tma_load_5d(smem + C::kK + h * 16384, &tk, kv_full, 64 * h, tbk.tb.lo[2] + o[2], tbk.tb.lo[1] + o[1],
                      tbk.tb.lo[0] + o[0], bh);
          tma_load_5d(smem + C::kV + h * 16384, &tv, kv_full, 64 * h, tbk.tb.lo[2] + o[2], tbk.tb.lo[1] + o[1],
                      tbk.tb.lo[0] + o[0], bh);
        }
        const int64_t slot0 = tile_slot0(g, bh, tile);
        BlockWalk bw;
        for (int i = 0; i < tbk.NB; ++i, ++G, bw.next(tbk)) {
          const uint32_t st = G % C::kStages, n = G / C::kStages;
          const int c1 = tbk.tb.lo[2] + bw.jx * g.bx, c2 = tbk.tb.lo[1] + bw.jy * g.by,
                    c3 = tbk.tb.lo[0] + bw.jt * g.bt;
          if (!(ok = WAIT(qd_empty + st, (n & 1) ^ 1))) break;
          mbar_arrive_expect_tx(qd_full + st, 4 * g.R * 128 + 2048);
          qd_arm |= 1u << st;
          qd_par = (qd_par & ~(1u << st)) | ((n & 1) << st);
          uint8_t* sq = smem + C::kQ + st * 2 * kBox;
          for (int h = 0; h < 2; ++h) {
            tma_load_5d(sq + h * 16384, &tq, qd_full + st, 64 * h, c1, c2, c3, bh);
            tma_load_5d(sq + kBox + h * 16384, &tdo, qd_full + st, 64 * h, c1, c2, c3, bh);
          }
          bulk_load(smem + C::kExt + st * 4096, a.ext + slot0 + i * 128, 2048, qd_full + st);
        }
        ++W;
      }
      if (!ok) {
        if (kv_arm) mbar_wait<set_status_bwd>(kv_full, kv_par, abort_flag, false);
        for (int s = 0; s < C::kStages; ++s)
          if (qd_arm & (1u << s)) mbar_wait<set_status_bwd>(qd_full + s, (qd_par >> s) & 1, abort_flag, false);
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ issuer of S'^T, dP'^T
    if (lane == 0) {
      constexpr uint32_t idS = idesc_bf16(128, 128, 0);
      const uint32_t sK = smem_u32(smem + C::kK), sV = smem_u32(smem + C::kV), sQ = smem_u32(smem + C::kQ);
      const uint64_t dOnesS = noswz_desc(smem_u32(smem + C::kOnes), 2048, 128);
      const uint64_t dOnesD = dmove(dOnesS, 4096);
      const uint64_t dExt0 = noswz_desc(smem_u32(smem + C::kExt), 2048, 128);
      uint32_t G = 0, W = 0;
      bool ok = true;
      for (int w = blockIdx.x; w < a.items && ok; w += gridDim.x) {
        int bh, tile, kb;
        decode_item(g, w, bh, tile, kb);
        TileBlocks tbk;
        tile_blocks(g, tile, tbk);
        if (kb >= tbk.NB) continue;
        if (!(ok = WAIT(kv_full, W & 1))) break;
        for (int i = 0; i < tbk.NB; ++i, ++G) {
          const uint32_t st = G % C::kStages;
          if (!(ok = WAIT(qd_full + st, (G / C::kStages) & 1))) break;
          // the S'^T columns hold box G-1's packed P'^T until its dV product is done
          if (G > 0 && !(ok = WAIT(p_empty, (G - 1) & 1))) break;
          tc_fence_after();
          const uint32_t sq = sQ + st * 2 * kBox, sdo = sq + kBox;
          const uint64_t de = dmove(dExt0, st * 4096);
#pragma unroll
          for (int ks = 0; ks < kD / 16; ++ks)
            umma_bf16(tmem + C::kColST, sw128_desc(sK + kmaj_off(ks), 16, 1024), sw128_desc(sq + kmaj_off(ks), 16, 1024),
                      idS, ks > 0);
          umma_bf16(tmem + C::kColST, dOnesS, de, idS, 1u);
          umma_commit(s_full);
          // the dP'^T columns hold box G-1's packed dS^T until its dK product is done
          if (G > 0 && !(ok = WAIT(p_empty + 1, (G - 1) & 1))) break;
          tc_fence_after();
#pragma unroll
          for (int ks = 0; ks < kD / 16; ++ks)
            umma_bf16(tmem + C::kColDP, sw128_desc(sV + kmaj_off(ks), 16, 1024),
                      sw128_desc(sdo + kmaj_off(ks), 16, 1024), idS, ks > 0);
          umma_bf16(tmem + C::kColDP, dOnesD, de, idS, 1u);
          umma_commit(s_full + 1);
          if (i == tbk.NB - 1) umma_commit(kv_empty);  // K, V of this item no longer read
        }
        ++W;
      }
      umma_commit(drain);
      mbar_wait<set_status_bwd>(drain, 0, abort_flag, false);
    }
  } else if (warp == kIssuerA) {
    // ------------------------------------------------------------ issuer of dV += P'^T dO, dK += dS^T Q
    if (lane == 0) {
      constexpr uint32_t idA = idesc_bf16(128, kD, 1);  // B MN-major (K = queries, N = d)
      const uint32_t sQ = smem_u32(smem + C::kQ);
      uint32_t G = 0, W = 0;
      bool ok = true;
      for (int w = blockIdx.x; w < a.items && ok; w += gridDim.x) {
        int bh, tile, kb;
        decode_item(g, w, bh, tile, kb);
        TileBlocks tbk;
        tile_blocks(g, tile, tbk);
        if (kb >= tbk.NB) continue;
        for (int i = 0; i < tbk.NB; ++i, ++G) {
          const uint32_t st = G % C::kStages;
          const uint32_t sq = sQ + st * 2 * kBox, sdo = sq + kBox;
          // p_full[c](G) implies s_full[c](G): the score product that read this
          // stage is complete, so the qd_empty commit below covers every reader
          if (!(ok = WAIT(p_full, G & 1))) break;
          if (i == 0 && !(ok = WAIT(acc_empty, (W & 1) ^ 1))) break;
          tc_fence_after();
#pragma unroll
          for (int ks = 0; ks < 8; ++ks)
            umma_bf16_ts(tmem + C::kColDV, tmem + C::kColST + inplace_col(ks),
                         sw128_desc(sdo + ks * 2048, 16384, 1024), idA, (i > 0 || ks > 0) ? 1u : 0u);
          umma_commit(p_empty);
          if (!(ok = WAIT(p_full + 1, G & 1))) break;
          tc_fence_after();
#pragma unroll
          for (int ks = 0; ks < 8; ++ks)
            umma_bf16_ts(tmem + C::kColDK, tmem + C::kColDP + inplace_col(ks),
                         sw128_desc(sq + ks * 2048, 16384, 1024), idA, (i > 0 || ks > 0) ? 1u : 0u);
          umma_commit(p_empty + 1);
          umma_commit(qd_empty + st);
        }
        if (!ok) break;
        umma_commit(acc_full);
        ++W;
      }
      umma_commit(drain + 1);
      mbar_wait<set_status_bwd>(drain + 1, 0, abort_flag, false);
    }
  } else {
    // ------------------------------------------------------------ elementwise + epilogue (row = key)
    const int quad = warp & 3;
    const int c4 = (warp - kMath0) >> 2;  // query columns [32 c4, 32 c4 + 32)
    const int row = quad * 32 + lane;
    const uint32_t tl = tmem + ((uint32_t)(quad * 32) << 16);
    const uint64_t s2 = f2pack(g.scale_log2, g.scale_log2);
    uint32_t G = 0, W = 0;
    bool ok = true;
    for (int w = blockIdx.x; w < a.items && ok; w += gridDim.x) {
      int bh, tile, kb;
      decode_item(g, w, bh, tile, kb);
      TileBlocks tbk;
      tile_blocks(g, tile, tbk);
      if (kb >= tbk.NB) continue;
      for (int i = 0; i < tbk.NB && ok; ++i, ++G) {
        if (!(ok = WAIT(s_full, G & 1))) break;
        tc_fence_after();
        uint32_t sv[32], dv[32], pk[16];
        tmem_ld32(tl + C::kColST + c4 * 32, sv);
        tmem_wait_ld(sv);
        kv_p(sv, s2, pk);  // sv <- P'^T (FP32), pk <- P'^T (BF16 pairs)
        tmem_st16(tl + C::kColST + c4 * 32, pk);
        tmem_wait_st();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(p_full);
        if (!(ok = WAIT(s_full + 1, G & 1))) break;
        tc_fence_after();
        tmem_ld32(tl + C::kColDP + c4 * 32, dv);
        tmem_wait_ld(dv);
        kv_ds(sv, dv, pk);  // dS^T = P'^T dP'^T (BF16 pairs)
        tmem_st16(tl + C::kColDP + c4 * 32, pk);
        tmem_wait_st();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(p_full + 1);
      }
      if (!ok) break;
      // ---- epilogue: this thread's key row of dK, dV (columns [32 c4, 32 c4 + 32))
      if (!(ok = WAIT(acc_full, W & 1))) break;
      tc_fence_after();
      int ko[3], kl[3];
      block_origin(g, tbk, kb, ko);
      block_row(g, ko, row, kl);
      const bool kvalid = inside(tbk, kl);
      const int p[3] = {tbk.tb.lo[0] + kl[0], tbk.tb.lo[1] + kl[1], tbk.tb.lo[2] + kl[2]};
      const int64_t tok = kvalid ? ((int64_t)p[0] * g.G[1] + p[1]) * g.G[2] + p[2] : 0;
      const bool single = kvalid && single_cover(g, p);
      const int64_t slot = tile_slot0(g, bh, tile) + kb * 128 + row;
      const int c0 = c4 * 32;
      // both accumulators into registers, then they are released at once: the
      // next item's first gradient products may overwrite them during the stores
      uint32_t rk[32], rv[32];
      tmem_ld32(tl + C::kColDK + c0, rk);
      tmem_ld32(tl + C::kColDV + c0, rv);
      tmem_wait_ld(rk);
      tmem_wait_ld(rv);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acc_empty);
      row_store<32, OutT>(rk, g.scale, kvalid, single, static_cast<OutT*>(a.dk) + ((int64_t)bh * g.N + tok) * kD + c0,
                          a.dk_s + slot * kD + c0);
      row_store<32, OutT>(rv, 1.f, kvalid, single, static_cast<OutT*>(a.dv) + ((int64_t)bh * g.N + tok) * kD + c0,
                          a.dv_s + slot * kD + c0);
      ++W;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// =============================================================== dQ
// Q and dOut of the item are copied once into TMEM (the A operands of S and
// dP), so the score products read only K (resp. V) from shared memory: with
// both operands there, an N = 128 K-step moves 8 KB against the SM's 128
// bytes per clock and the products would wait on shared memory.  That leaves
// no TMEM for separate dS buffers: each math warp packs its dS over the first
// 16 of the 32 dP columns it read, and the next box's dP waits for this box's
// dQ product.  S is released as soon as it is read, so the next box's S runs
// during the exponentials and the dQ product.
struct Q128 {
  static constexpr int kStages = 2;  // (K, V, key-bias row) ring
  static constexpr int kQ = 0;       // Q, dOut of the item, copied into TMEM by the math warps
  static constexpr int kDO = kBox;
  static constexpr int kK = 2 * kBox;  // stage s: K at kK + s*2*kBox, V after it
  // Key-mask extension operands (as in the forward): A = 1 in K-column 0 of
  // 128 rows, and per stage the key box's bias row (0, or -1e30 for a padding
  // key or a key outside the tile), each followed by 2 KB of zeros.
  static constexpr int kOnes = kK + kStages * 2 * kBox;
  static constexpr int kBias = kOnes + 4096;
  static constexpr int kBar = kBias + kStages * 4096;
  // qd_full, qd_empty, qt_full, kv_full[S], kv_empty[S], s_full[2], s_empty, p_full, p_empty,
  // acc_full, acc_empty, drain[2]   (s_full[0]: S, s_full[1]: dP)
  static constexpr int kNumBars = 3 + 2 * kStages + 2 + 4 + 4;
  static constexpr int kMisc = kBar + kNumBars * 8;
  static constexpr int kSmem = kMisc + 16 + 1024;
  // TMEM: S 0, dP (then dS packed) 128, dQ 256, Q (packed) 384, dOut (packed) 448
  static constexpr uint32_t kColS = 0, kColDP = 128, kColDQ = 256, kColQ = 384, kColDO = 448;
};

template <typename OutT>
__global__ void __launch_bounds__(kThreadsB, 1)
    dq128_kernel(const __grid_constant__ CUtensorMap tq, const __grid_constant__ CUtensorMap tk,
                 const __grid_constant__ CUtensorMap tv, const __grid_constant__ CUtensorMap tdo, const BwdArgs a) {
  using C = Q128;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::kBar);
  uint64_t* qd_full = bars;
  uint64_t* qd_empty = bars + 1;
  uint64_t* qt_full = bars + 2;
  uint64_t* kv_full = bars + 3;
  uint64_t* kv_empty = kv_full + C::kStages;
  uint64_t* s_full = kv_empty + C::kStages;  // [2]
  uint64_t* s_empty = s_full + 2;
  uint64_t* p_full = s_empty + 1;
  uint64_t* p_empty = p_full + 1;
  uint64_t* acc_full = p_empty + 1;
  uint64_t* acc_empty = acc_full + 1;
  uint64_t* drain = acc_empty + 1;  // [2]: one per issuing thread
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + C::kMisc);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + C::kMisc + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  init_ext_operands(smem + C::kOnes, 1, false, smem + C::kBias, C::kStages);
  zero_pad_rows(smem, (2 + 2 * C::kStages) * 2, a.g.R);  // Q, dOut and the K / V ring (16 KB halves)
  fence_proxy_async_smem();
  if (threadIdx.x == 0) {
    mbar_init(qd_full, 1);
    mbar_init(qd_empty, kMathW);
    mbar_init(qt_full, kMathW);
    for (int s = 0; s < C::kStages; ++s) {
      mbar_init(kv_full + s, 1);
      mbar_init(kv_empty + s, 1);
    }
    mbar_init(s_full, 1);
    mbar_init(s_full + 1, 1);
    mbar_init(s_empty, kMathW);
    mbar_init(p_full, kMathW);
    mbar_init(p_empty, 1);
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, kMathW);
    mbar_init(drain, 1);
    mbar_init(drain + 1, 1);
    *abort_flag = 0;
    fence_mbar_init();
    prefetch_tmap(&tq);
    prefetch_tmap(&tk);
    prefetch_tmap(&tv);
    prefetch_tmap(&tdo);
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
    // ------------------------------------------------------------ TMA producer (lane 0) and
    // key-mask rows (all lanes, for key boxes with padding rows or keys outside the tile)
    const uint32_t neg = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(-1e30f));
    uint32_t G = 0, W = 0;
    uint32_t qd_arm = 0, qd_par = 0, kv_arm = 0, kv_par = 0;
    bool ok = true;
    for (int w = blockIdx.x; w < a.items && ok; w += gridDim.x) {
      int bh, tile, qb;
      decode_item(g, w, bh, tile, qb);
      TileBlocks tbk;
      tile_blocks(g, tile, tbk);
      if (qb >= tbk.NB) continue;
      int o[3];
      block_origin(g, tbk, qb, o);
      if (lane == 0) {
        // the staging buffer is free once the math warps copied the previous item's Q, dOut
        if ((ok = WAIT(qd_empty, (W & 1) ^ 1))) {
          mbar_arrive_expect_tx(qd_full, 4 * g.R * 128);
          qd_arm = 1;
          qd_par = W & 1;
          for (int h = 0; h < 2; ++h) {
            tma_load_5d(smem + C::kQ + h * 16384, &tq, qd_full, 64 * h, tbk.tb.lo[2] + o[2], tbk.tb.lo[1] + o[1],
                        tbk.tb.lo[0] + o[0], bh);
            tma_load_5d(smem + C::kDO + h * 16384, &tdo, qd_full, 64 * h, tbk.tb.lo[2] + o[2], tbk.tb.lo[1] + o[1],
                        tbk.tb.lo[0] + o[0], bh);
          }
        }
      }
      if (!(ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0)) break;
      for (int j = 0; j < tbk.NB; ++j, ++G) {
        const uint32_t st = G % C::kStages, n = G / C::kStages;
        int ko[3];
        block_origin(g, tbk, j, ko);
        // the stage (K, V and its bias row) is free once box G - kStages is done
        if (lane == 0) ok = WAIT(kv_empty + st, (n & 1) ^ 1);
        if (!(ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0)) break;
        if (!block_full(g, tbk, ko)) {
          for (int r = lane; r < 128; r += 32) {
            int kl[3];
            block_row(g, ko, r, kl);
            *reinterpret_cast<uint4*>(smem + C::kBias + st * 4096 + r * 16) =
                make_uint4(inside(tbk, kl) ? 0u : neg, 0u, 0u, 0u);
          }
          fence_proxy_async_smem();
        }
        __syncwarp();
        if (lane == 0) {
          mbar_arrive_expect_tx(kv_full + st, 4 * g.R * 128);
          kv_arm |= 1u << st;
          kv_par = (kv_par & ~(1u << st)) | ((n & 1) << st);
          uint8_t* sk = smem + C::kK + st * 2 * kBox;
          for (int h = 0; h < 2; ++h) {
            tma_load_5d(sk + h * 16384, &tk, kv_full + st, 64 * h, tbk.tb.lo[2] + ko[2], tbk.tb.lo[1] + ko[1],
                        tbk.tb.lo[0] + ko[0], bh);
            tma_load_5d(sk + kBox + h * 16384, &tv, kv_full + st, 64 * h, tbk.tb.lo[2] + ko[2],
                        tbk.tb.lo[1] + ko[1], tbk.tb.lo[0] + ko[0], bh);
          }
        }
      }
      ++W;
    }
    if (!ok && lane == 0) {
      if (qd_arm) mbar_wait<set_status_bwd>(qd_full, qd_par, abort_flag, false);
      for (int s = 0; s < C::kStages; ++s)
        if (kv_arm & (1u << s)) mbar_wait<set_status_bwd>(kv_full + s, (kv_par >> s) & 1, abort_flag, false);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ issuer of S, dP
    if (lane == 0) {
      constexpr uint32_t idS = idesc_bf16(128, 128, 0);
      const uint32_t sK = smem_u32(smem + C::kK);
      const uint64_t dOnes = noswz_desc(smem_u32(smem + C::kOnes), 2048, 128);
      const uint64_t dBias0 = noswz_desc(smem_u32(smem + C::kBias), 2048, 128);
      uint32_t G = 0, W = 0;
      bool ok = true;
      for (int w = blockIdx.x; w < a.items && ok; w += gridDim.x) {
        int bh, tile, qb;
        decode_item(g, w, bh, tile, qb);
        TileBlocks tbk;
        tile_blocks(g, tile, tbk);
        if (qb >= tbk.NB) continue;
        if (!(ok = WAIT(qt_full, W & 1))) break;  // Q, dOut in TMEM
        const bool all_full = tile_all_full(g, tbk);
        BlockWalk bw;
        for (int j = 0; j < tbk.NB; ++j, ++G, bw.next(tbk)) {
          const uint32_t st = G % C::kStages;
          // a masked box's bias row was filled by the producer warp
          const bool masked = !all_full && !bw.full(g, tbk);
          if (!(ok = WAIT(kv_full + st, (G / C::kStages) & 1))) break;
          if (G > 0 && !(ok = WAIT(s_empty, (G - 1) & 1))) break;  // S of box G-1 read
          tc_fence_after();
          const uint32_t sk = sK + st * 2 * kBox, sv = sk + kBox;
#pragma unroll
          for (int ks = 0; ks < kD / 16; ++ks)
            umma_bf16_ts(tmem + C::kColS, tmem + C::kColQ + ks * 8, sw128_desc(sk + kmaj_off(ks), 16, 1024), idS,
                         ks > 0);
          // masked keys get -1e30, so P' = 0 there and dS = 0 follows
          if (masked) umma_bf16(tmem + C::kColS, dOnes, dmove(dBias0, st * 4096), idS, 1u);
          umma_commit(s_full);
          // the dP columns hold box G-1's packed dS until its dQ product is done
          if (G > 0 && !(ok = WAIT(p_empty, (G - 1) & 1))) break;
          tc_fence_after();
#pragma unroll
          for (int ks = 0; ks < kD / 16; ++ks)
            umma_bf16_ts(tmem + C::kColDP, tmem + C::kColDO + ks * 8, sw128_desc(sv + kmaj_off(ks), 16, 1024), idS,
                         ks > 0);
          umma_commit(s_full + 1);
        }
        ++W;
      }
      umma_commit(drain);
      mbar_wait<set_status_bwd>(drain, 0, abort_flag, false);
    }
  } else if (warp == kIssuerA) {
    // ------------------------------------------------------------ issuer of dQ += dS K
    if (lane == 0) {
      constexpr uint32_t idA = idesc_bf16(128, kD, 1);  // B MN-major (K = keys, N = d)
      const uint32_t sK = smem_u32(smem + C::kK);
      uint32_t G = 0, W = 0;
      bool ok = true;
      for (int w = blockIdx.x; w < a.items && ok; w += gridDim.x) {
        int bh, tile, qb;
        decode_item(g, w, bh, tile, qb);
        TileBlocks tbk;
        tile_blocks(g, tile, tbk);
        if (qb >= tbk.NB) continue;
        for (int j = 0; j < tbk.NB; ++j, ++G) {
          const uint32_t st = G % C::kStages;
          // p_full(G) implies s_full[0,1](G): the score products of this stage
          // are complete, so the kv_empty commit below covers every reader
          if (!(ok = WAIT(p_full, G & 1))) break;
          if (j == 0 && !(ok = WAIT(acc_empty, (W & 1) ^ 1))) break;
          tc_fence_after();
          const uint32_t sk = sK + st * 2 * kBox;
#pragma unroll
          for (int ks = 0; ks < 8; ++ks)
            umma_bf16_ts(tmem + C::kColDQ, tmem + C::kColDP + inplace_col(ks), sw128_desc(sk + ks * 2048, 16384, 1024),
                         idA, (j > 0 || ks > 0) ? 1u : 0u);
          umma_commit(p_empty);
          umma_commit(kv_empty + st);
        }
        if (!ok) break;
        umma_commit(acc_full);
        ++W;
      }
      umma_commit(drain + 1);
      mbar_wait<set_status_bwd>(drain + 1, 0, abort_flag, false);
    }
  } else {
    // ------------------------------------------------------------ elementwise + epilogue (row = query)
    const int quad = warp & 3;
    const int c4 = (warp - kMath0) >> 2;  // key columns [32 c4, 32 c4 + 32)
    const int row = quad * 32 + lane;
    const uint32_t tl = tmem + ((uint32_t)(quad * 32) << 16);
    const float sl2 = g.scale_log2;
    // Q and dOut of a query box: shared memory -> TMEM (A operands of S, dP),
    // elements [32 c4, 32 c4 + 32) of the row (16-byte units 4 (c4 & 1) .. +4
    // of the 64-element half c4 >> 1)
    auto copy_qdo = [&](uint32_t par) -> bool {
      if (!WAIT(qd_full, par)) return false;
      const uint32_t half = (uint32_t)(c4 >> 1) * 16384;
      uint32_t r16[16];
      ld_swizzled_row<4>(smem_u32(smem + C::kQ) + half, row, 4 * (c4 & 1), r16);
      tmem_st16(tl + C::kColQ + 16 * c4, r16);
      ld_swizzled_row<4>(smem_u32(smem + C::kDO) + half, row, 4 * (c4 & 1), r16);
      tmem_st16(tl + C::kColDO + 16 * c4, r16);
      tmem_wait_st();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(qd_empty);
        mbar_arrive(qt_full);
      }
      return true;
    };
    uint32_t G = 0, W = 0;
    bool ok = true, staged = false;  // staged: this item's Q, dOut were copied during the previous item
    for (int w = blockIdx.x; w < a.items && ok; w += gridDim.x) {
      int bh, tile, qb;
      decode_item(g, w, bh, tile, qb);
      TileBlocks tbk;
      tile_blocks(g, tile, tbk);
      if (qb >= tbk.NB) continue;
      const int64_t qslot = tile_slot0(g, bh, tile) + qb * 128 + row;
      const float nL = a.lse2c[qslot];  // -lse' (-inf for padding rows)
      const float nD = a.dd[qslot];     // -D
      if (!staged && !(ok = copy_qdo(W & 1))) break;
      staged = false;
      // the next item's Q, dOut are copied once this item's last score
      // products are complete, so its first S and dP run during this item's
      // epilogue
      bool has_next = false;
      for (int wn = w + gridDim.x; wn < a.items && !has_next; wn += gridDim.x) {
        int bh2, tile2, qb2;
        decode_item(g, wn, bh2, tile2, qb2);
        TileBlocks t2;
        tile_blocks(g, tile2, t2);
        has_next = qb2 < t2.NB;
      }
      for (int j = 0; j < tbk.NB && ok; ++j, ++G) {
        if (!(ok = WAIT(s_full, G & 1))) break;
        tc_fence_after();
        uint32_t sv[32], dv[32], pk[16];
        tmem_ld32(tl + C::kColS + c4 * 32, sv);
        tmem_wait_ld(sv);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(s_empty);  // the next box's S may overwrite this one
        q_p(sv, sl2, nL);  // sv <- P' (FP32); masked keys carry -1e30 from the extension step
        if (!(ok = WAIT(s_full + 1, G & 1))) break;
        tc_fence_after();
        tmem_ld32(tl + C::kColDP + c4 * 32, dv);
        tmem_wait_ld(dv);
        q_ds(sv, dv, nD, pk);
        // dS over the dP columns this warp read: dP of box G was computed after
        // the dQ product of box G-1 had read its dS there
        tmem_st16(tl + C::kColDP + c4 * 32, pk);
        tmem_wait_st();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(p_full);
        // s_full[1] of the last box covers every score product of the item:
        // Q, dOut in TMEM are no longer read
        if (j == tbk.NB - 1 && has_next) {
          if (!(ok = copy_qdo((W + 1) & 1))) break;
          staged = true;
        }
      }
      if (!ok) break;
      if (!(ok = WAIT(acc_full, W & 1))) break;
      tc_fence_after();
      int qo[3], ql[3];
      block_origin(g, tbk, qb, qo);
      block_row(g, qo, row, ql);
      const bool qvalid = inside(tbk, ql);
      const int p[3] = {tbk.tb.lo[0] + ql[0], tbk.tb.lo[1] + ql[1], tbk.tb.lo[2] + ql[2]};
      const int64_t tok = qvalid ? ((int64_t)p[0] * g.G[1] + p[1]) * g.G[2] + p[2] : 0;
      const bool single = qvalid && single_cover(g, p);
      const int c0 = c4 * 32;
      uint32_t rq[32];
      tmem_ld32(tl + C::kColDQ + c0, rq);
      tmem_wait_ld(rq);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acc_empty);  // released before the stores
      row_store<32, OutT>(rq, g.scale, qvalid, single, static_cast<OutT*>(a.dq) + ((int64_t)bh * g.N + tok) * kD + c0,
                          a.dq_s + qslot * kD + c0);
      ++W;
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
cudaError_t run_bwd128(const Geom& g, const __nv_bfloat16* q, const __nv_bfloat16* k, const __nv_bfloat16* v,
                       const __nv_bfloat16* dout, const float* lse2c, const float* dd, const void* ext, void* dq,
                       void* dk, void* dv, float* dq_s, float* dk_s, float* dv_s, cudaStream_t st) {
  if (!ext || reinterpret_cast<uintptr_t>(ext) % 16) return cudaErrorInvalidValue;
  BwdArgs a;
  a.g = g;
  a.lse2c = lse2c;
  a.dd = dd;
  a.ext = static_cast<const uint4*>(ext);
  a.dq = dq;
  a.dk = dk;
  a.dv = dv;
  a.dq_s = dq_s;
  a.dk_s = dk_s;
  a.dv_s = dv_s;
  const int64_t items = (int64_t)g.B * g.nh * g.ntiles * g.nbmax_tot;
  if (items >= (1LL << 31)) return cudaErrorNotSupported;
  a.items = (int)items;
  const int BH = g.B * g.nh;
  CUtensorMap mq, mk, mv, mdo;
  if (!make_tmap_5d(&mq, q, kD, g.G[2], g.G[1], g.G[0], BH, g.bx, g.by, g.bt) ||
      !make_tmap_5d(&mk, k, kD, g.G[2], g.G[1], g.G[0], BH, g.bx, g.by, g.bt) ||
      !make_tmap_5d(&mv, v, kD, g.G[2], g.G[1], g.G[0], BH, g.bx, g.by, g.bt) ||
      !make_tmap_5d(&mdo, dout, kD, g.G[2], g.G[1], g.G[0], BH, g.bx, g.by, g.bt))
    return cudaErrorInvalidValue;
  const int grid = (int)(a.items < num_sms() ? a.items : num_sms());
  auto k1 = dkdv128_kernel<OutT>;
  cudaError_t e = cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, Kv128::kSmem);
  if (e != cudaSuccess) return e;
  prof_begin(kKBwdDkdv, st);
  k1<<<grid, kThreadsB, Kv128::kSmem, st>>>(mq, mk, mv, mdo, a);
  prof_end(kKBwdDkdv, st);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  auto k2 = dq128_kernel<OutT>;
  e = cudaFuncSetAttribute(k2, cudaFuncAttributeMaxDynamicSharedMemorySize, Q128::kSmem);
  if (e != cudaSuccess) return e;
  prof_begin(kKBwdDq, st);
  k2<<<grid, kThreadsB, Q128::kSmem, st>>>(mq, mk, mv, mdo, a);
  prof_end(kKBwdDq, st);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sm103_bwd(const Geom& g, const __nv_bfloat16* q, const __nv_bfloat16* k, const __nv_bfloat16* v,
                             const __nv_bfloat16* dout, const float* lse2c, const float* dd, const void* ext,
                             void* dq, void* dk, void* dv, int out_dtype, float* dq_s, float* dk_s, float* dv_s,
                             uint32_t, cudaStream_t st) {
  if (g.d == 64)
    return launch_sm103_bwd64(g, q, k, v, dout, lse2c, dd, ext, dq, dk, dv, out_dtype, dq_s, dk_s, dv_s, st);
  if (g.d != kD) return cudaErrorNotSupported;
  if (out_dtype == GATTN_BF16)
    return run_bwd128<__nv_bfloat16>(g, q, k, v, dout, lse2c, dd, ext, dq, dk, dv, dq_s, dk_s, dv_s, st);
  return run_bwd128<float>(g, q, k, v, dout, lse2c, dd, ext, dq, dk, dv, dq_s, dk_s, dv_s, st);
}

}  // namespace gattn
