// sm103_bwd64.cu -- BF16 tensor-core backward of STORM-GPA tile attention for
// head size d = 64 on GB300 (sm_103a).  Two deterministic kernels (no atomics):
//
//   dK/dV kernel, one work item per (batch*head, tile, 128-key box kb):
//     for every 128-query box i of the tile:
//       S'^T  = K Q_i^T  + 1 x_i^T,  x = -lse' / (scale log2 e)      M = N = 128, 4 + 1 K-steps
//       dP'^T = V dO_i^T + 1 y_i^T,  y = -D                          M = N = 128, 4 + 1 K-steps
//       P'^T = exp2(scale log2e S'^T),  dS^T = P'^T * dP'^T          math warps, BF16 pairs -> TMEM
//       dV += P'^T dO_i,  dK += dS^T Q_i                             A from TMEM, FP32 in TMEM
//   dQ kernel, one work item per (batch*head, tile, 128-query box qb):
//     for every 128-key box j of the tile:
//       S = Q K_j^T, dP = dO V_j^T (Q, dO copied once per item into TMEM),
//       dS = P' (dP - D) (keys outside the tile masked), dQ += dS K_j.
//
// Why this shape on this part: a tcgen05 MMA step with N = 64 costs about 54
// SM cycles against 64 for N = 128, so the score products run over whole
// 128-token boxes; only the gradient products (N = d = 64) keep the narrow
// shape.  The packed P'/dS operand has its own TMEM columns, so the next box's
// score products start as soon as the math warps have read the current scores
// (s_empty), while the gradient products of the current box wait only for
// the packed values (p_full).  The two score chains (S and dP) have their own
// ready/free barriers: the math warps exponentiate S while dP is still being
// computed, and the next box's S chain starts once S (not S and dP) was read.  The packed operand and its gradient products
// come in two halves (K-steps 0..3 and 4..7, written by the warps of column
// groups 0-1 and 2-3) with a ready and a free barrier each: a half of box G can
// be written while the other half of box G-1 is still being read, so the
// barrier round trips between the math warps and the gradient-product issuer
// overlap tensor work instead of stalling it.  In the dK/dV kernel the per-query statistics
// (-lse' and -D are per column there) enter through one extra K = 16 MMA step
// against a constant A operand of ones, instead of a broadcast load per
// element: the prep pass writes each slot's values as sums of three BF16 terms
// (FP32-accurate), K-columns 0..2 for -lse' / (scale log2 e) and 3..5 for -D.
//
// The merge weight of the Hann-weighted overlap average (arXiv 2604.16590,
// Sec. III-C) enters through lse' = lse - log2(w_t / sum w), which makes P'
// the probabilities of the per-tile gradient dO_t = (w_t / sum w) dOut, and
// D = dOut . O_t.  Rows covered by one tile are written straight to
// dQ/dK/dV; multiply-covered rows go to FP32 per-tile slots that the merge
// kernel sums in fixed tile order.
//
// Warp roles: warp 0 TMA producer, warp 1 TMEM allocator + issuer of the
// score products, warp 2 issuer of the gradient products, warps 3..18
// elementwise math + epilogue: one TMEM lane = one box row, four warps per
// lane quadrant, each taking 32 of the row's 128 columns (a warp reads its
// scores with one load per operand and releases them at once; four warps per
// SM sub-partition hide the TMEM and MUFU latencies).  Several issuing
// threads, because a thread's shared-memory accesses (an mbarrier wait
// included) are held until the tcgen05.mma it issued before them have drained
// from the tensor pipe: with one issuer every wait between two product groups
// empties the pipe; with two, one thread's waits overlap the other's MMAs.
// The dQ kernel gives the dP chain a third issuer (warp 19), so that the next
// box's S chain goes out as soon as the current S was read, whatever the dP
// chain still has in the pipe (dQ kernel 313 -> 300 ms on the paper-regime
// workload).  In the dK/dV kernel the same split measured slower (401 -> 430
// ms): there the next S chain then overtakes the current dP chain, which the
// math warps wait for, so one thread keeps issuing S, dP, S, dP in that order.
// (The d = 128 dQ kernel, whose dP chain waits for the previous dQ product,
// was slower with the split as well: 6.21 -> 6.45 s on the long-context case.)
// The tensor pipe interleaves the threads' streams; the barriers below order
// every TMEM region and shared-memory stage they share.
#include "sm103_bwd_common.cuh"

GATTN_DEFINE_STATUS(sm103_bwd64)

namespace gattn {
namespace {
using namespace sm103;

__device__ void set_status_bwd64(uint32_t c) { set_status(c); }
#define WAIT(bar, par) mbar_wait<set_status_bwd64>((bar), (par), abort_flag)

constexpr int kD = 64;
constexpr int kBox = 128 * kD * 2;  // one 128-token box of one operand, BF16, 16 KB
constexpr int kMath64 = kMathW;      // math warps: 4 per TMEM lane quadrant
constexpr int kThreads64 = kThreadsB;  // dK/dV kernel
constexpr int kIssuerD = kMath0 + kMath64;  // dQ kernel: issuer of the dP chain (after the math warps)
constexpr int kThreadsQ64 = kThreadsB + 32;

// =============================================================== dK / dV
struct Kv64 {
  static constexpr int kStages = 4;  // (Q, dOut, statistics rows) ring
  // two (K, V) buffers, items alternate: buffer b holds K at kK + 2 b kBox, V after it
  static constexpr int kK = 0;
  static constexpr int kQ = 4 * kBox;  // stage s: Q at kQ + s*2*kBox, dOut after it
  // Extension operands, K-major without swizzle: 128 rows x 16 B (K-columns
  // 0..7) followed by 2 KB of zeros (K-columns 8..15, lbo = 2048).
  static constexpr int kOnes = kQ + kStages * 2 * kBox;  // A: ones in K 0..2 at kOnes, ones in K 3..5 at kOnes+4096
  static constexpr int kExt = kOnes + 2 * 4096;            // B, stage s at kExt + s*4096: the 128 statistics rows
  static constexpr int kBar = kExt + kStages * 4096;
  // kv_full[2], kv_empty[2], qd_full[S], qd_empty[S], s_full[2], s_empty[2], p_full[2], p_empty[2],
  // acc_full, acc_empty, drain[2]   (s_*[0]: the S chain, s_*[1]: the dP chain)
  static constexpr int kNumBars = 4 + 2 * kStages + 12;
  static constexpr int kMisc = kBar + kNumBars * 8;
  static constexpr int kSmem = kMisc + 16 + 1024;
  // TMEM: S'^T 0, dP'^T 128, P'^T (packed) 256, dS^T (packed) 320, dV 384, dK 448
  static constexpr uint32_t kColST = 0, kColDP = 128, kColP = 256, kColDS = 320, kColDV = 384, kColDK = 448;
};

template <typename OutT>
__global__ void __launch_bounds__(kThreads64, 1)
    dkdv64_kernel(const __grid_constant__ CUtensorMap tq, const __grid_constant__ CUtensorMap tk,
                  const __grid_constant__ CUtensorMap tv, const __grid_constant__ CUtensorMap tdo,
                  const BwdArgs a) {
  using C = Kv64;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::kBar);
  uint64_t* kv_full = bars;       // [2]
  uint64_t* kv_empty = bars + 2;  // [2]
  uint64_t* qd_full = bars + 4;
  uint64_t* qd_empty = qd_full + C::kStages;
  uint64_t* s_full = qd_empty + C::kStages;
  uint64_t* s_empty = s_full + 2;
  uint64_t* p_full = s_empty + 2;   // [2]: one per half of the packed operand
  uint64_t* p_empty = p_full + 2;   // [2]
  uint64_t* acc_full = p_empty + 2;
  uint64_t* acc_empty = acc_full + 1;
  uint64_t* drain = acc_empty + 1;  // [2]: one per issuing thread
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + C::kMisc);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + C::kMisc + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // constant A operands of the extension step (128 rows of ones in K 0..2,
  // resp. 3..5) and the zero halves (K 8..15) of every extension operand
  for (int r = threadIdx.x; r < 2 * 256 + C::kStages * 128; r += kThreads64) {
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    uint8_t* dst;
    if (r < 512) {
      const int blk = r >> 8, rr = r & 255;  // blk 0: ones in K 0..2, 1: ones in K 3..5; rows 128..255 zero
      if (rr < 128) v = blk == 0 ? make_uint4(0x3F803F80u, 0x00003F80u, 0u, 0u)   // (1, 1, 1, 0, 0, 0, 0, 0)
                                 : make_uint4(0u, 0x3F800000u, 0x3F803F80u, 0u);  // (0, 0, 0, 1, 1, 1, 0, 0)
      dst = smem + C::kOnes + blk * 4096 + rr * 16;
    } else {
      const int q = r - 512;
      dst = smem + C::kExt + (q >> 7) * 4096 + 2048 + (q & 127) * 16;
    }
    *reinterpret_cast<uint4*>(dst) = v;
  }
  zero_pad_rows(smem, 4 + 2 * C::kStages, a.g.R);  // both K, V buffers and the Q / dOut ring
  fence_proxy_async_smem();
  if (threadIdx.x == 0) {
    for (int b = 0; b < 2; ++b) {
      mbar_init(kv_full + b, 1);
      mbar_init(kv_empty + b, 1);
    }
    for (int s = 0; s < C::kStages; ++s) {
      mbar_init(qd_full + s, 1);
      mbar_init(qd_empty + s, 1);
    }
    for (int c = 0; c < 2; ++c) {
      mbar_init(s_full + c, 1);
      mbar_init(s_empty + c, kMath64);
    }
    for (int h = 0; h < 2; ++h) {
      mbar_init(p_full + h, kMath64 / 2);
      mbar_init(p_empty + h, 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, kMath64);
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
        // K, V of this item go to buffer W & 1 while the previous item still reads the other
        const uint32_t kb2 = W & 1, kn = (W >> 1) & 1;
        if (!(ok = WAIT(kv_empty + kb2, kn ^ 1))) break;
        mbar_arrive_expect_tx(kv_full + kb2, 2 * g.R * 128);
        kv_arm |= 1u << kb2;
        kv_par = (kv_par & ~(1u << kb2)) | (kn << kb2);
        uint8_t* skv = smem + C::kK + kb2 * 2 * kBox;
        tma_load_5d(skv, &tk, kv_full + kb2, 0, tbk.tb.lo[2] + o[2], tbk.tb.lo[1] + o[1], tbk.tb.lo[0] + o[0], bh);
        tma_load_5d(skv + kBox, &tv, kv_full + kb2, 0, tbk.tb.lo[2] + o[2], tbk.tb.lo[1] + o[1], tbk.tb.lo[0] + o[0],
                    bh);
        const int64_t slot0 = tile_slot0(g, bh, tile);
        int jt = 0, jy = 0, jx = 0;
        for (int i = 0; i < tbk.NB; ++i, ++G) {
          const uint32_t st = G % C::kStages, n = G / C::kStages;
          const int c1 = tbk.tb.lo[2] + (jx * g.bx), c2 = tbk.tb.lo[1] + (jy * g.by), c3 = tbk.tb.lo[0] + (jt * g.bt);
          if (++jx == tbk.nb[2]) {
            jx = 0;
            if (++jy == tbk.nb[1]) {
              jy = 0;
              ++jt;
            }
          }
          if (!(ok = WAIT(qd_empty + st, (n & 1) ^ 1))) break;
          mbar_arrive_expect_tx(qd_full + st, 2 * g.R * 128 + 2048);
          qd_arm |= 1u << st;
          qd_par = (qd_par & ~(1u << st)) | ((n & 1) << st);
          uint8_t* sq = smem + C::kQ + st * 2 * kBox;
          tma_load_5d(sq, &tq, qd_full + st, 0, c1, c2, c3, bh);
          tma_load_5d(sq + kBox, &tdo, qd_full + st, 0, c1, c2, c3, bh);
          bulk_load(smem + C::kExt + st * 4096, a.ext + slot0 + i * 128, 2048, qd_full + st);
        }
        ++W;
      }
      if (!ok) {
        for (int b = 0; b < 2; ++b)
          if (kv_arm & (1u << b)) mbar_wait<set_status_bwd64>(kv_full + b, (kv_par >> b) & 1, abort_flag, false);
        for (int s = 0; s < C::kStages; ++s)
          if (qd_arm & (1u << s)) mbar_wait<set_status_bwd64>(qd_full + s, (qd_par >> s) & 1, abort_flag, false);
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ issuer of S'^T, dP'^T
    if (lane == 0) {
      constexpr uint32_t idS = idesc_bf16(128, 128, 0);
      const uint64_t dK0 = sw128_desc(smem_u32(smem + C::kK), 16, 1024);
      const uint64_t dQ0 = sw128_desc(smem_u32(smem + C::kQ), 16, 1024);
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
        const uint32_t kb2 = W & 1;
        if (!(ok = WAIT(kv_full + kb2, (W >> 1) & 1))) break;
        const uint64_t dK = dmove(dK0, kb2 * 2 * kBox), dV = dmove(dK, kBox);
        for (int i = 0; i < tbk.NB; ++i, ++G) {
          const uint32_t st = G % C::kStages;
          if (!(ok = WAIT(qd_full + st, (G / C::kStages) & 1))) break;
          if (G > 0 && !(ok = WAIT(s_empty, (G - 1) & 1))) break;  // S'^T of box G-1 read
          tc_fence_after();
          const uint64_t dq = dmove(dQ0, st * 2 * kBox), ddo = dmove(dq, kBox), de = dmove(dExt0, st * 4096);
#pragma unroll
          for (int ks = 0; ks < kD / 16; ++ks)
            umma_bf16(tmem + C::kColST, dmove(dK, ks * 32), dmove(dq, ks * 32), idS, ks > 0);
          umma_bf16(tmem + C::kColST, dOnesS, de, idS, 1u);
          umma_commit(s_full);
          if (G > 0 && !(ok = WAIT(s_empty + 1, (G - 1) & 1))) break;  // dP'^T of box G-1 read
          tc_fence_after();
#pragma unroll
          for (int ks = 0; ks < kD / 16; ++ks)
            umma_bf16(tmem + C::kColDP, dmove(dV, ks * 32), dmove(ddo, ks * 32), idS, ks > 0);
          umma_bf16(tmem + C::kColDP, dOnesD, de, idS, 1u);
          umma_commit(s_full + 1);
          if (i == tbk.NB - 1) umma_commit(kv_empty + kb2);  // K, V of this item no longer read
        }
        ++W;
      }
      umma_commit(drain);
      mbar_wait<set_status_bwd64>(drain, 0, abort_flag, false);
    }
  } else if (warp == kIssuerA) {
    // ------------------------------------------------------------ issuer of dV += P'^T dO, dK += dS^T Q
    if (lane == 0) {
      constexpr uint32_t idA = idesc_bf16(128, kD, 1);
      const uint64_t dQ0 = sw128_desc(smem_u32(smem + C::kQ), 16384, 1024);  // MN-major (K = queries)
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
          // p_full(G) implies s_full(G): the score products of this stage are
          // complete, so the qd_empty commit below covers every reader
          const uint64_t bq = dmove(dQ0, st * 2 * kBox), bdo = dmove(bq, kBox);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            if (!(ok = WAIT(p_full + h, G & 1))) break;
            if (i == 0 && h == 0 && !(ok = WAIT(acc_empty, (W & 1) ^ 1))) break;
            tc_fence_after();
#pragma unroll
            for (int k4 = 0; k4 < 4; ++k4) {
              const int ks = 4 * h + k4;
              const uint32_t acc = (i > 0 || ks > 0) ? 1u : 0u;
              umma_bf16_ts(tmem + C::kColDV, tmem + C::kColP + ks * 8, dmove(bdo, ks * 2048), idA, acc);
              umma_bf16_ts(tmem + C::kColDK, tmem + C::kColDS + ks * 8, dmove(bq, ks * 2048), idA, acc);
            }
            umma_commit(p_empty + h);
          }
          if (!ok) break;
          umma_commit(qd_empty + st);
        }
        if (!ok) break;
        umma_commit(acc_full);
        ++W;
      }
      umma_commit(drain + 1);
      mbar_wait<set_status_bwd64>(drain + 1, 0, abort_flag, false);
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
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(s_empty);  // the next box's S'^T may overwrite this one
        kv_p(sv, s2, pk);  // sv <- P'^T (FP32), pk <- P'^T (BF16 pairs)
        // this half's gradient products of box G-1 are done with the packed operand
        if (G > 0 && !(ok = WAIT(p_empty + (c4 >> 1), (G - 1) & 1))) break;
        tc_fence_after();
        tmem_st16(tl + C::kColP + c4 * 16, pk);
        if (!(ok = WAIT(s_full + 1, G & 1))) break;
        tc_fence_after();
        tmem_ld32(tl + C::kColDP + c4 * 32, dv);
        tmem_wait_ld(dv);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(s_empty + 1);  // the next box's dP'^T may overwrite this one
        kv_ds(sv, dv, pk);  // dS^T = P'^T dP'^T (BF16 pairs)
        tmem_st16(tl + C::kColDS + c4 * 16, pk);
        tmem_wait_st();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(p_full + (c4 >> 1));
      }
      if (!ok) break;
      // ---- epilogue: this thread's key row of dK, dV (columns [16 c4, 16 c4 + 16))
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
      const int c0 = c4 * 16;
      // both accumulators into registers, then they are released at once: the
      // next item's first gradient products may overwrite them during the stores
      uint32_t rk[16], rv[16];
      tmem_ld16(tl + C::kColDK + c0, rk);
      tmem_ld16(tl + C::kColDV + c0, rv);
      tmem_wait_ld(rk);
      tmem_wait_ld(rv);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acc_empty);
      row_store<16, OutT>(rk, g.scale, kvalid, single, static_cast<OutT*>(a.dk) + ((int64_t)bh * g.N + tok) * kD + c0,
                        a.dk_s + slot * kD + c0);
      row_store<16, OutT>(rv, 1.f, kvalid, single, static_cast<OutT*>(a.dv) + ((int64_t)bh * g.N + tok) * kD + c0,
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
struct Q64 {
  static constexpr int kStages = 4;  // (K, V) ring
  static constexpr int kQ = 0;
  static constexpr int kDO = kBox;
  static constexpr int kK = 2 * kBox;  // stage s: K at kK + s*2*kBox, V after it
  // Key-mask extension operands (as in the forward): A = 1 in K-column 0 of
  // 128 rows, and per stage the key block's bias row (0, or -1e30 for a
  // padding key or a key outside the tile), each followed by 2 KB of zeros.
  static constexpr int kOnes = kK + kStages * 2 * kBox;
  static constexpr int kBias = kOnes + 4096;
  static constexpr int kBar = kBias + kStages * 4096;
  // qd_full, qd_empty, qt_full, kv_full[S], kv_empty[S], s_full[2], s_empty[2], p_full[2], p_empty[2],
  // acc_full, acc_empty, drain[3]   (s_*[0]: the S chain, s_*[1]: the dP chain)
  static constexpr int kNumBars = 3 + 2 * kStages + 13;
  static constexpr int kMisc = kBar + kNumBars * 8;
  static constexpr int kSmem = kMisc + 16 + 1024;
  // TMEM: S 0, dP 128, dS buffer 0 (packed) 256, dQ 320, Q (packed) 384, dOut (packed) 416, dS buffer 1 448
  static constexpr uint32_t kColS = 0, kColDP = 128, kColDQ = 320, kColQ = 384, kColDO = 416;
  __device__ static uint32_t col_ds(uint32_t b) { return b ? 448u : 256u; }
};

template <typename OutT>
__global__ void __launch_bounds__(kThreadsQ64, 1)
    dq64_kernel(const __grid_constant__ CUtensorMap tq, const __grid_constant__ CUtensorMap tk,
                const __grid_constant__ CUtensorMap tv, const __grid_constant__ CUtensorMap tdo, const BwdArgs a) {
  using C = Q64;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::kBar);
  uint64_t* qd_full = bars;
  uint64_t* qd_empty = bars + 1;
  uint64_t* qt_full = bars + 2;
  uint64_t* kv_full = bars + 3;
  uint64_t* kv_empty = kv_full + C::kStages;
  uint64_t* s_full = kv_empty + C::kStages;
  uint64_t* s_empty = s_full + 2;
  uint64_t* p_full = s_empty + 2;   // [2]: one per dS buffer
  uint64_t* p_empty = p_full + 2;   // [2]
  uint64_t* acc_full = p_empty + 2;
  uint64_t* acc_empty = acc_full + 1;
  uint64_t* drain = acc_empty + 1;  // [3]: one per issuing thread
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + C::kMisc);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + C::kMisc + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  zero_pad_rows(smem, 2 + 2 * C::kStages, a.g.R);  // Q, dOut and the K / V ring
  for (int r = threadIdx.x; r < (1 + C::kStages) * 256; r += kThreadsQ64) {
    const int blk = r >> 8, rr = r & 255;
    const uint4 v = (blk == 0 && rr < 128) ? make_uint4(0x00003F80u, 0u, 0u, 0u) : make_uint4(0u, 0u, 0u, 0u);
    if (blk == 0 || rr >= 128) *reinterpret_cast<uint4*>(smem + C::kOnes + blk * 4096 + rr * 16) = v;
  }
  fence_proxy_async_smem();
  if (threadIdx.x == 0) {
    mbar_init(qd_full, 1);
    mbar_init(qd_empty, kMath64);
    mbar_init(qt_full, kMath64);
    for (int s = 0; s < C::kStages; ++s) {
      mbar_init(kv_full + s, 1);
      mbar_init(kv_empty + s, 1);
    }
    for (int c = 0; c < 2; ++c) {
      mbar_init(s_full + c, 1);
      mbar_init(s_empty + c, kMath64);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(p_full + b, kMath64);
      mbar_init(p_empty + b, 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, kMath64);
    mbar_init(drain, 1);
    mbar_init(drain + 1, 1);
    mbar_init(drain + 2, 1);
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
    // key-mask rows (all lanes, for key blocks with padding rows or keys outside the tile)
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
        if ((ok = WAIT(qd_empty, (W & 1) ^ 1))) {
          mbar_arrive_expect_tx(qd_full, 2 * g.R * 128);
          qd_arm = 1;
          qd_par = W & 1;
          tma_load_5d(smem + C::kQ, &tq, qd_full, 0, tbk.tb.lo[2] + o[2], tbk.tb.lo[1] + o[1], tbk.tb.lo[0] + o[0],
                      bh);
          tma_load_5d(smem + C::kDO, &tdo, qd_full, 0, tbk.tb.lo[2] + o[2], tbk.tb.lo[1] + o[1],
                      tbk.tb.lo[0] + o[0], bh);
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
          mbar_arrive_expect_tx(kv_full + st, 2 * g.R * 128);
          kv_arm |= 1u << st;
          kv_par = (kv_par & ~(1u << st)) | ((n & 1) << st);
          uint8_t* sk = smem + C::kK + st * 2 * kBox;
          tma_load_5d(sk, &tk, kv_full + st, 0, tbk.tb.lo[2] + ko[2], tbk.tb.lo[1] + ko[1], tbk.tb.lo[0] + ko[0], bh);
          tma_load_5d(sk + kBox, &tv, kv_full + st, 0, tbk.tb.lo[2] + ko[2], tbk.tb.lo[1] + ko[1],
                      tbk.tb.lo[0] + ko[0], bh);
        }
      }
      ++W;
    }
    if (!ok && lane == 0) {
      if (qd_arm) mbar_wait<set_status_bwd64>(qd_full, qd_par, abort_flag, false);
      for (int s = 0; s < C::kStages; ++s)
        if (kv_arm & (1u << s)) mbar_wait<set_status_bwd64>(kv_full + s, (kv_par >> s) & 1, abort_flag, false);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ issuer of S
    if (lane == 0) {
      constexpr uint32_t idS = idesc_bf16(128, 128, 0);
      const uint64_t dK0 = sw128_desc(smem_u32(smem + C::kK), 16, 1024);
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
          // a masked block's bias row was filled by the producer warp
          const bool masked = !all_full && !bw.full(g, tbk);
          if (!(ok = WAIT(kv_full + st, (G / C::kStages) & 1))) break;
          if (G > 0 && !(ok = WAIT(s_empty, (G - 1) & 1))) break;  // S of box G-1 read
          tc_fence_after();
          const uint64_t dk = dmove(dK0, st * 2 * kBox);
#pragma unroll
          for (int ks = 0; ks < kD / 16; ++ks)
            umma_bf16_ts(tmem + C::kColS, tmem + C::kColQ + ks * 8, dmove(dk, ks * 32), idS, ks > 0);
          // masked keys get -1e30, so P' = 0 there and dS = 0 follows
          if (masked) umma_bf16(tmem + C::kColS, dOnes, dmove(dBias0, st * 4096), idS, 1u);
          umma_commit(s_full);
        }
        ++W;
      }
      umma_commit(drain);
      mbar_wait<set_status_bwd64>(drain, 0, abort_flag, false);
    }
  } else if (warp == kIssuerD) {
    // ------------------------------------------------------------ issuer of dP (its own thread, as in
    // the dK/dV kernel)
    if (lane == 0) {
      constexpr uint32_t idS = idesc_bf16(128, 128, 0);
      const uint64_t dK0 = sw128_desc(smem_u32(smem + C::kK), 16, 1024);
      uint32_t G = 0, W = 0;
      bool ok = true;
      for (int w = blockIdx.x; w < a.items && ok; w += gridDim.x) {
        int bh, tile, qb;
        decode_item(g, w, bh, tile, qb);
        TileBlocks tbk;
        tile_blocks(g, tile, tbk);
        if (qb >= tbk.NB) continue;
        if (!(ok = WAIT(qt_full, W & 1))) break;  // Q, dOut in TMEM
        for (int j = 0; j < tbk.NB; ++j, ++G) {
          const uint32_t st = G % C::kStages;
          if (!(ok = WAIT(kv_full + st, (G / C::kStages) & 1))) break;
          if (G > 0 && !(ok = WAIT(s_empty + 1, (G - 1) & 1))) break;  // dP of box G-1 read
          tc_fence_after();
          const uint64_t dv = dmove(dK0, st * 2 * kBox + kBox);
#pragma unroll
          for (int ks = 0; ks < kD / 16; ++ks)
            umma_bf16_ts(tmem + C::kColDP, tmem + C::kColDO + ks * 8, dmove(dv, ks * 32), idS, ks > 0);
          umma_commit(s_full + 1);
        }
        ++W;
      }
      umma_commit(drain + 2);
      mbar_wait<set_status_bwd64>(drain + 2, 0, abort_flag, false);
    }
  } else if (warp == kIssuerA) {
    // ------------------------------------------------------------ issuer of dQ += dS K
    if (lane == 0) {
      constexpr uint32_t idA = idesc_bf16(128, kD, 1);
      const uint64_t bK0 = sw128_desc(smem_u32(smem + C::kK), 16384, 1024);  // MN-major (K = keys)
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
          // p_full(G) implies s_full(G): the score products of this stage are
          // complete, so the kv_empty commit below covers every reader.  dS is
          // double-buffered: box G uses buffer G & 1.
          const uint32_t b = G & 1;
          if (!(ok = WAIT(p_full + b, (G >> 1) & 1))) break;
          if (j == 0 && !(ok = WAIT(acc_empty, (W & 1) ^ 1))) break;
          tc_fence_after();
          const uint64_t bk = dmove(bK0, st * 2 * kBox);
#pragma unroll
          for (int ks = 0; ks < 8; ++ks)
            umma_bf16_ts(tmem + C::kColDQ, tmem + C::col_ds(b) + ks * 8, dmove(bk, ks * 2048), idA,
                         (j > 0 || ks > 0) ? 1u : 0u);
          umma_commit(p_empty + b);
          umma_commit(kv_empty + st);
        }
        if (!ok) break;
        umma_commit(acc_full);
        ++W;
      }
      umma_commit(drain + 1);
      mbar_wait<set_status_bwd64>(drain + 1, 0, abort_flag, false);
    }
  } else {
    // ------------------------------------------------------------ elementwise + epilogue (row = query)
    const int quad = warp & 3;
    const int c4 = (warp - kMath0) >> 2;  // key columns [32 c4, 32 c4 + 32)
    const int row = quad * 32 + lane;
    const uint32_t tl = tmem + ((uint32_t)(quad * 32) << 16);
    const float sl2 = g.scale_log2;
    uint32_t G = 0, W = 0;
    bool ok = true;
    for (int w = blockIdx.x; w < a.items && ok; w += gridDim.x) {
      int bh, tile, qb;
      decode_item(g, w, bh, tile, qb);
      TileBlocks tbk;
      tile_blocks(g, tile, tbk);
      if (qb >= tbk.NB) continue;
      const int64_t qslot = tile_slot0(g, bh, tile) + qb * 128 + row;
      const float nL = a.lse2c[qslot];  // -lse' (-inf for padding rows)
      const float nD = a.dd[qslot];     // -D
      // Q and dOut of the query box: shared memory -> TMEM (A operands of S, dP),
      // elements [16 c4, 16 c4 + 16) of the row.  The previous item's products
      // are complete (its acc_full was waited on).
      if (!(ok = WAIT(qd_full, W & 1))) break;
      {
        uint32_t r8[8];
        ld_swizzled_row<2>(smem_u32(smem + C::kQ), row, 2 * c4, r8);
        tmem_st8(tl + C::kColQ + 8 * c4, r8);
        ld_swizzled_row<2>(smem_u32(smem + C::kDO), row, 2 * c4, r8);
        tmem_st8(tl + C::kColDO + 8 * c4, r8);
        tmem_wait_st();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(qd_empty);
          mbar_arrive(qt_full);
        }
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
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(s_empty + 1);  // the next box's dP may overwrite this one
        q_ds(sv, dv, nD, pk);
        // dS buffer G & 1 is free once the dQ products of box G-2 are done
        const uint32_t b = G & 1;
        if (G > 1 && !(ok = WAIT(p_empty + b, ((G >> 1) - 1) & 1))) break;
        tc_fence_after();
        tmem_st16(tl + C::col_ds(b) + c4 * 16, pk);
        tmem_wait_st();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(p_full + b);
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
      const int c0 = c4 * 16;
      uint32_t rq[16];
      tmem_ld16(tl + C::kColDQ + c0, rq);
      tmem_wait_ld(rq);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acc_empty);  // released before the stores
      row_store<16, OutT>(rq, g.scale, qvalid, single, static_cast<OutT*>(a.dq) + ((int64_t)bh * g.N + tok) * kD + c0,
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
cudaError_t run_bwd64(const Geom& g, const __nv_bfloat16* q, const __nv_bfloat16* k, const __nv_bfloat16* v,
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
  auto k1 = dkdv64_kernel<OutT>;
  cudaError_t e = cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, Kv64::kSmem);
  if (e != cudaSuccess) return e;
  prof_begin(kKBwdDkdv, st);
  k1<<<grid, kThreads64, Kv64::kSmem, st>>>(mq, mk, mv, mdo, a);
  prof_end(kKBwdDkdv, st);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  auto k2 = dq64_kernel<OutT>;
  e = cudaFuncSetAttribute(k2, cudaFuncAttributeMaxDynamicSharedMemorySize, Q64::kSmem);
  if (e != cudaSuccess) return e;
  prof_begin(kKBwdDq, st);
  k2<<<grid, kThreadsQ64, Q64::kSmem, st>>>(mq, mk, mv, mdo, a);
  prof_end(kKBwdDq, st);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sm103_bwd64(const Geom& g, const __nv_bfloat16* q, const __nv_bfloat16* k, const __nv_bfloat16* v,
                               const __nv_bfloat16* dout, const float* lse2c, const float* dd, const void* ext,
                               void* dq, void* dk, void* dv, int out_dtype, float* dq_s, float* dk_s, float* dv_s,
                               cudaStream_t st) {
  if (g.d != kD) return cudaErrorNotSupported;
  if (out_dtype == GATTN_BF16)
    return run_bwd64<__nv_bfloat16>(g, q, k, v, dout, lse2c, dd, ext, dq, dk, dv, dq_s, dk_s, dv_s, st);
  return run_bwd64<float>(g, q, k, v, dout, lse2c, dd, ext, dq, dk, dv, dq_s, dk_s, dv_s, st);
}

}  // namespace gattn
