// sm103_bwd.cu -- BF16 tensor-core backward of STORM-GPA tile attention on
// GB300 (sm_103a), general head size (d = 128; d = 64 runs the TMEM-operand
// kernels of sm103_bwd64.cu).  Two deterministic kernels (no atomics):
//
//   dKdV kernel, one work item per (batch*head, tile, 128-key block kb):
//     for every 64-query half-block i of the tile:
//       S^T  = K_kb Q_i^T            tcgen05 -> TMEM (double-buffered)
//       dP^T = V_kb dOut_i^T         tcgen05 -> TMEM (double-buffered)
//       P'^T = exp2(s S^T log2e - lse'_i)        (softmax warps, BF16 -> smem)
//       dS^T = P'^T (dP^T - D_i)                 (softmax warps, BF16 -> smem)
//       dV  += P'^T dOut_i,  dK += dS^T Q_i      tcgen05, FP32 accumulators in TMEM
//   dQ kernel, one work item per (batch*head, tile, 128-query block qb):
//     for every 64-key half-block j:  S = Q K_j^T, dP = dOut V_j^T,
//       dS = P' (dP - D) (keys outside the tile masked), dQ += dS K_j.
//
// The merge weight of the Hann-weighted overlap average (arXiv 2604.16590,
// Sec. III-C) enters through the per-row statistics the prep pass writes
// (negated, -lse' and -D, so each element costs one packed FMA for the exp2
// argument and one packed add + multiply for dS): lse' = lse - log2(w_t/sum w)
// makes P' = (w_t / sum w) P, the probabilities of the per-tile gradient
// dO_t = (w_t / sum w) dOut, and D = dOut . O_t.  P is recomputed from lse' (never stored).  Rows covered by
// one tile are written straight to dQ/dK/dV; multiply-covered rows go to FP32
// per-tile slots that the merge kernel sums in fixed tile order.
//
// Warp roles: warp 0 TMA producer, warp 1 TMEM allocator + single-thread MMA
// issuer, warps 2..9 elementwise math + epilogue: one TMEM lane = one block row,
// two warps per lane quadrant, each taking half of the row's columns (eight
// math warps keep two warps per SM sub-partition to hide TMEM and MUFU latency).
#include "sm103_bwd_common.cuh"

GATTN_DEFINE_STATUS(sm103_bwd)

namespace gattn {
namespace {
using namespace sm103;

__device__ void set_status_bwd(uint32_t c) { set_status(c); }
#define WAIT(bar, par) mbar_wait<set_status_bwd>((bar), (par), abort_flag)

// =============================================================== dK / dV
template <int D>
struct KvCfg {
  static constexpr int kHalves = D / 64;
  static constexpr int kBlock = 128 * D * 2;
  static constexpr int kStages = D == 64 ? 2 : 1;  // (Q, dOut, lse', D) ring
  static constexpr int kK = 0;
  static constexpr int kV = kBlock;
  static constexpr int kQ = 2 * kBlock;             // stage s: Q at kQ + s*2*kBlock, dOut after it
  static constexpr int kStat = kQ + kStages * 2 * kBlock;  // stage s: 128 lse' + 128 D floats
  static constexpr int kP = kStat + kStages * 1024;        // 2 buffers x (P'^T 16 KB + dS^T 16 KB)
  static constexpr int kBar = kP + 2 * 32768;
  // kv_full, kv_empty, qd_full[S], qd_empty[S], st_full[2], st_empty[2], p_full[2], p_empty[2],
  // acc_full, acc_empty, drain
  static constexpr int kNumBars = 2 + 2 * kStages + 8 + 3;
  static constexpr int kMisc = kBar + kNumBars * 8;
  static constexpr int kSmem = kMisc + 16 + 1024;
  // TMEM columns: S^T[2] 0/64, dP^T[2] 128/192, dV 256, dK 256 + D
  static constexpr uint32_t kColST = 0, kColDP = 128, kColDV = 256, kColDK = 256 + D;
};

template <int D, typename OutT>
__global__ void __launch_bounds__(kThreads, 1)
    sm103_dkdv_kernel(const __grid_constant__ CUtensorMap tq, const __grid_constant__ CUtensorMap tk,
                      const __grid_constant__ CUtensorMap tv, const __grid_constant__ CUtensorMap tdo,
                      const BwdArgs a) {
  using C = KvCfg<D>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::kBar);
  uint64_t* kv_full = bars;
  uint64_t* kv_empty = bars + 1;
  uint64_t* qd_full = bars + 2;
  uint64_t* qd_empty = qd_full + C::kStages;
  uint64_t* st_full = qd_empty + C::kStages;
  uint64_t* st_empty = st_full + 2;
  uint64_t* p_full = st_empty + 2;
  uint64_t* p_empty = p_full + 2;
  uint64_t* acc_full = p_empty + 2;
  uint64_t* acc_empty = acc_full + 1;
  uint64_t* drain = acc_empty + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + C::kMisc);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + C::kMisc + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  zero_pad_rows(smem, (2 + 2 * C::kStages) * C::kHalves, a.g.R);  // K, V and the Q / dOut ring
  if (threadIdx.x == 0) {
    mbar_init(kv_full, 1);
    mbar_init(kv_empty, 1);
    for (int s = 0; s < C::kStages; ++s) {
      mbar_init(qd_full + s, 1);
      mbar_init(qd_empty + s, 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(st_full + s, 1);
      mbar_init(st_empty + s, kMathWarps);
      mbar_init(p_full + s, kMathWarps);
      mbar_init(p_empty + s, 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, kMathWarps);
    mbar_init(drain, 1);
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
        mbar_arrive_expect_tx(kv_full, 2 * C::kHalves * g.R * 128);
        kv_arm = 1;
        kv_par = W & 1;
        for (int h = 0; h < C::kHalves; ++h) {
          tma_load_5d(smem + C::kK + h * 16384, &tk, kv_full, 64 * h, tbk.tb.lo[2] + o[2], tbk.tb.lo[1] + o[1],
                      tbk.tb.lo[0] + o[0], bh);
          tma_load_5d(smem + C::kV + h * 16384, &tv, kv_full, 64 * h, tbk.tb.lo[2] + o[2], tbk.tb.lo[1] + o[1],
                      tbk.tb.lo[0] + o[0], bh);
        }
        const int64_t slot0 = tile_slot0(g, bh, tile);
        for (int i = 0; i < tbk.NB; ++i, ++G) {
          const uint32_t st = G % C::kStages, n = G / C::kStages;
          block_origin(g, tbk, i, o);
          if (!(ok = WAIT(qd_empty + st, (n & 1) ^ 1))) break;
          mbar_arrive_expect_tx(qd_full + st, 2 * C::kHalves * g.R * 128 + 1024);
          qd_arm |= 1u << st;
          qd_par = (qd_par & ~(1u << st)) | ((n & 1) << st);
          uint8_t* sq = smem + C::kQ + st * 2 * C::kBlock;
          for (int h = 0; h < C::kHalves; ++h) {
            tma_load_5d(sq + h * 16384, &tq, qd_full + st, 64 * h, tbk.tb.lo[2] + o[2], tbk.tb.lo[1] + o[1],
                        tbk.tb.lo[0] + o[0], bh);
            tma_load_5d(sq + C::kBlock + h * 16384, &tdo, qd_full + st, 64 * h, tbk.tb.lo[2] + o[2],
                        tbk.tb.lo[1] + o[1], tbk.tb.lo[0] + o[0], bh);
          }
          bulk_load(smem + C::kStat + st * 1024, a.lse2c + slot0 + i * 128, 512, qd_full + st);
          bulk_load(smem + C::kStat + st * 1024 + 512, a.dd + slot0 + i * 128, 512, qd_full + st);
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
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      constexpr uint32_t idS = idesc_bf16(128, 64, 0);
      constexpr uint32_t idA = idesc_bf16(128, D, 1);
      const uint32_t sK = smem_u32(smem + C::kK), sV = smem_u32(smem + C::kV), sQ = smem_u32(smem + C::kQ),
                     sP = smem_u32(smem + C::kP);
      uint32_t G = 0, H = 0, W = 0;
      bool ok = true;
      for (int w = blockIdx.x; w < a.items && ok; w += gridDim.x) {
        int bh, tile, kb;
        decode_item(g, w, bh, tile, kb);
        TileBlocks tbk;
        tile_blocks(g, tile, tbk);
        if (kb >= tbk.NB) continue;
        if (!(ok = WAIT(kv_full, W & 1))) break;
        tc_fence_after();
        const uint32_t G0 = G, H0 = H;
        // dV/dK accumulation of half-block h (this item's halves start at H0)
        auto issue_acc = [&](uint32_t h) -> bool {
          const uint32_t b = h & 1;
          const uint32_t gbox = G0 + ((h - H0) >> 1), half = (h - H0) & 1, st = gbox % C::kStages;
          if (!WAIT(p_full + b, (h >> 1) & 1)) return false;
          if (h == H0 && !WAIT(acc_empty, (W & 1) ^ 1)) return false;
          tc_fence_after();
          const uint32_t sq = sQ + st * 2 * C::kBlock + half * 8192;
          const uint32_t sdo = sq + C::kBlock;
          const uint32_t pb = sP + b * 32768, dsb = pb + 16384;
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {
            const uint32_t acc = (h != H0 || ks > 0) ? 1u : 0u;
            umma_bf16(tmem + C::kColDV, sw128_desc(pb + ks * 32, 16, 1024), sw128_desc(sdo + ks * 2048, 16384, 1024),
                      idA, acc);
            umma_bf16(tmem + C::kColDK, sw128_desc(dsb + ks * 32, 16, 1024), sw128_desc(sq + ks * 2048, 16384, 1024),
                      idA, acc);
          }
          umma_commit(p_empty + b);
          if (half == 1) umma_commit(qd_empty + st);
          return true;
        };
        // The dV/dK product of half h is issued after the S^T/dP^T products of
        // half h+1 (so the tensor pipe has work while the softmax warps finish h).
        // With a single (Q, dOut) stage the next box's load waits for the last
        // half of the previous box to be consumed, so that half is flushed first.
        bool pending = false;
        for (int i = 0; i < tbk.NB && ok; ++i, ++G) {
          const uint32_t st = G % C::kStages;
          if (C::kStages == 1 && pending) {
            if (!(ok = issue_acc(H - 1))) break;
            pending = false;
          }
          if (!(ok = WAIT(qd_full + st, (G / C::kStages) & 1))) break;
          for (int half = 0; half < 2; ++half, ++H) {
            const uint32_t b = H & 1;
            if (!(ok = WAIT(st_empty + b, ((H >> 1) & 1) ^ 1))) break;
            tc_fence_after();
            const uint32_t sq = sQ + st * 2 * C::kBlock + half * 8192;
            const uint32_t sdo = sQ + st * 2 * C::kBlock + C::kBlock + half * 8192;
#pragma unroll
            for (int ks = 0; ks < D / 16; ++ks) {
              umma_bf16(tmem + C::kColST + b * 64, sw128_desc(sK + kmaj_off(ks), 16, 1024),
                        sw128_desc(sq + kmaj_off(ks), 16, 1024), idS, ks > 0);
              umma_bf16(tmem + C::kColDP + b * 64, sw128_desc(sV + kmaj_off(ks), 16, 1024),
                        sw128_desc(sdo + kmaj_off(ks), 16, 1024), idS, ks > 0);
            }
            umma_commit(st_full + b);
            if (i == tbk.NB - 1 && half == 1) umma_commit(kv_empty);
            if (pending && !(ok = issue_acc(H - 1))) break;
            pending = true;
          }
        }
        if (!ok) break;
        if (pending && !(ok = issue_acc(H - 1))) break;
        umma_commit(acc_full);
        ++W;
      }
      umma_commit(drain);
      mbar_wait<set_status_bwd>(drain, 0, abort_flag, false);
    }
  } else {
    // ------------------------------------------------------------ elementwise + epilogue (row = key)
    const int quad = warp & 3;
    const int ch = (warp - 2) >> 2;  // which 32 of the 64 query columns of a half block
    const int row = quad * 32 + lane;
    const uint32_t tl = tmem + ((uint32_t)(quad * 32) << 16);
    const uint32_t sP = smem_u32(smem + C::kP);
    const float sl2 = g.scale_log2;
    uint32_t G = 0, H = 0, W = 0;
    bool ok = true;
    for (int w = blockIdx.x; w < a.items && ok; w += gridDim.x) {
      int bh, tile, kb;
      decode_item(g, w, bh, tile, kb);
      TileBlocks tbk;
      tile_blocks(g, tile, tbk);
      if (kb >= tbk.NB) continue;
      for (int i = 0; i < tbk.NB && ok; ++i, ++G) {
        const uint32_t st = G % C::kStages;
        if (!(ok = WAIT(qd_full + st, (G / C::kStages) & 1))) break;
        const float* sL = reinterpret_cast<const float*>(smem + C::kStat + st * 1024);
        const float* sD = sL + 128;
        for (int half = 0; half < 2; ++half, ++H) {
          const uint32_t b = H & 1;
          if (!(ok = WAIT(st_full + b, (H >> 1) & 1))) break;
          tc_fence_after();
          uint32_t sv[32], dv[32];
          tmem_ld32(tl + C::kColST + b * 64 + ch * 32, sv);
          tmem_ld32(tl + C::kColDP + b * 64 + ch * 32, dv);
          tmem_wait_ld(sv);
          tmem_wait_ld(dv);
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(st_empty + b);
          // P' = exp2(s S^T log2e - lse'), dS^T = P' (dP^T - D); the stage holds -lse', -D
          uint32_t pp[16], pd[16];
          const float4* nL4 = reinterpret_cast<const float4*>(sL + half * 64 + ch * 32);
          const float4* nD4 = reinterpret_cast<const float4*>(sD + half * 64 + ch * 32);
          const uint64_t s2 = f2pack(sl2, sl2);
#pragma unroll
          for (int c4 = 0; c4 < 8; ++c4) {
            const float4 l = nL4[c4], dn = nD4[c4];
            const int c = 4 * c4;
            float a0, a1, a2, a3;
            f2unpack(ffma2(u2pack(sv[c], sv[c + 1]), s2, f2pack(l.x, l.y)), a0, a1);
            f2unpack(ffma2(u2pack(sv[c + 2], sv[c + 3]), s2, f2pack(l.z, l.w)), a2, a3);
            const float p0 = ex2(a0), p1 = ex2(a1), p2 = ex2(a2), p3 = ex2(a3);
            float e0, e1, e2, e3;
            f2unpack(fmul2(f2pack(p0, p1), fadd2(u2pack(dv[c], dv[c + 1]), f2pack(dn.x, dn.y))), e0, e1);
            f2unpack(fmul2(f2pack(p2, p3), fadd2(u2pack(dv[c + 2], dv[c + 3]), f2pack(dn.z, dn.w))), e2, e3);
            pp[2 * c4] = pack_bf16(p0, p1);
            pp[2 * c4 + 1] = pack_bf16(p2, p3);
            pd[2 * c4] = pack_bf16(e0, e1);
            pd[2 * c4 + 1] = pack_bf16(e2, e3);
          }
          if (!(ok = WAIT(p_empty + b, ((H >> 1) & 1) ^ 1))) break;
          store_row32(sP + b * 32768, row, ch, pp);
          store_row32(sP + b * 32768 + 16384, row, ch, pd);
          fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) mbar_arrive(p_full + b);
        }
      }
      if (!ok) break;
      // ---- epilogue: this thread's key row of dK, dV (its half of the columns)
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
      const int c0 = ch * (D / 2);
      tmem_row_epilogue<D / 2, OutT>(tl + C::kColDK + c0, g.scale, kvalid, single,
                                     static_cast<OutT*>(a.dk) + ((int64_t)bh * g.N + tok) * D + c0,
                                     a.dk_s + slot * D + c0);
      tmem_row_epilogue<D / 2, OutT>(tl + C::kColDV + c0, 1.f, kvalid, single,
                                     static_cast<OutT*>(a.dv) + ((int64_t)bh * g.N + tok) * D + c0,
                                     a.dv_s + slot * D + c0);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acc_empty);
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
template <int D>
struct QCfg {
  static constexpr int kHalves = D / 64;
  static constexpr int kBlock = 128 * D * 2;
  static constexpr int kStages = D == 64 ? 3 : 2;  // (K, V) ring
  static constexpr int kQ = 0;
  static constexpr int kDO = kBlock;
  static constexpr int kK = 2 * kBlock;            // stage s: K at kK + s*2*kBlock, V after it
  static constexpr int kDS = kK + kStages * 2 * kBlock;  // 2 buffers x 16 KB (dS, 128 queries x 64 keys)
  static constexpr int kBar = kDS + 2 * 16384;
  // qd_full, qd_empty, kv_full[S], kv_empty[S], s_full[2], s_empty[2], ds_full[2], ds_empty[2],
  // acc_full, acc_empty, drain
  static constexpr int kNumBars = 2 + 2 * kStages + 8 + 3;
  static constexpr int kMisc = kBar + kNumBars * 8;
  static constexpr int kSmem = kMisc + 16 + 1024;
  // TMEM columns: S[2] 0/64, dP[2] 128/192, dQ 256
  static constexpr uint32_t kColS = 0, kColDP = 128, kColDQ = 256;
};

// dS = P' (dP - D) for 32 key columns of this thread's query row, packed to
// BF16; nL = -lse', nD = -D of the row; keys outside the tile masked to 0.

template <int D, typename OutT>
__global__ void __launch_bounds__(kThreads, 1)
    sm103_dq_kernel(const __grid_constant__ CUtensorMap tq, const __grid_constant__ CUtensorMap tk,
                    const __grid_constant__ CUtensorMap tv, const __grid_constant__ CUtensorMap tdo,
                    const BwdArgs a) {
  using C = QCfg<D>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::kBar);
  uint64_t* qd_full = bars;
  uint64_t* qd_empty = bars + 1;
  uint64_t* kv_full = bars + 2;
  uint64_t* kv_empty = kv_full + C::kStages;
  uint64_t* s_full = kv_empty + C::kStages;
  uint64_t* s_empty = s_full + 2;
  uint64_t* ds_full = s_empty + 2;
  uint64_t* ds_empty = ds_full + 2;
  uint64_t* acc_full = ds_empty + 2;
  uint64_t* acc_empty = acc_full + 1;
  uint64_t* drain = acc_empty + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + C::kMisc);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + C::kMisc + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  zero_pad_rows(smem, (2 + 2 * C::kStages) * C::kHalves, a.g.R);  // Q, dOut and the K / V ring
  if (threadIdx.x == 0) {
    mbar_init(qd_full, 1);
    mbar_init(qd_empty, 1);
    for (int s = 0; s < C::kStages; ++s) {
      mbar_init(kv_full + s, 1);
      mbar_init(kv_empty + s, 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(s_full + s, 1);
      mbar_init(s_empty + s, kMathWarps);
      mbar_init(ds_full + s, kMathWarps);
      mbar_init(ds_empty + s, 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, kMathWarps);
    mbar_init(drain, 1);
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
    if (lane == 0) {
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
        if (!(ok = WAIT(qd_empty, (W & 1) ^ 1))) break;
        mbar_arrive_expect_tx(qd_full, 2 * C::kHalves * g.R * 128);
        qd_arm = 1;
        qd_par = W & 1;
        for (int h = 0; h < C::kHalves; ++h) {
          tma_load_5d(smem + C::kQ + h * 16384, &tq, qd_full, 64 * h, tbk.tb.lo[2] + o[2], tbk.tb.lo[1] + o[1],
                      tbk.tb.lo[0] + o[0], bh);
          tma_load_5d(smem + C::kDO + h * 16384, &tdo, qd_full, 64 * h, tbk.tb.lo[2] + o[2], tbk.tb.lo[1] + o[1],
                      tbk.tb.lo[0] + o[0], bh);
        }
        for (int j = 0; j < tbk.NB; ++j, ++G) {
          const uint32_t st = G % C::kStages, n = G / C::kStages;
          block_origin(g, tbk, j, o);
          if (!(ok = WAIT(kv_empty + st, (n & 1) ^ 1))) break;
          mbar_arrive_expect_tx(kv_full + st, 2 * C::kHalves * g.R * 128);
          kv_arm |= 1u << st;
          kv_par = (kv_par & ~(1u << st)) | ((n & 1) << st);
          uint8_t* sk = smem + C::kK + st * 2 * C::kBlock;
          for (int h = 0; h < C::kHalves; ++h) {
            tma_load_5d(sk + h * 16384, &tk, kv_full + st, 64 * h, tbk.tb.lo[2] + o[2], tbk.tb.lo[1] + o[1],
                        tbk.tb.lo[0] + o[0], bh);
            tma_load_5d(sk + C::kBlock + h * 16384, &tv, kv_full + st, 64 * h, tbk.tb.lo[2] + o[2],
                        tbk.tb.lo[1] + o[1], tbk.tb.lo[0] + o[0], bh);
          }
        }
        ++W;
      }
      if (!ok) {
        if (qd_arm) mbar_wait<set_status_bwd>(qd_full, qd_par, abort_flag, false);
        for (int s = 0; s < C::kStages; ++s)
          if (kv_arm & (1u << s)) mbar_wait<set_status_bwd>(kv_full + s, (kv_par >> s) & 1, abort_flag, false);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idS = idesc_bf16(128, 64, 0);
      constexpr uint32_t idA = idesc_bf16(128, D, 1);
      const uint32_t sQ = smem_u32(smem + C::kQ), sDO = smem_u32(smem + C::kDO), sK = smem_u32(smem + C::kK),
                     sDS = smem_u32(smem + C::kDS);
      uint32_t G = 0, H = 0, W = 0;
      bool ok = true;
      for (int w = blockIdx.x; w < a.items && ok; w += gridDim.x) {
        int bh, tile, qb;
        decode_item(g, w, bh, tile, qb);
        TileBlocks tbk;
        tile_blocks(g, tile, tbk);
        if (qb >= tbk.NB) continue;
        if (!(ok = WAIT(qd_full, W & 1))) break;
        tc_fence_after();
        const uint32_t G0 = G, H0 = H;
        auto issue_dq = [&](uint32_t h) -> bool {
          const uint32_t b = h & 1;
          const uint32_t gbox = G0 + ((h - H0) >> 1), half = (h - H0) & 1, st = gbox % C::kStages;
          if (!WAIT(ds_full + b, (h >> 1) & 1)) return false;
          if (h == H0 && !WAIT(acc_empty, (W & 1) ^ 1)) return false;
          tc_fence_after();
          const uint32_t sk = sK + st * 2 * C::kBlock + half * 8192;
#pragma unroll
          for (int ks = 0; ks < 4; ++ks)
            umma_bf16(tmem + C::kColDQ, sw128_desc(sDS + b * 16384 + ks * 32, 16, 1024),
                      sw128_desc(sk + ks * 2048, 16384, 1024), idA, (h != H0 || ks > 0) ? 1u : 0u);
          umma_commit(ds_empty + b);
          if (half == 1) umma_commit(kv_empty + st);
          return true;
        };
        for (int j = 0; j < tbk.NB && ok; ++j, ++G) {
          const uint32_t st = G % C::kStages;
          if (!(ok = WAIT(kv_full + st, (G / C::kStages) & 1))) break;
          for (int half = 0; half < 2; ++half, ++H) {
            const uint32_t b = H & 1;
            if (!(ok = WAIT(s_empty + b, ((H >> 1) & 1) ^ 1))) break;
            tc_fence_after();
            const uint32_t sk = sK + st * 2 * C::kBlock + half * 8192;
            const uint32_t sv = sk + C::kBlock;
#pragma unroll
            for (int ks = 0; ks < D / 16; ++ks) {
              umma_bf16(tmem + C::kColS + b * 64, sw128_desc(sQ + kmaj_off(ks), 16, 1024),
                        sw128_desc(sk + kmaj_off(ks), 16, 1024), idS, ks > 0);
              umma_bf16(tmem + C::kColDP + b * 64, sw128_desc(sDO + kmaj_off(ks), 16, 1024),
                        sw128_desc(sv + kmaj_off(ks), 16, 1024), idS, ks > 0);
            }
            umma_commit(s_full + b);
            if (j == tbk.NB - 1 && half == 1) umma_commit(qd_empty);
            if (H > H0 && !(ok = issue_dq(H - 1))) break;
          }
        }
        if (!ok) break;
        if (!(ok = issue_dq(H - 1))) break;
        umma_commit(acc_full);
        ++W;
      }
      umma_commit(drain);
      mbar_wait<set_status_bwd>(drain, 0, abort_flag, false);
    }
  } else {
    // ------------------------------------------------------------ elementwise + epilogue (row = query)
    const int quad = warp & 3;
    const int ch = (warp - 2) >> 2;  // which 32 of the 64 key columns of a half block
    const int row = quad * 32 + lane;
    const uint32_t tl = tmem + ((uint32_t)(quad * 32) << 16);
    const uint32_t sDS = smem_u32(smem + C::kDS);
    const float sl2 = g.scale_log2;
    uint32_t G = 0, H = 0, W = 0;
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
      for (int j = 0; j < tbk.NB && ok; ++j, ++G) {
        int ko[3];
        block_origin(g, tbk, j, ko);
        const bool full = block_full(g, tbk, ko);
        uint32_t kmask[2] = {~0u, ~0u};
        if (!full) {
#pragma unroll
          for (int h2 = 0; h2 < 2; ++h2) {
            int kl[3];
            block_row(g, ko, h2 * 64 + ch * 32 + lane, kl);
            kmask[h2] = __ballot_sync(0xffffffffu, inside(tbk, kl));
          }
        }
        for (int half = 0; half < 2; ++half, ++H) {
          const uint32_t b = H & 1;
          if (!(ok = WAIT(s_full + b, (H >> 1) & 1))) break;
          tc_fence_after();
          uint32_t sv[32], dv[32];
          tmem_ld32(tl + C::kColS + b * 64 + ch * 32, sv);
          tmem_ld32(tl + C::kColDP + b * 64 + ch * 32, dv);
          tmem_wait_ld(sv);
          tmem_wait_ld(dv);
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(s_empty + b);
          uint32_t pk[16];
          if (full)
            dq_half<false>(sv, dv, 0u, sl2, nL, nD, pk);
          else
            dq_half<true>(sv, dv, kmask[half], sl2, nL, nD, pk);
          if (!(ok = WAIT(ds_empty + b, ((H >> 1) & 1) ^ 1))) break;
          store_row32(sDS + b * 16384, row, ch, pk);
          fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) mbar_arrive(ds_full + b);
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
      const int c0 = ch * (D / 2);
      tmem_row_epilogue<D / 2, OutT>(tl + C::kColDQ + c0, g.scale, qvalid, single,
                                     static_cast<OutT*>(a.dq) + ((int64_t)bh * g.N + tok) * D + c0,
                                     a.dq_s + qslot * D + c0);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acc_empty);
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

template <int D, typename OutT>
cudaError_t run_bwd(const Geom& g, const __nv_bfloat16* q, const __nv_bfloat16* k, const __nv_bfloat16* v,
                    const __nv_bfloat16* dout, const float* lse2c, const float* dd, void* dq, void* dk, void* dv,
                    float* dq_s, float* dk_s, float* dv_s, cudaStream_t st) {
  BwdArgs a;
  a.g = g;
  a.lse2c = lse2c;
  a.dd = dd;
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
  if (!make_tmap_5d(&mq, q, D, g.G[2], g.G[1], g.G[0], BH, g.bx, g.by, g.bt) ||
      !make_tmap_5d(&mk, k, D, g.G[2], g.G[1], g.G[0], BH, g.bx, g.by, g.bt) ||
      !make_tmap_5d(&mv, v, D, g.G[2], g.G[1], g.G[0], BH, g.bx, g.by, g.bt) ||
      !make_tmap_5d(&mdo, dout, D, g.G[2], g.G[1], g.G[0], BH, g.bx, g.by, g.bt))
    return cudaErrorInvalidValue;
  const int grid = (int)(a.items < num_sms() ? a.items : num_sms());
  auto k1 = sm103_dkdv_kernel<D, OutT>;
  cudaError_t e = cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, KvCfg<D>::kSmem);
  if (e != cudaSuccess) return e;
  prof_begin(kKBwdDkdv, st);
  k1<<<grid, kThreads, KvCfg<D>::kSmem, st>>>(mq, mk, mv, mdo, a);
  prof_end(kKBwdDkdv, st);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  auto k2 = sm103_dq_kernel<D, OutT>;
  e = cudaFuncSetAttribute(k2, cudaFuncAttributeMaxDynamicSharedMemorySize, QCfg<D>::kSmem);
  if (e != cudaSuccess) return e;
  prof_begin(kKBwdDq, st);
  k2<<<grid, kThreads, QCfg<D>::kSmem, st>>>(mq, mk, mv, mdo, a);
  prof_end(kKBwdDq, st);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sm103_bwd(const Geom& g, const __nv_bfloat16* q, const __nv_bfloat16* k, const __nv_bfloat16* v,
                             const __nv_bfloat16* dout, const float* lse2c, const float* dd, const void* ext,
                             void* dq, void* dk,
                             void* dv, int out_dtype, float* dq_s, float* dk_s, float* dv_s, uint32_t,
                             cudaStream_t st) {
  const bool bf = out_dtype == GATTN_BF16;
  using bf16 = __nv_bfloat16;
  if (g.d == 64)
    return launch_sm103_bwd64(g, q, k, v, dout, lse2c, dd, ext, dq, dk, dv, out_dtype, dq_s, dk_s, dv_s, st);
  if (g.d == 128)
    return bf ? run_bwd<128, bf16>(g, q, k, v, dout, lse2c, dd, dq, dk, dv, dq_s, dk_s, dv_s, st)
              : run_bwd<128, float>(g, q, k, v, dout, lse2c, dd, dq, dk, dv, dq_s, dk_s, dv_s, st);
  return cudaErrorNotSupported;
}

}  // namespace gattn
