// sm103_fwd.cu -- BF16 tensor-core forward of STORM-GPA tile attention on
// GB300 (sm_103a): tcgen05 MMAs with FP32 accumulators in TMEM, TMA-staged
// Q/K/V blocks, warp-specialised pipeline, fused tile epilogue.
//
// Per extended tile t (arXiv 2604.16590, Sec. III-C), for every 128-query block
// of the tile the CTA streams the tile's 128-key blocks (flash-style online
// softmax, the FlashAttention of Sec. III-D Level 5):
//   S_j  = Q K_j^T                      tcgen05, BF16 x BF16 -> FP32 (TMEM)
//   m_j  = max(m_{j-1}, rowmax(s S_j))  log2 domain
//   P_j  = exp2(s S_j log2e - m_j)      -> BF16, shared memory (SW128, K-major)
//   PV_j = P_j V_j                      tcgen05 -> FP32 (TMEM), V read MN-major
//   O   <- O exp2(m_O - m_{j}) + PV_j   FP32 registers (no TMEM read-modify-write)
// The epilogue writes O / l for rows covered by one tile straight to the output
// and parks multiply-covered rows (FP32) for the deterministic Hann merge, and
// stores the row log-sum-exp for the backward.
//
// Warp roles (192 threads, one CTA per SM, persistent over work items
// (batch*head, tile, query block)):
//   warp 0      TMA producer (Q once per item; K_j, V_j through a ring of stages)
//   warp 1      TMEM allocator + single-thread tcgen05 MMA issuer
//   warps 2..5  softmax + epilogue, one query row per thread (TMEM lane)
// TMEM: columns [0,256) two S buffers, [256, 256+d) the P V block product.
#include "internal.cuh"
#include "sm103_common.cuh"

GATTN_DEFINE_STATUS(sm103_fwd)

namespace gattn {
namespace {
using namespace sm103;

template <int D>
struct FwdCfg {
  static constexpr int kHalves = D / 64;            // 128-byte column chunks of a row
  static constexpr int kBlock = 128 * D * 2;        // bytes of one Q/K/V block
  static constexpr int kStages = D == 64 ? 3 : 2;   // K/V ring depth
  static constexpr int kPBytes = 128 * 128 * 2;
  static constexpr int kQ = 0;
  static constexpr int kK = kQ + kBlock;
  static constexpr int kV = kK + kStages * kBlock;
  static constexpr int kP = kV + kStages * kBlock;
  static constexpr int kBar = kP + kPBytes;
  // q_full, q_empty, k_full[S], k_empty[S], v_full[S], v_empty[S], s_full[2], s_empty[2], p_full, pv_done, drain
  static constexpr int kNumBars = 2 + 4 * kStages + 4 + 3;
  static constexpr int kMisc = kBar + kNumBars * 8;
  static constexpr int kSmem = kMisc + 16 + 1024;   // + slack for 1024-byte alignment
  static constexpr uint32_t kTmemCols = 512;
  static constexpr uint32_t kColO = 256;
};

struct FwdArgs {
  Geom g;
  void* out;
  float* lse2;
  float* ot;
  int items;  // B*nh * ntiles * nbmax_tot
};

__device__ __forceinline__ void decode_item(const FwdArgs& a, int w, int& bh, int& tile, int& qb) {
  qb = w % a.g.nbmax_tot;
  const int r = w / a.g.nbmax_tot;
  tile = r % a.g.ntiles;
  bh = r / a.g.ntiles;
}

__device__ void set_status_fwd(uint32_t c) { set_status(c); }

// Fold block Gp's P V (TMEM, relative to max mprev) into the FP32 register
// accumulator O (relative to max mO): O <- O exp2(mO - mprev) + PV.
template <int D>
__device__ __forceinline__ bool accumulate_pv(float (&O)[D], float& mO, float mprev, uint32_t Gp, uint32_t tO,
                                              uint64_t* pv_done, volatile int* abort_flag) {
  if (!sm103::mbar_wait<set_status_fwd>(pv_done, Gp & 1, abort_flag)) return false;
  sm103::tc_fence_after();
  const float sc = sm103::ex2(mO - mprev);
  uint32_t r[32];
#pragma unroll
  for (int c = 0; c < D / 32; ++c) {
    sm103::tmem_ld32(tO + c * 32, r);
    sm103::tmem_wait_ld(r);
#pragma unroll
    for (int i = 0; i < 32; ++i) O[c * 32 + i] = fmaf(O[c * 32 + i], sc, __uint_as_float(r[i]));
  }
  mO = mprev;
  return true;
}


// Online-softmax state of one query row.
template <int D>
struct RowState {
  float O[D];  // sum of P V relative to max mO
  float m;     // running row max (log2 domain, scaled)
  float l;     // running row sum relative to m
  float mO;    // max the register accumulator O is expressed against
  __device__ __forceinline__ void init() {
#pragma unroll
    for (int e = 0; e < D; ++e) O[e] = 0.f;
    m = -INFINITY;
    l = 0.f;
    mO = -INFINITY;
  }
};

template <int N>
__device__ __forceinline__ float tree_max(float (&v)[N]) {
#pragma unroll
  for (int w = N / 2; w >= 1; w /= 2)
#pragma unroll
    for (int i = 0; i < w; ++i) v[i] = fmaxf(v[i], v[i + w]);
  return v[0];
}
template <int N>
__device__ __forceinline__ float tree_sum(float (&v)[N]) {
#pragma unroll
  for (int w = N / 2; w >= 1; w /= 2)
#pragma unroll
    for (int i = 0; i < w; ++i) v[i] += v[i + w];
  return v[0];
}

// Exponentiate 32 scores of TMEM chunk c into BF16 P in shared memory
// (128-byte swizzled, K-major: row = query, 64 keys per 128-byte line).
template <bool MASK>
__device__ __forceinline__ void exp_store_chunk(const uint32_t (&r)[32], int c, uint32_t mbits, float sl2, float mnew,
                                                float (&acc)[8], uint32_t sP, int row) {
  uint32_t pk[16];
#pragma unroll
  for (int i = 0; i < 32; i += 2) {
    float p0 = sm103::ex2(fmaf(__uint_as_float(r[i]), sl2, -mnew));
    float p1 = sm103::ex2(fmaf(__uint_as_float(r[i + 1]), sl2, -mnew));
    if (MASK) {
      p0 = (mbits >> i) & 1u ? p0 : 0.f;
      p1 = (mbits >> (i + 1)) & 1u ? p1 : 0.f;
    }
    acc[(i >> 1) & 7] += p0 + p1;
    pk[i >> 1] = sm103::pack_bf16(p0, p1);
  }
  const uint32_t base = sP + (c >> 1) * 16384 + row * 128;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const uint32_t unit = ((c & 1) * 4 + u) ^ (row & 7);
    sm103::st_shared_v4(base + unit * 16, pk[4 * u], pk[4 * u + 1], pk[4 * u + 2], pk[4 * u + 3]);
  }
}

template <bool MASK>
__device__ __forceinline__ void chunk_max(const uint32_t (&r)[32], uint32_t mbits, float (&mx)[8]) {
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    float x = __uint_as_float(r[i]);
    if (MASK) x = (mbits >> i) & 1u ? x : -INFINITY;
    mx[i & 7] = fmaxf(mx[i & 7], x);
  }
}

// One 128-key block of the online softmax for this thread's query row:
// row max, fold of the previous block's P V (if any), P = exp2(...) to shared
// memory, row-sum update.  For d = 64 the whole 128-column score row is kept
// in registers; for d = 128 (larger accumulator) the scores are read from
// TMEM twice, 64 columns at a time.
template <int D, bool MASK>
__device__ __forceinline__ bool softmax_block(RowState<D>& rs, uint32_t tS, uint32_t tO, uint32_t sP, int row,
                                              const uint32_t (&kmask)[4], float sl2, bool has_prev, uint32_t G,
                                              uint64_t* pv_done, volatile int* abort_flag) {
  using namespace sm103;
  float mx[8], acc[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    mx[i] = -INFINITY;
    acc[i] = 0.f;
  }
  uint32_t r0[32], r1[32];
  if constexpr (D == 64) {
    uint32_t r2[32], r3[32];
    tmem_ld32(tS, r0);
    tmem_ld32(tS + 32, r1);
    tmem_ld32(tS + 64, r2);
    tmem_ld32(tS + 96, r3);
    tmem_wait_ld(r0);
    tmem_wait_ld(r1);
    tmem_wait_ld(r2);
    tmem_wait_ld(r3);
    chunk_max<MASK>(r0, kmask[0], mx);
    chunk_max<MASK>(r1, kmask[1], mx);
    chunk_max<MASK>(r2, kmask[2], mx);
    chunk_max<MASK>(r3, kmask[3], mx);
    const float mnew = fmaxf(rs.m, tree_max(mx) * sl2);
    if (has_prev && !accumulate_pv<D>(rs.O, rs.mO, rs.m, G - 1, tO, pv_done, abort_flag)) return false;
    exp_store_chunk<MASK>(r0, 0, kmask[0], sl2, mnew, acc, sP, row);
    exp_store_chunk<MASK>(r1, 1, kmask[1], sl2, mnew, acc, sP, row);
    exp_store_chunk<MASK>(r2, 2, kmask[2], sl2, mnew, acc, sP, row);
    exp_store_chunk<MASK>(r3, 3, kmask[3], sl2, mnew, acc, sP, row);
    rs.l = rs.l * ex2(rs.m - mnew) + tree_sum(acc);
    rs.m = mnew;
  } else {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      tmem_ld32(tS + 64 * h, r0);
      tmem_ld32(tS + 64 * h + 32, r1);
      tmem_wait_ld(r0);
      tmem_wait_ld(r1);
      chunk_max<MASK>(r0, kmask[2 * h], mx);
      chunk_max<MASK>(r1, kmask[2 * h + 1], mx);
    }
    const float mnew = fmaxf(rs.m, tree_max(mx) * sl2);
    if (has_prev && !accumulate_pv<D>(rs.O, rs.mO, rs.m, G - 1, tO, pv_done, abort_flag)) return false;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      tmem_ld32(tS + 64 * h, r0);
      tmem_ld32(tS + 64 * h + 32, r1);
      tmem_wait_ld(r0);
      tmem_wait_ld(r1);
      exp_store_chunk<MASK>(r0, 2 * h, kmask[2 * h], sl2, mnew, acc, sP, row);
      exp_store_chunk<MASK>(r1, 2 * h + 1, kmask[2 * h + 1], sl2, mnew, acc, sP, row);
    }
    rs.l = rs.l * ex2(rs.m - mnew) + tree_sum(acc);
    rs.m = mnew;
  }
  return true;
}

template <int D, typename OutT>
__global__ void __launch_bounds__(192, 1)
    sm103_fwd_kernel(const __grid_constant__ CUtensorMap tq, const __grid_constant__ CUtensorMap tk,
                     const __grid_constant__ CUtensorMap tv, const FwdArgs a) {
  using C = FwdCfg<D>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::kBar);
  uint64_t* q_full = bars + 0;
  uint64_t* q_empty = bars + 1;
  uint64_t* k_full = bars + 2;
  uint64_t* k_empty = k_full + C::kStages;
  uint64_t* v_full = k_empty + C::kStages;
  uint64_t* v_empty = v_full + C::kStages;
  uint64_t* s_full = v_empty + C::kStages;
  uint64_t* s_empty = s_full + 2;
  uint64_t* p_full = s_empty + 2;
  uint64_t* pv_done = p_full + 1;
  uint64_t* drain = pv_done + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + C::kMisc);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + C::kMisc + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    mbar_init(q_full, 1);
    mbar_init(q_empty, 1);
    for (int s = 0; s < C::kStages; ++s) {
      mbar_init(k_full + s, 1);
      mbar_init(k_empty + s, 1);
      mbar_init(v_full + s, 1);
      mbar_init(v_empty + s, 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(s_full + s, 1);
      mbar_init(s_empty + s, 4);
    }
    mbar_init(p_full, 4);
    mbar_init(pv_done, 1);
    mbar_init(drain, 1);
    *abort_flag = 0;
    fence_mbar_init();
    prefetch_tmap(&tq);
    prefetch_tmap(&tk);
    prefetch_tmap(&tv);
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, C::kTmemCols);
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
      // arming record for the abort drain: bit s of k_arm/v_arm = stage s armed at
      // least once, bit s of k_par/v_par = parity of its latest arming
      uint32_t k_arm = 0, v_arm = 0, k_par = 0, v_par = 0, q_arm = 0, q_par = 0;
      bool ok = true;
      for (int w = blockIdx.x; w < a.items && ok; w += gridDim.x) {
        int bh, tile, qb;
        decode_item(a, w, bh, tile, qb);
        TileBlocks tbk;
        tile_blocks(g, tile, tbk);
        if (qb >= tbk.NB) continue;
        int o[3];
        block_origin(g, tbk, qb, o);
        if (!(ok = mbar_wait<set_status_fwd>(q_empty, (W & 1) ^ 1, abort_flag))) break;
        mbar_arrive_expect_tx(q_full, C::kBlock);
        q_arm = 1;
        q_par = W & 1;
        for (int h = 0; h < C::kHalves; ++h)
          tma_load_5d(smem + C::kQ + h * 16384, &tq, q_full, 64 * h, tbk.tb.lo[2] + o[2], tbk.tb.lo[1] + o[1],
                      tbk.tb.lo[0] + o[0], bh);
        for (int j = 0; j < tbk.NB; ++j, ++G) {
          const uint32_t st = G % C::kStages, n = G / C::kStages;
          block_origin(g, tbk, j, o);
          const int c1 = tbk.tb.lo[2] + o[2], c2 = tbk.tb.lo[1] + o[1], c3 = tbk.tb.lo[0] + o[0];
          if (!(ok = mbar_wait<set_status_fwd>(k_empty + st, (n & 1) ^ 1, abort_flag))) break;
          mbar_arrive_expect_tx(k_full + st, C::kBlock);
          k_arm |= 1u << st;
          k_par = (k_par & ~(1u << st)) | ((n & 1) << st);
          for (int h = 0; h < C::kHalves; ++h)
            tma_load_5d(smem + C::kK + st * C::kBlock + h * 16384, &tk, k_full + st, 64 * h, c1, c2, c3, bh);
          if (!(ok = mbar_wait<set_status_fwd>(v_empty + st, (n & 1) ^ 1, abort_flag))) break;
          mbar_arrive_expect_tx(v_full + st, C::kBlock);
          v_arm |= 1u << st;
          v_par = (v_par & ~(1u << st)) | ((n & 1) << st);
          for (int h = 0; h < C::kHalves; ++h)
            tma_load_5d(smem + C::kV + st * C::kBlock + h * 16384, &tv, v_full + st, 64 * h, c1, c2, c3, bh);
        }
        ++W;
      }
      if (!ok) {
        // let every load this thread issued land before the CTA exits
        if (q_arm) mbar_wait<set_status_fwd>(q_full, q_par, abort_flag, false);
        for (int s = 0; s < C::kStages; ++s) {
          if (k_arm & (1u << s)) mbar_wait<set_status_fwd>(k_full + s, (k_par >> s) & 1, abort_flag, false);
          if (v_arm & (1u << s)) mbar_wait<set_status_fwd>(v_full + s, (v_par >> s) & 1, abort_flag, false);
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      constexpr uint32_t idS = idesc_bf16(128, 128, 0);
      constexpr uint32_t idO = idesc_bf16(128, D, 1);
      const uint32_t sQ = smem_u32(smem + C::kQ), sK = smem_u32(smem + C::kK), sV = smem_u32(smem + C::kV),
                     sP = smem_u32(smem + C::kP);
      uint32_t G = 0, W = 0;
      bool ok = true;
      auto issue_pv = [&](uint32_t Gp) -> bool {
        const uint32_t st = Gp % C::kStages;
        if (!mbar_wait<set_status_fwd>(v_full + st, (Gp / C::kStages) & 1, abort_flag)) return false;
        if (!mbar_wait<set_status_fwd>(p_full, Gp & 1, abort_flag)) return false;
        tc_fence_after();
#pragma unroll
        for (int ks = 0; ks < 8; ++ks) {
          const uint64_t ad = sw128_desc(sP + (ks >> 2) * 16384 + (ks & 3) * 32, 16, 1024);
          const uint64_t bd = sw128_desc(sV + st * C::kBlock + ks * 2048, 16384, 1024);
          umma_bf16(tmem + C::kColO, ad, bd, idO, ks > 0);
        }
        umma_commit(pv_done);
        umma_commit(v_empty + st);
        return true;
      };
      for (int w = blockIdx.x; w < a.items && ok; w += gridDim.x) {
        int bh, tile, qb;
        decode_item(a, w, bh, tile, qb);
        TileBlocks tbk;
        tile_blocks(g, tile, tbk);
        if (qb >= tbk.NB) continue;
        if (!(ok = mbar_wait<set_status_fwd>(q_full, W & 1, abort_flag))) break;
        tc_fence_after();
        for (int j = 0; j < tbk.NB; ++j, ++G) {
          const uint32_t st = G % C::kStages, sb = G & 1;
          if (!(ok = mbar_wait<set_status_fwd>(k_full + st, (G / C::kStages) & 1, abort_flag))) break;
          if (!(ok = mbar_wait<set_status_fwd>(s_empty + sb, ((G >> 1) & 1) ^ 1, abort_flag))) break;
          tc_fence_after();
#pragma unroll
          for (int ks = 0; ks < D / 16; ++ks) {
            const uint32_t off = (ks >> 2) * 16384 + (ks & 3) * 32;
            umma_bf16(tmem + sb * 128, sw128_desc(sQ + off, 16, 1024), sw128_desc(sK + st * C::kBlock + off, 16, 1024),
                      idS, ks > 0);
          }
          umma_commit(s_full + sb);
          umma_commit(k_empty + st);
          if (j == tbk.NB - 1) umma_commit(q_empty);
          if (j > 0 && !(ok = issue_pv(G - 1))) break;
        }
        if (!ok) break;
        if (!(ok = issue_pv(G - 1))) break;
        ++W;
      }
      // all issued MMAs complete before TMEM is released
      umma_commit(drain);
      mbar_wait<set_status_fwd>(drain, 0, abort_flag, false);
    }
  } else {
    // ------------------------------------------------------------ softmax + epilogue
    const int quad = warp & 3;
    const int row = quad * 32 + lane;  // TMEM lane = block row
    const uint32_t tl = tmem + ((uint32_t)(quad * 32) << 16);
    const uint32_t sP = smem_u32(smem + C::kP);
    uint32_t G = 0;
    bool ok = true;
    for (int w = blockIdx.x; w < a.items && ok; w += gridDim.x) {
      int bh, tile, qb;
      decode_item(a, w, bh, tile, qb);
      TileBlocks tbk;
      tile_blocks(g, tile, tbk);
      if (qb >= tbk.NB) continue;
      int qo[3], ql[3];
      block_origin(g, tbk, qb, qo);
      block_row(g, qo, row, ql);
      const bool qvalid = inside(tbk, ql);

      RowState<D> rs;
      rs.init();
      for (int j = 0; j < tbk.NB; ++j, ++G) {
        const uint32_t sb = G & 1;
        int ko[3];
        block_origin(g, tbk, j, ko);
        // key validity of the block's 128 columns, one ballot per 32 columns
        uint32_t kmask[4];
        const bool full = block_full(g, tbk, ko);
        if (!full) {
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            int kl[3];
            block_row(g, ko, c * 32 + lane, kl);
            kmask[c] = __ballot_sync(0xffffffffu, inside(tbk, kl));
          }
        }
        if (!(ok = mbar_wait<set_status_fwd>(s_full + sb, (G >> 1) & 1, abort_flag))) break;
        tc_fence_after();
        if (full)
          ok = softmax_block<D, false>(rs, tl + sb * 128, tl + C::kColO, sP, row, kmask, g.scale_log2, j > 0, G, pv_done, abort_flag);
        else
          ok = softmax_block<D, true>(rs, tl + sb * 128, tl + C::kColO, sP, row, kmask, g.scale_log2, j > 0, G, pv_done, abort_flag);
        if (!ok) break;
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(s_empty + sb);
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(p_full);
      }
      if (!ok) break;
      if (!(ok = accumulate_pv<D>(rs.O, rs.mO, rs.m, G - 1, tl + C::kColO, pv_done, abort_flag))) break;
      tc_fence_before();
      // ---- epilogue
      if (qvalid) {
        const int64_t slot = tile_slot0(g, bh, tile) + qb * 128 + row;
        a.lse2[slot] = rs.m + __log2f(rs.l);
        const int p[3] = {tbk.tb.lo[0] + ql[0], tbk.tb.lo[1] + ql[1], tbk.tb.lo[2] + ql[2]};
        const int64_t tok = ((int64_t)p[0] * g.G[1] + p[1]) * g.G[2] + p[2];
        const float inv = 1.f / rs.l;
        if (single_cover(g, p)) {
          OutT* dst = static_cast<OutT*>(a.out) + ((int64_t)bh * g.N + tok) * D;
#pragma unroll
          for (int e = 0; e < D; e += 4)
            store4<OutT>(dst + e, make_float4(rs.O[e] * inv, rs.O[e + 1] * inv, rs.O[e + 2] * inv, rs.O[e + 3] * inv));
        } else {
          float* dst = a.ot + slot * D;
#pragma unroll
          for (int e = 0; e < D; e += 4)
            store4<float>(dst + e, make_float4(rs.O[e] * inv, rs.O[e + 1] * inv, rs.O[e + 2] * inv, rs.O[e + 3] * inv));
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, C::kTmemCols);
  }
}

template <int D, typename OutT>
cudaError_t run_fwd(const Geom& g, const __nv_bfloat16* q, const __nv_bfloat16* k, const __nv_bfloat16* v, void* out,
                    float* lse2, float* ot, cudaStream_t st) {
  using C = FwdCfg<D>;
  FwdArgs a;
  a.g = g;
  a.out = out;
  a.lse2 = lse2;
  a.ot = ot;
  const int64_t items = (int64_t)g.B * g.nh * g.ntiles * g.nbmax_tot;
  if (items >= (1LL << 31)) return cudaErrorNotSupported;
  a.items = (int)items;
  const int BH = g.B * g.nh;
  CUtensorMap mq, mk, mv;
  if (!make_tmap_5d(&mq, q, D, g.G[2], g.G[1], g.G[0], BH, g.bx, g.by, g.bt) ||
      !make_tmap_5d(&mk, k, D, g.G[2], g.G[1], g.G[0], BH, g.bx, g.by, g.bt) ||
      !make_tmap_5d(&mv, v, D, g.G[2], g.G[1], g.G[0], BH, g.bx, g.by, g.bt))
    return cudaErrorInvalidValue;
  auto kern = sm103_fwd_kernel<D, OutT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmem);
  if (e != cudaSuccess) return e;
  const int grid = (int)(a.items < num_sms() ? a.items : num_sms());
  kern<<<grid, 192, C::kSmem, st>>>(mq, mk, mv, a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sm103_fwd(const Geom& g, const __nv_bfloat16* q, const __nv_bfloat16* k, const __nv_bfloat16* v,
                             void* out, int out_dtype, float* lse2, float* ot, uint32_t, cudaStream_t st) {
  const bool bf = out_dtype == GATTN_BF16;
  if (g.d == 64)
    return bf ? run_fwd<64, __nv_bfloat16>(g, q, k, v, out, lse2, ot, st) : run_fwd<64, float>(g, q, k, v, out, lse2, ot, st);
  if (g.d == 128)
    return bf ? run_fwd<128, __nv_bfloat16>(g, q, k, v, out, lse2, ot, st)
              : run_fwd<128, float>(g, q, k, v, out, lse2, ot, st);
  return cudaErrorNotSupported;
}

}  // namespace gattn
