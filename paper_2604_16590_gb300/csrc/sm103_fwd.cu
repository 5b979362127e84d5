// sm103_fwd.cu -- BF16 tensor-core forward of STORM-GPA tile attention on
// GB300 (sm_103a): tcgen05 MMAs with FP32 accumulators in TMEM, TMA-staged
// Q/K/V blocks, warp-specialised pipeline, fused tile epilogue.
//
// Per extended tile t (arXiv 2604.16590, Sec. III-C), for every 128-query block
// of the tile the CTA streams the tile's 128-key blocks (flash-style online
// softmax, the FlashAttention of Sec. III-D Level 5):
//   S_j  = Q K_j^T                      tcgen05, A = Q from TMEM, B = K from smem -> FP32 TMEM
//   m_j  = max(m_{j-1}, rowmax(s S_j))  log2 domain
//   P_j  = exp2(s S_j log2e - m_j)      -> BF16 pairs written into TMEM (tcgen05.st)
//   PV_j = P_j V_j                      tcgen05, A = P from TMEM, B = V (MN-major) from smem
//   O   <- O exp2(m_O - m_{j}) + PV_j   FP32 registers (no TMEM read-modify-write)
// Keeping Q and P in tensor memory leaves shared memory with only the TMA'd K/V
// blocks and the B-operand reads (about 64 KB per 128x128 block instead of
// 144 KB): the 128 B/clk shared-memory read path otherwise limits the MMAs.
// The epilogue writes O / l for rows covered by one tile straight to the output
// and parks multiply-covered rows (FP32) for the deterministic Hann merge, and
// stores the row log-sum-exp for the backward.
//
// Warp roles (320 threads, one CTA per SM, persistent over work items
// (batch*head, tile, query block)):
//   warp 0      TMA producer (Q once per item; K_j, V_j through a ring of stages)
//   warp 1      TMEM allocator + issuer of the S = Q K^T products
//   warps 2..9  softmax + epilogue: one query row per TMEM lane, two warps per
//               lane quadrant splitting each row's keys and output columns
//               (two math warps per SM sub-partition hide TMEM/MUFU latency)
//   warp 10     issuer of the P V products
// Two issuing threads, because a thread's shared-memory accesses (an mbarrier
// wait included) are held until the tcgen05.mma it issued before them have
// drained from the tensor pipe: with one issuer every wait between the S and
// the P V products emptied the pipe; with two, one thread's waits overlap the
// other's MMAs.  The barriers order every TMEM region and stage they share.
// TMEM: columns [0,256) two S buffers, [256, 256+d) the P V block product,
// then 64 columns of P (BF16 pairs) and d/2 columns of Q (BF16 pairs).
#include <string.h>

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
  static constexpr int kStages = D == 64 ? 4 : 2;   // K/V ring depth
  static constexpr int kQ = 0;
  static constexpr int kK = kQ + kBlock;
  static constexpr int kV = kK + kStages * kBlock;
  static constexpr int kBar = kV + kStages * kBlock;
  // q_full, q_empty, qt_full, k_full[S], k_empty[S], v_full[S], v_empty[S], s_full[2], s_empty[2],
  // p_full, pv_done[2], o_empty, drain[2], never (test hook: nothing arrives on it)
  static constexpr int kNumBars = 3 + 4 * kStages + 4 + 7;
  static constexpr int kMisc = kBar + kNumBars * 8;
  static constexpr int kRed = kMisc + 16;           // float [3 slots][2 half][128 rows]
  static constexpr int kSmem = kRed + 3072 + 1024;  // + slack for 1024-byte alignment
  static constexpr uint32_t kTmemCols = 512;
  static constexpr int kPBufs = D == 64 ? 2 : 1;    // P buffers in TMEM
  static constexpr uint32_t kColO = 256;            // O accumulator, D columns
  static constexpr uint32_t kColP = 256 + D;        // kPBufs x 64 columns: 128 keys as BF16 pairs
  static constexpr uint32_t kColQ = 256 + D + 64 * kPBufs;  // D/2 columns: the query block as BF16 pairs
  static_assert(kColQ + D / 2 <= kTmemCols, "TMEM budget");
};

struct FwdArgs {
  Geom g;
  void* out;
  float* lse2;
  float* ot;
  int items;  // B*nh * ntiles * nbmax_tot
  uint32_t flags;  // GATTN_FLAG_*
  int pad_R;  // box rows of every geometry of the launch (rows pad_R..127 of each block are zeroed once)
  // ragged mode (serving): per-request descriptors and device-side counts
  const ReqDesc* reqs;
  const int64_t* counts;
};

// One work item (batch*head, tile, 128-row block) resolved to its problem.
struct Item {
  const Geom* g;
  const CUtensorMap* tq;
  const CUtensorMap* tk;
  const CUtensorMap* tv;
  void* out;
  float* lse2;  // may be null (no backward)
  float* ot;
  int bh, tile, blk;
  int req;  // request index (ragged mode), else -1
};

// Returns false (after recording GATTN_ERR_DEVICE_BOUNDS) if a ragged work
// item does not decode to a valid (request, head, tile, block); every role
// decodes the same item identically, so all of them skip it together.
template <bool RAGGED>
__device__ __forceinline__ bool resolve(const FwdArgs& a, const CUtensorMap* tq, const CUtensorMap* tk,
                                        const CUtensorMap* tv, int w, Item& it) {
  int req = -1;
  if constexpr (RAGGED) {
    // requests are sorted by item0: binary search for the last item0 <= w
    const int nreq = (int)a.counts[0];
    int lo = 0, hi = nreq - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (a.reqs[mid].item0 <= w) lo = mid;
      else hi = mid - 1;
    }
    if (nreq < 1 || w < a.reqs[lo].item0 || w >= a.reqs[lo].item0 + a.reqs[lo].items) {
      set_status(kStatusBounds);
      return false;
    }
    req = lo;
    const ReqDesc& r = a.reqs[lo];
    it.g = &r.g;
    it.tq = it.tk = it.tv = &r.tmap;
    it.out = r.out;
    it.lse2 = nullptr;
    it.ot = r.ot;
    w -= r.item0;
  } else {
    it.g = &a.g;
    it.tq = tq;
    it.tk = tk;
    it.tv = tv;
    it.out = a.out;
    it.lse2 = a.lse2;
    it.ot = a.ot;
  }
  const Geom& g = *it.g;
  it.blk = w % g.nbmax_tot;
  const int r = w / g.nbmax_tot;
  it.tile = r % g.ntiles;
  it.bh = r / g.ntiles;
  it.req = req;
  if (RAGGED && (it.bh >= g.B * g.nh || g.R != a.pad_R)) {
    set_status(kStatusBounds);
    return false;
  }
  return true;
}

template <bool RAGGED>
__device__ __forceinline__ int total_items(const FwdArgs& a) {
  if constexpr (RAGGED) return (int)a.counts[1];
  else return a.items;
}

__device__ void set_status_fwd(uint32_t c) { set_status(c); }

// Math warps: two per TMEM lane quadrant; the two warps of a quadrant share
// its 32 query rows, warp half `ch` owning keys [64 ch, 64 ch + 64) of every
// block (one 64-key chunk of P) and output columns [ch D/2, (ch+1) D/2).
constexpr int kMathWarps = 8;
constexpr int kThreads = 64 + 32 * kMathWarps + 32;
constexpr int kIssuerPV = 2 + kMathWarps;  // warp index of the P V issuer

// Online-softmax state of one query row, as held by one of its two threads.
// P = exp2(s S log2e - m) is formed against a reference max m that only moves
// when a row max exceeds it by more than kRescaleLog2 (then O in TMEM and l
// are rescaled once); O itself accumulates in TMEM across the key blocks.
constexpr float kRescaleLog2 = 8.f;
struct RowState {
  float m;   // reference max (log2 domain, scaled), same in both threads of the row
  float l;   // this thread's half of the row sum, relative to m
  float lc;  // Kahan compensation of l (the sum runs over every key block of the tile)
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

// named barrier of the two warps that share a TMEM lane quadrant
__device__ __forceinline__ void pair_sync(int quad) {
  asm volatile("bar.sync %0, 64;" ::"r"(quad + 1) : "memory");
}

// Exchange a per-row partial value with the partner thread (same row, other
// column half).  Slots 0/1 alternate between key blocks and slot 2 serves the
// epilogue, so a fast thread never overwrites a value its partner has not
// read yet (every reuse of a slot is separated by another pair barrier).
__device__ __forceinline__ float pair_exchange(float* red, int parity, int ch, int row, int quad, float v) {
  red[(parity * 2 + ch) * 128 + row] = v;
  pair_sync(quad);
  return red[(parity * 2 + (ch ^ 1)) * 128 + row];
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
    mx[(i >> 1) & 3] = sm103::fmax3(mx[(i >> 1) & 3], x0, x1);
  }
}

// exp2 of 32 scores -> 16 BF16 pairs (for TMEM), with the exp2 argument and the
// row sum formed by packed FP32 pair instructions
template <bool MASK>
__device__ __forceinline__ void exp_chunk(const uint32_t (&r)[32], uint32_t mbits, uint64_t s2, uint64_t nm2,
                                          uint64_t (&acc)[4], uint32_t* pk) {
  using namespace sm103;
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

// One 128-key block of the online softmax for this thread's half of a query
// row: partial row max (exchanged with the partner), fold of the previous
// block's P V into O, exp2 of its 64 scores into P (shared memory), row-sum.
// Rescale this thread's half (D/2 columns) of the O accumulator in TMEM by
// `f` (1 for rows that keep their reference max).  Warp-synchronous.
template <int D>
__device__ __forceinline__ void rescale_o(uint32_t tO, float f) {
  using namespace sm103;
  const uint64_t f2 = f2pack(f, f);
  uint32_t r[32];
#pragma unroll
  for (int c = 0; c < D / 64; ++c) {
    tmem_ld32(tO + c * 32, r);
    tmem_wait_ld(r);
#pragma unroll
    for (int i = 0; i < 32; i += 2) {
      float x, y;
      f2unpack(fmul2(u2pack(r[i], r[i + 1]), f2), x, y);
      r[i] = __float_as_uint(x);
      r[i + 1] = __float_as_uint(y);
    }
    tmem_st32(tO + c * 32, r);
  }
  tmem_wait_st();
}

// One 128-key block of the online softmax for this thread's half of a query
// row: partial row max (exchanged with the partner thread), lazy rescale of
// the reference max (and of O in TMEM, after the previous P V completed),
// exp2 of the 64 scores into BF16 P in TMEM, row-sum update.
template <int D, bool MASK>
__device__ __forceinline__ bool softmax_block(RowState& rs, uint32_t tS, uint32_t tO, uint32_t tP, int row, int ch,
                                              int quad, float* red, int parity, const uint32_t (&kmask)[2], float sl2,
                                              bool first,
                                              uint64_t* pv_last, uint32_t pv_last_par, uint64_t* p_free,
                                              uint32_t p_free_par, volatile int* abort_flag) {
  using namespace sm103;
  float mx[4];
  uint64_t acc[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    mx[i] = -INFINITY;
    acc[i] = f2pack(0.f, 0.f);
  }
  uint32_t r0[32], r1[32];
  tmem_ld32(tS, r0);
  tmem_ld32(tS + 32, r1);
  tmem_wait_ld(r0);
  tmem_wait_ld(r1);
  chunk_max<MASK>(r0, kmask[0], mx);
  chunk_max<MASK>(r1, kmask[1], mx);
  const float mine = fmaxf(fmaxf(mx[0], mx[1]), fmaxf(mx[2], mx[3]));
  const float other = pair_exchange(red, parity, ch, row, quad, mine);
  const float mblk = fmaxf(mine, other) * sl2;
  if (first) {
    rs.m = mblk;  // O is written fresh by this block's P V
  } else {
    const bool grow = mblk > rs.m + kRescaleLog2;
    if (__any_sync(0xffffffffu, grow)) {
      // O must not be in flight: wait for the previous block's P V
      if (!mbar_wait<set_status_fwd>(pv_last, pv_last_par, abort_flag)) return false;
      tc_fence_after();
      const float f = grow ? ex2(rs.m - mblk) : 1.f;
      rescale_o<D>(tO, f);
      rs.l *= f;
      rs.lc *= f;
      if (grow) rs.m = mblk;
    }
  }
  const uint64_t s2 = f2pack(sl2, sl2), nm2 = f2pack(-rs.m, -rs.m);
  uint32_t pk0[16], pk1[16];
  exp_chunk<MASK>(r0, kmask[0], s2, nm2, acc, pk0);
  exp_chunk<MASK>(r1, kmask[1], s2, nm2, acc, pk1);
  // this P buffer is free once the P V product that last read it completed
  if (!mbar_wait<set_status_fwd>(p_free, p_free_par, abort_flag)) return false;
  tc_fence_after();
  tmem_st16(tP, pk0);  // keys [64 ch, 64 ch + 64) -> P columns [32 ch, 32 ch + 32)
  tmem_st16(tP + 16, pk1);
  float lsum = 0.f;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float x, y;
    f2unpack(acc[i], x, y);
    lsum += x + y;
  }
  {  // compensated: tiles of the long temporal context span thousands of key blocks
    const float y = lsum - rs.lc;
    const float t = rs.l + y;
    rs.lc = (t - rs.l) - y;
    rs.l = t;
  }
  tmem_wait_st();
  return true;
}

template <int D, typename OutT, bool RAGGED>
__global__ void __launch_bounds__(kThreads, 1)
    sm103_fwd_kernel(const __grid_constant__ CUtensorMap tq, const __grid_constant__ CUtensorMap tk,
                     const __grid_constant__ CUtensorMap tv, const FwdArgs a) {
  using C = FwdCfg<D>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::kBar);
  uint64_t* q_full = bars + 0;
  uint64_t* q_empty = bars + 1;
  uint64_t* qt_full = bars + 2;
  uint64_t* k_full = bars + 3;
  uint64_t* k_empty = k_full + C::kStages;
  uint64_t* v_full = k_empty + C::kStages;
  uint64_t* v_empty = v_full + C::kStages;
  uint64_t* s_full = v_empty + C::kStages;
  uint64_t* s_empty = s_full + 2;
  uint64_t* p_full = s_empty + 2;
  uint64_t* pv_done = p_full + 1;  // [2], one per P buffer
  uint64_t* o_empty = pv_done + 2;
  uint64_t* drain = o_empty + 1;  // [2]: one per issuing thread
  uint64_t* never = drain + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + C::kMisc);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + C::kMisc + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  zero_pad_rows(smem, (1 + 2 * C::kStages) * C::kHalves, a.pad_R);  // Q and the K and V rings
  if (threadIdx.x == 0) {
    mbar_init(q_full, 1);
    mbar_init(q_empty, kMathWarps);
    mbar_init(qt_full, kMathWarps);
    for (int s = 0; s < C::kStages; ++s) {
      mbar_init(k_full + s, 1);
      mbar_init(k_empty + s, 1);
      mbar_init(v_full + s, 1);
      mbar_init(v_empty + s, 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(s_full + s, 1);
      mbar_init(s_empty + s, kMathWarps);
    }
    mbar_init(p_full, kMathWarps);
    mbar_init(pv_done, 1);
    mbar_init(pv_done + 1, 1);
    mbar_init(o_empty, kMathWarps);
    mbar_init(drain, 1);
    mbar_init(drain + 1, 1);
    mbar_init(never, 1);
    *abort_flag = 0;
    fence_mbar_init();
    if (!RAGGED) {
      prefetch_tmap(&tq);
      prefetch_tmap(&tk);
      prefetch_tmap(&tv);
    }
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, C::kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int n_items = total_items<RAGGED>(a);

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      uint32_t G = 0, W = 0;
      // arming record for the abort drain: bit s of k_arm/v_arm = stage s armed at
      // least once, bit s of k_par/v_par = parity of its latest arming
      uint32_t k_arm = 0, v_arm = 0, k_par = 0, v_par = 0, q_arm = 0, q_par = 0;
      int last_req = -1;
      bool ok = true;
      for (int w = blockIdx.x; w < n_items && ok; w += gridDim.x) {
        Item it;
        if (!resolve<RAGGED>(a, &tq, &tk, &tv, w, it)) continue;
        const Geom& g = *it.g;
        const int bh = it.bh, tile = it.tile, qb = it.blk;
        TileBlocks tbk;
        tile_blocks(g, tile, tbk);
        if (qb >= tbk.NB) continue;
        if (RAGGED && it.req != last_req) {
          tmap_acquire(it.tq);  // this launch's descriptor table may hold a new map here
          last_req = it.req;
        }
        int o[3];
        block_origin(g, tbk, qb, o);
        if (!(ok = mbar_wait<set_status_fwd>(q_empty, (W & 1) ^ 1, abort_flag))) break;
        mbar_arrive_expect_tx(q_full, C::kHalves * g.R * 128);
        q_arm = 1;
        q_par = W & 1;
        for (int h = 0; h < C::kHalves; ++h)
          tma_load_5d(smem + C::kQ + h * 16384, it.tq, q_full, 64 * h, tbk.tb.lo[2] + o[2], tbk.tb.lo[1] + o[1],
                      tbk.tb.lo[0] + o[0], bh);
        for (int j = 0; j < tbk.NB; ++j, ++G) {
          const uint32_t st = G % C::kStages, n = G / C::kStages;
          block_origin(g, tbk, j, o);
          const int c1 = tbk.tb.lo[2] + o[2], c2 = tbk.tb.lo[1] + o[1], c3 = tbk.tb.lo[0] + o[0];
          if (!(ok = mbar_wait<set_status_fwd>(k_empty + st, (n & 1) ^ 1, abort_flag))) break;
          mbar_arrive_expect_tx(k_full + st, C::kHalves * g.R * 128);
          k_arm |= 1u << st;
          k_par = (k_par & ~(1u << st)) | ((n & 1) << st);
          for (int h = 0; h < C::kHalves; ++h)
            tma_load_5d(smem + C::kK + st * C::kBlock + h * 16384, it.tk, k_full + st, 64 * h, c1, c2, c3, bh);
          if (!(ok = mbar_wait<set_status_fwd>(v_empty + st, (n & 1) ^ 1, abort_flag))) break;
          mbar_arrive_expect_tx(v_full + st, C::kHalves * g.R * 128);
          v_arm |= 1u << st;
          v_par = (v_par & ~(1u << st)) | ((n & 1) << st);
          for (int h = 0; h < C::kHalves; ++h)
            tma_load_5d(smem + C::kV + st * C::kBlock + h * 16384, it.tv, v_full + st, 64 * h, c1, c2, c3, bh);
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
    // ------------------------------------------------------------ issuer of S = Q K^T
    if (lane == 0) {
      constexpr uint32_t idS = idesc_bf16(128, 128, 0);
      const uint64_t dK0 = sw128_desc(smem_u32(smem + C::kK), 16, 1024);
      uint32_t G = 0, W = 0;
      bool ok = true;
      if (a.flags & GATTN_FLAG_TEST_STALL)  // failure-detection hook: a wait that cannot complete
        ok = mbar_wait<set_status_fwd>(never, 0, abort_flag, true, 20000000ull);
      for (int w = blockIdx.x; w < n_items && ok; w += gridDim.x) {
        Item it;
        if (!resolve<RAGGED>(a, &tq, &tk, &tv, w, it)) continue;
        TileBlocks tbk;
        tile_blocks(*it.g, it.tile, tbk);
        if (it.blk >= tbk.NB) continue;
        if (!(ok = mbar_wait<set_status_fwd>(qt_full, W & 1, abort_flag))) break;  // Q in TMEM
        for (int j = 0; j < tbk.NB; ++j, ++G) {
          const uint32_t st = G % C::kStages, sb = G & 1;
          if (!(ok = mbar_wait<set_status_fwd>(k_full + st, (G / C::kStages) & 1, abort_flag))) break;
          if (!(ok = mbar_wait<set_status_fwd>(s_empty + sb, ((G >> 1) & 1) ^ 1, abort_flag))) break;
          tc_fence_after();
          const uint64_t dk = dmove(dK0, st * C::kBlock);
#pragma unroll
          for (int ks = 0; ks < D / 16; ++ks)
            umma_bf16_ts(tmem + sb * 128, tmem + C::kColQ + ks * 8, dmove(dk, (ks >> 2) * 16384 + (ks & 3) * 32),
                         idS, ks > 0);
          umma_commit(s_full + sb);
          umma_commit(k_empty + st);
        }
        ++W;
      }
      // all issued MMAs complete before TMEM is released
      umma_commit(drain);
      mbar_wait<set_status_fwd>(drain, 0, abort_flag, false);
    }
  } else if (warp == kIssuerPV) {
    // ------------------------------------------------------------ issuer of O += P V
    if (lane == 0) {
      constexpr uint32_t idO = idesc_bf16(128, D, 1);
      const uint64_t dV0 = sw128_desc(smem_u32(smem + C::kV), 16384, 1024);  // MN-major (K = keys)
      uint32_t G = 0, W = 0;
      bool ok = true;
      for (int w = blockIdx.x; w < n_items && ok; w += gridDim.x) {
        Item it;
        if (!resolve<RAGGED>(a, &tq, &tk, &tv, w, it)) continue;
        TileBlocks tbk;
        tile_blocks(*it.g, it.tile, tbk);
        if (it.blk >= tbk.NB) continue;
        for (int j = 0; j < tbk.NB; ++j, ++G) {
          const uint32_t st = G % C::kStages, pb = G % C::kPBufs;
          if (!(ok = mbar_wait<set_status_fwd>(v_full + st, (G / C::kStages) & 1, abort_flag))) break;
          if (!(ok = mbar_wait<set_status_fwd>(p_full, G & 1, abort_flag))) break;
          if (j == 0 && !(ok = mbar_wait<set_status_fwd>(o_empty, (W & 1) ^ 1, abort_flag))) break;
          tc_fence_after();
          const uint64_t dv = dmove(dV0, st * C::kBlock);
#pragma unroll
          for (int ks = 0; ks < 8; ++ks)
            umma_bf16_ts(tmem + C::kColO, tmem + C::kColP + pb * 64 + ks * 8, dmove(dv, ks * 2048), idO,
                         (j > 0 || ks > 0) ? 1u : 0u);
          umma_commit(pv_done + pb);
          umma_commit(v_empty + st);
        }
        if (!ok) break;
        ++W;
      }
      umma_commit(drain + 1);
      mbar_wait<set_status_fwd>(drain + 1, 0, abort_flag, false);
    }
  } else {
    // ------------------------------------------------------------ softmax + epilogue
    const int quad = warp & 3;
    const int ch = (warp - 2) >> 2;    // key half of every block / output-column half
    const int row = quad * 32 + lane;  // TMEM lane = block row
    const uint32_t tl = tmem + ((uint32_t)(quad * 32) << 16);
    const uint32_t tO = tl + C::kColO + ch * (D / 2);
    float* red = reinterpret_cast<float*>(smem + C::kRed);
    uint32_t G = 0, W = 0;
    bool ok = true;
    for (int w = blockIdx.x; w < n_items && ok; w += gridDim.x) {
      Item it;
      if (!resolve<RAGGED>(a, &tq, &tk, &tv, w, it)) continue;
      const Geom& g = *it.g;
      const int bh = it.bh, tile = it.tile, qb = it.blk;
      TileBlocks tbk;
      tile_blocks(g, tile, tbk);
      if (qb >= tbk.NB) continue;
      int qo[3], ql[3];
      block_origin(g, tbk, qb, qo);
      block_row(g, qo, row, ql);
      const bool qvalid = inside(tbk, ql);

      // the query block: shared memory (TMA) -> registers -> TMEM (A operand of S = Q K^T)
      if (!(ok = mbar_wait<set_status_fwd>(q_full, W & 1, abort_flag))) break;
      {
        const uint32_t sQ = smem_u32(smem + C::kQ);
        if constexpr (D == 64) {
          uint32_t qr[16];
          ld_swizzled_row<4>(sQ, row, 4 * ch, qr);  // elements [32 ch, 32 ch + 32)
          tmem_st16(tl + C::kColQ + 16 * ch, qr);
        } else {
          uint32_t qr[32];
          ld_swizzled_row<8>(sQ + ch * 16384, row, 0, qr);  // elements [64 ch, 64 ch + 64)
          tmem_st32(tl + C::kColQ + 32 * ch, qr);
        }
        tmem_wait_st();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(q_empty);
          mbar_arrive(qt_full);
        }
      }

      RowState rs;
      rs.m = -INFINITY;
      rs.l = 0.f;
      rs.lc = 0.f;
      // key-block coordinates stepped incrementally (no divisions in the loop)
      int jt = 0, jy = 0, jx = 0;
      for (int j = 0; j < tbk.NB; ++j, ++G) {
        const uint32_t sb = G & 1, pb = G % C::kPBufs;
        const int ko[3] = {jt * g.bt, jy * g.by, jx * g.bx};
        if (++jx == tbk.nb[2]) {
          jx = 0;
          if (++jy == tbk.nb[1]) {
            jy = 0;
            ++jt;
          }
        }
        // validity of this thread's 64 key columns, one ballot per 32
        uint32_t kmask[2] = {~0u, ~0u};
        const bool full = block_full(g, tbk, ko);
        if (!full) {
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            int kl[3];
            block_row(g, ko, ch * 64 + c * 32 + lane, kl);
            kmask[c] = __ballot_sync(0xffffffffu, inside(tbk, kl));
          }
        }
        if (!(ok = mbar_wait<set_status_fwd>(s_full + sb, (G >> 1) & 1, abort_flag))) break;
        tc_fence_after();
        const uint32_t tS = tl + sb * 128 + ch * 64;
        const uint32_t tP = tl + C::kColP + pb * 64 + ch * 32;
        // previous block's P V (for a rescale of O) and the P V that last read this P buffer
        uint64_t* pv_last = pv_done + (G - 1) % C::kPBufs;
        const uint32_t pv_last_par = ((G - 1) / C::kPBufs) & 1;
        const uint32_t p_free_par = ((G / C::kPBufs) & 1) ^ 1;
        if (full)
          ok = softmax_block<D, false>(rs, tS, tO, tP, row, ch, quad, red, sb, kmask, g.scale_log2, j == 0, pv_last,
                                       pv_last_par, pv_done + pb, p_free_par, abort_flag);
        else
          ok = softmax_block<D, true>(rs, tS, tO, tP, row, ch, quad, red, sb, kmask, g.scale_log2, j == 0, pv_last,
                                      pv_last_par, pv_done + pb, p_free_par, abort_flag);
        if (!ok) break;
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(s_empty + sb);
          mbar_arrive(p_full);
        }
      }
      if (!ok) break;
      // ---- epilogue: wait for the last P V, full row sum from the two halves, O / l
      if (!(ok = mbar_wait<set_status_fwd>(pv_done + (G - 1) % C::kPBufs, ((G - 1) / C::kPBufs) & 1, abort_flag)))
        break;
      tc_fence_after();
      const float l = rs.l + pair_exchange(red, 2, ch, row, quad, rs.l);  // slot 2: epilogue only
      const float inv = 1.f / l;
      const int64_t slot = tile_slot0(g, bh, tile) + qb * 128 + row;
      if (qvalid && ch == 0 && it.lse2) it.lse2[slot] = rs.m + __log2f(l);
      const int p[3] = {tbk.tb.lo[0] + ql[0], tbk.tb.lo[1] + ql[1], tbk.tb.lo[2] + ql[2]};
      const int64_t tok = qvalid ? ((int64_t)p[0] * g.G[1] + p[1]) * g.G[2] + p[2] : 0;
      const bool single = qvalid && single_cover(g, p);
      const int c0 = ch * (D / 2);
      OutT* dst_out = static_cast<OutT*>(it.out) + ((int64_t)bh * g.N + tok) * D + c0;
      float* dst_scr = it.ot + slot * D + c0;
      uint32_t r[32];
#pragma unroll
      for (int c = 0; c < D / 64; ++c) {
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
      if (lane == 0) mbar_arrive(o_empty);
      ++W;
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
                    float* lse2, float* ot, uint32_t flags, cudaStream_t st) {
  using C = FwdCfg<D>;
  FwdArgs a;
  a.g = g;
  a.out = out;
  a.lse2 = lse2;
  a.ot = ot;
  a.reqs = nullptr;
  a.counts = nullptr;
  a.flags = flags;
  a.pad_R = g.R;
  const int64_t items = (int64_t)g.B * g.nh * g.ntiles * g.nbmax_tot;
  if (items >= (1LL << 31)) return cudaErrorNotSupported;
  a.items = (int)items;
  const int BH = g.B * g.nh;
  CUtensorMap mq, mk, mv;
  if (!make_tmap_5d(&mq, q, D, g.G[2], g.G[1], g.G[0], BH, g.bx, g.by, g.bt) ||
      !make_tmap_5d(&mk, k, D, g.G[2], g.G[1], g.G[0], BH, g.bx, g.by, g.bt) ||
      !make_tmap_5d(&mv, v, D, g.G[2], g.G[1], g.G[0], BH, g.bx, g.by, g.bt))
    return cudaErrorInvalidValue;
  auto kern = sm103_fwd_kernel<D, OutT, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmem);
  if (e != cudaSuccess) return e;
  const int grid = (int)(a.items < num_sms() ? a.items : num_sms());
  kern<<<grid, kThreads, C::kSmem, st>>>(mq, mk, mv, a);
  return cudaGetLastError();
}

template <int D>
cudaError_t run_fwd_ragged(const ReqDesc* reqs, const int64_t* counts, int pad_R, cudaStream_t st) {
  using C = FwdCfg<D>;
  FwdArgs a;
  memset(&a, 0, sizeof(a));
  a.reqs = reqs;
  a.counts = counts;
  a.pad_R = pad_R;
  CUtensorMap dummy;
  memset(&dummy, 0, sizeof(dummy));
  auto kern = sm103_fwd_kernel<D, __nv_bfloat16, true>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmem);
  if (e != cudaSuccess) return e;
  kern<<<num_sms(), kThreads, C::kSmem, st>>>(dummy, dummy, dummy, a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sm103_fwd_ragged(const ReqDesc* reqs, const int64_t* counts, int d, int box_rows,
                                    cudaStream_t st) {
  if (d == 64) return launch_sm103_fwd64_ragged(reqs, counts, box_rows, st);
  if (d == 128) return run_fwd_ragged<128>(reqs, counts, box_rows, st);
  return cudaErrorNotSupported;
}

cudaError_t launch_sm103_fwd(const Geom& g, const __nv_bfloat16* q, const __nv_bfloat16* k, const __nv_bfloat16* v,
                             void* out, int out_dtype, float* lse2, float* ot, uint32_t flags, cudaStream_t st) {
  const bool bf = out_dtype == GATTN_BF16;
  if (g.d == 64) return launch_sm103_fwd64(g, q, k, v, out, out_dtype, lse2, ot, flags, st);
  if (g.d == 128)
    return bf ? run_fwd<128, __nv_bfloat16>(g, q, k, v, out, lse2, ot, flags, st)
              : run_fwd<128, float>(g, q, k, v, out, lse2, ot, flags, st);
  return cudaErrorNotSupported;
}

}  // namespace gattn
