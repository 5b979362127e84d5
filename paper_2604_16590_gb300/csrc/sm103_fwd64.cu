// sm103_fwd64.cu -- BF16 tensor-core forward of STORM-GPA tile attention for
// head size d = 64 on GB300 (sm_103a): two query boxes per work item, each
// with its own scores, probabilities and output in tensor memory.
//
// Per extended tile t (arXiv 2604.16590, Sec. III-C) and pair of 128-query
// boxes (A, B) of the tile, the CTA streams the tile's 128-key boxes once for
// both query boxes (flash-style online softmax, the FlashAttention of
// Sec. III-D Level 5):
//   S_x  = Q_x K_j^T                    tcgen05, A = Q_x, B = K_j (both shared memory)
//   m_x  = max(m_x, rowmax(s S_x))      log2 domain, lazily moved (threshold 8)
//   P_x  = exp2(s S_x log2e - m_x)      BF16 pairs -> TMEM
//   O_x += P_x V_j                      tcgen05, A = P_x from TMEM, B = V_j (MN-major)
// A softmax thread reads its row's 128 scores into registers at once and
// releases S_x, so S_x(j+1) is computed while the exponentials of box j run;
// P_x(j) waits only for P V_x(j-1).  With two boxes in flight the tensor pipe
// and the exp unit are busy at the same time.  The epilogue writes O / l for
// rows covered by one tile straight to the output and parks multiply-covered
// rows (FP32) for the deterministic Hann merge, and stores the row log-sum-exp.
//
// Warp roles (384 threads = three warpgroups, one CTA per SM, persistent over
// work items (batch*head, tile, box pair)):
//   warp 0        TMA producer (Q_A, Q_B once per item; K_j, V_j through a ring)
//   warp 1        TMEM allocator + issuer of the S products
//   warp 2        issuer of the P V products (a thread's mbarrier waits stall
//                 until its own issued MMAs drain, so the two product streams
//                 come from two threads)
//   warp 3        key-mask writer: for a key block with padding rows or rows
//                 outside the tile, the bias row of its stage (see below)
//   warps 4..7    softmax + epilogue of box A, warps 8..11 of box B: one warp
//                 per TMEM lane quadrant, one thread per query row owning all
//                 128 key columns (no cross-warp reduction)
// Registers: the first warpgroup gives up registers (setmaxnreg) so that the
// softmax threads hold a whole row of scores: 128 x 72 + 2 x 128 x 216 =
// 384 x 168, the launch's allocation.
// TMEM (512 columns): S_x at 128 x, P_x at 256 + 64 x, O_x at 384 + 64 x.
//
// Key masking without a masked softmax: a key block that contains padding rows
// or keys outside the tile gets one more K = 16 step in its S product, a
// column of ones times the block's bias row (0 or -1e30 per key), so the
// masked scores arrive as -1e30 and their probabilities are exactly 0.  The
// softmax threads then run one branch-free form for every block (a second,
// masked form of the exponential loop measured 19 % slower even where it was
// never taken).
//
// Ragged mode (the serving engine): the work items of all active requests in
// one launch; each item resolves through the request table in device memory
// (tensor map over the request's state z = Q = K = V, geometry, outputs), and
// the producer acquires a request's tensor map before its first load from it.
#include <string.h>

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
constexpr int kSoft0 = 4;           // first softmax warp
constexpr int kThreadsF = 384;
constexpr uint32_t kRegsLow = 72, kRegsHigh = 216;  // 128 x 72 + 256 x 216 = 384 x 168
constexpr float kRescaleLog2 = 8.f;

struct Cfg {
  // two Q buffers (items alternate): buffer b holds Q_A at kQ + 2 b kBox, Q_B after it
  static constexpr int kQ = 0;
  static constexpr int kK = 4 * kBox;
  static constexpr int kV = kK + kStages * kBox;
  // Key-mask extension operands, K-major without swizzle (128 rows x 16 B,
  // then 2 KB of zeros for K-columns 8..15): the A operand has 1 in K-column 0
  // of every row; stage s of the B operand holds the key block's bias
  // (0 for a key of the tile, -1e30 for a padding row or a key outside it).
  static constexpr int kOnes = kV + kStages * kBox;
  static constexpr int kBias = kOnes + 4096;
  static constexpr int kBar = kBias + kStages * 4096;
  // q_full[2], q_empty[2], k_full[S], k_empty[S], v_full[S], v_empty[S],
  // per box: s_full, s_empty, p_full, p_empty, o_full, o_empty; drain[2], never
  static constexpr int kNumBars = 4 + 4 * kStages + 2 * 6 + 3;
  static constexpr int kMisc = kBar + kNumBars * 8;
  static constexpr int kSmem = kMisc + 16 + 1024;
};
__device__ __forceinline__ uint32_t col_s(int x) { return 128u * x; }
__device__ __forceinline__ uint32_t col_p(int x) { return 256u + 64u * x; }
__device__ __forceinline__ uint32_t col_o(int x) { return 384u + 64u * x; }

struct Fwd64Args {
  Geom g;
  void* out;
  float* lse2;
  float* ot;
  int items;  // B*nh * ntiles * box pairs
  uint32_t flags;
  int pad_R;  // box rows of every geometry of the launch (rows pad_R..127 of each block are zeroed once)
  // ragged mode (serving): per-request descriptors and device-side counts
  const ReqDesc* reqs;
  const int64_t* counts;
};

// One work item: a (batch*head, tile, pair of query boxes) of a geometry.
struct Item {
  const Geom* g;
  const CUtensorMap* tq;
  const CUtensorMap* tk;
  const CUtensorMap* tv;
  void* out;
  float* lse2;  // may be null (no backward)
  float* ot;
  int bh, tile, pair;
  int req;  // request index (ragged mode), else -1
};

__host__ __device__ __forceinline__ int box_pairs(const Geom& g) { return (g.nbmax_tot + 1) / 2; }

// Returns false (after recording GATTN_ERR_DEVICE_BOUNDS) if a ragged work item
// does not decode to a valid (request, head, tile, pair); every role decodes
// the same item identically, so all of them skip it together.
template <bool RAGGED>
__device__ __forceinline__ bool resolve(const Fwd64Args& a, const CUtensorMap* tq, const CUtensorMap* tk,
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
  const int np = box_pairs(g);
  it.pair = w % np;
  const int r = w / np;
  it.tile = r % g.ntiles;
  it.bh = r / g.ntiles;
  it.req = req;
  if (RAGGED && (it.bh >= g.B * g.nh || g.d != kD || g.R != a.pad_R)) {
    set_status(kStatusBounds);
    return false;
  }
  return true;
}

// running max of 32 scores into 4 partial maxima (3-input max)
__device__ __forceinline__ void chunk_max(const uint32_t* r, float (&mx)[4]) {
#pragma unroll
  for (int i = 0; i < 32; i += 2)
    mx[(i >> 1) & 3] = fmax3(mx[(i >> 1) & 3], __uint_as_float(r[i]), __uint_as_float(r[i + 1]));
}

// exp2 of 32 scores -> 16 BF16 pairs, row sum in packed FP32 pairs
__device__ __forceinline__ void exp_chunk(const uint32_t* r, uint64_t s2, uint64_t nm2, uint64_t (&acc)[4],
                                          uint32_t (&pk)[16]) {
#pragma unroll
  for (int i = 0; i < 32; i += 2) {
    float a0, a1;
    f2unpack(ffma2(u2pack(r[i], r[i + 1]), s2, nm2), a0, a1);
    const float p0 = ex2(a0), p1 = ex2(a1);
    acc[(i >> 1) & 3] = fadd2(acc[(i >> 1) & 3], f2pack(p0, p1));
    pk[i >> 1] = pack_bf16(p0, p1);
  }
}

// multiply this thread's 64 O columns by f
__device__ __forceinline__ void rescale_o(uint32_t tO, float f) {
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
}

template <typename OutT, bool RAGGED>
__global__ void __launch_bounds__(kThreadsF, 1)
    fwd64_kernel(const __grid_constant__ CUtensorMap tq, const __grid_constant__ CUtensorMap tk,
                 const __grid_constant__ CUtensorMap tv, const Fwd64Args a) {
  using C = Cfg;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::kBar);
  uint64_t* q_full = bars;       // [2]
  uint64_t* q_empty = bars + 2;  // [2]
  uint64_t* k_full = bars + 4;
  uint64_t* k_empty = k_full + kStages;
  uint64_t* v_full = k_empty + kStages;
  uint64_t* v_empty = v_full + kStages;
  uint64_t* boxbar = v_empty + kStages;  // [x * 6 + i]
  auto s_full = [&](int x) { return boxbar + 6 * x; };
  auto s_empty = [&](int x) { return boxbar + 6 * x + 1; };
  auto p_full = [&](int x) { return boxbar + 6 * x + 2; };
  auto p_empty = [&](int x) { return boxbar + 6 * x + 3; };
  auto o_full = [&](int x) { return boxbar + 6 * x + 4; };
  auto o_empty = [&](int x) { return boxbar + 6 * x + 5; };
  uint64_t* drain = boxbar + 12;  // [2]
  uint64_t* never = drain + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + C::kMisc);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + C::kMisc + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  zero_pad_rows(smem, 4 + 2 * kStages, a.pad_R);  // both Q buffers, the K and V rings
  // the ones operand (1 in K-column 0 of each of its 128 rows) and the zero
  // K-columns 8..15 of it and of every bias stage
  for (int r = threadIdx.x; r < (1 + kStages) * 256; r += kThreadsF) {
    const int blk = r >> 8, rr = r & 255;
    const uint4 v = (blk == 0 && rr < 128) ? make_uint4(0x00003F80u, 0u, 0u, 0u) : make_uint4(0u, 0u, 0u, 0u);
    if (blk == 0 || rr >= 128) *reinterpret_cast<uint4*>(smem + C::kOnes + blk * 4096 + rr * 16) = v;
  }
  fence_proxy_async_smem();
  if (threadIdx.x == 0) {
    for (int b = 0; b < 2; ++b) {
      mbar_init(q_full + b, 1);
      mbar_init(q_empty + b, 1);
    }
    for (int s = 0; s < kStages; ++s) {
      mbar_init(k_full + s, 2);  // the K load (producer) and the stage's bias row (mask writer)
      mbar_init(k_empty + s, 1);
      mbar_init(v_full + s, 1);
      mbar_init(v_empty + s, 1);
    }
    for (int x = 0; x < 2; ++x) {
      mbar_init(s_full(x), 1);
      mbar_init(s_empty(x), 4);
      mbar_init(p_full(x), 4);
      mbar_init(p_empty(x), 1);
      mbar_init(o_full(x), 1);
      mbar_init(o_empty(x), 4);
    }
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
    tmem_alloc(tmem_slot, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int n_items = RAGGED ? (int)a.counts[1] : a.items;

  if (warp < kSoft0) {
    setmaxnreg_dec<kRegsLow>();
    if (warp == 0 && lane == 0) {
      // ---------------------------------------------------------- TMA producer
      uint32_t G = 0, W = 0;
      uint32_t q_arm = 0, q_par = 0, k_arm = 0, k_par = 0, v_arm = 0, v_par = 0;
      int last_req = -1;
      bool ok = true;
      for (int w = blockIdx.x; w < n_items && ok; w += gridDim.x) {
        Item it;
        if (!resolve<RAGGED>(a, &tq, &tk, &tv, w, it)) continue;
        const Geom& g = *it.g;
        const int bh = it.bh;
        TileBlocks tbk;
        tile_blocks(g, it.tile, tbk);
        const int qa = 2 * it.pair;
        if (qa >= tbk.NB) continue;
        const int nact = qa + 1 < tbk.NB ? 2 : 1;
        if (RAGGED && it.req != last_req) {
          tmap_acquire(it.tq);  // this launch's descriptor table may hold a new map here
          last_req = it.req;
        }
        // Q of this item goes to buffer W & 1, so it loads while the previous
        // item's score products still read the other buffer
        const uint32_t qb = W & 1, qn = (W >> 1) & 1;
        if (!(ok = WAIT(q_empty + qb, qn ^ 1))) break;
        mbar_arrive_expect_tx(q_full + qb, nact * g.R * 128);
        q_arm |= 1u << qb;
        q_par = (q_par & ~(1u << qb)) | (qn << qb);
        for (int x = 0; x < nact; ++x) {
          int o[3];
          block_origin(g, tbk, qa + x, o);
          tma_load_5d(smem + C::kQ + (2 * qb + x) * kBox, it.tq, q_full + qb, 0, tbk.tb.lo[2] + o[2],
                      tbk.tb.lo[1] + o[1], tbk.tb.lo[0] + o[0], bh);
        }
        int jt = 0, jy = 0, jx = 0;
        for (int j = 0; j < tbk.NB; ++j, ++G) {
          const uint32_t st = G % kStages, n = G / kStages;
          const int c1 = tbk.tb.lo[2] + (jx * g.bx), c2 = tbk.tb.lo[1] + (jy * g.by), c3 = tbk.tb.lo[0] + (jt * g.bt);
          if (++jx == tbk.nb[2]) {
            jx = 0;
            if (++jy == tbk.nb[1]) {
              jy = 0;
              ++jt;
            }
          }
          if (!(ok = WAIT(k_empty + st, (n & 1) ^ 1))) break;
          mbar_arrive_expect_tx(k_full + st, g.R * 128);
          k_arm |= 1u << st;
          k_par = (k_par & ~(1u << st)) | ((n & 1) << st);
          tma_load_5d(smem + C::kK + st * kBox, it.tk, k_full + st, 0, c1, c2, c3, bh);
          if (!(ok = WAIT(v_empty + st, (n & 1) ^ 1))) break;
          mbar_arrive_expect_tx(v_full + st, g.R * 128);
          v_arm |= 1u << st;
          v_par = (v_par & ~(1u << st)) | ((n & 1) << st);
          tma_load_5d(smem + C::kV + st * kBox, it.tv, v_full + st, 0, c1, c2, c3, bh);
        }
        ++W;
      }
      if (!ok) {
        // let every load this thread issued land before the CTA exits
        for (int b = 0; b < 2; ++b)
          if (q_arm & (1u << b)) mbar_wait<set_status_f64>(q_full + b, (q_par >> b) & 1, abort_flag, false);
        for (int s = 0; s < kStages; ++s) {
          if (k_arm & (1u << s)) mbar_wait<set_status_f64>(k_full + s, (k_par >> s) & 1, abort_flag, false);
          if (v_arm & (1u << s)) mbar_wait<set_status_f64>(v_full + s, (v_par >> s) & 1, abort_flag, false);
        }
      }
    } else if (warp == 1 && lane == 0) {
      // ---------------------------------------------------------- issuer of S_x = Q_x K^T
      constexpr uint32_t idS = idesc_bf16(128, 128, 0);
      const uint64_t dQ0 = sw128_desc(smem_u32(smem + C::kQ), 16, 1024);
      const uint64_t dK0 = sw128_desc(smem_u32(smem + C::kK), 16, 1024);
      const uint64_t dOnes = noswz_desc(smem_u32(smem + C::kOnes), 2048, 128);
      const uint64_t dBias0 = noswz_desc(smem_u32(smem + C::kBias), 2048, 128);
      uint32_t G = 0, W = 0, GX0 = 0, GX1 = 0;
      bool ok = true;
      if (a.flags & GATTN_FLAG_TEST_STALL)  // failure-detection hook: a wait that cannot complete
        ok = mbar_wait<set_status_f64>(never, 0, abort_flag, true, 20000000ull);
      for (int w = blockIdx.x; w < n_items && ok; w += gridDim.x) {
        Item it;
        if (!resolve<RAGGED>(a, &tq, &tk, &tv, w, it)) continue;
        const Geom& g = *it.g;
        TileBlocks tbk;
        tile_blocks(g, it.tile, tbk);
        const int qa = 2 * it.pair;
        if (qa >= tbk.NB) continue;
        const int nact = qa + 1 < tbk.NB ? 2 : 1;
        const uint32_t qb = W & 1;
        if (!(ok = WAIT(q_full + qb, (W >> 1) & 1))) break;  // Q_A, Q_B of this item in shared memory
        const bool all_full = tile_all_full(g, tbk);
        BlockWalk bw;
        for (int j = 0; j < tbk.NB && ok; ++j, ++G, bw.next(tbk)) {
          const uint32_t st = G % kStages;
          // a masked block's bias row was filled by the mask writer
          const bool masked = !all_full && !bw.full(g, tbk);
          if (!(ok = WAIT(k_full + st, (G / kStages) & 1))) break;
          const uint64_t dk = dmove(dK0, st * kBox), db = dmove(dBias0, st * 4096);
#pragma unroll
          for (int x = 0; x < 2; ++x) {
            if (x >= nact) break;
            uint32_t& gx = x == 0 ? GX0 : GX1;
            // S_x is free once the softmax threads have read the previous scores
            if (gx > 0 && !(ok = WAIT(s_empty(x), (gx - 1) & 1))) break;
            tc_fence_after();
            const uint64_t dq = dmove(dQ0, (2 * qb + x) * kBox);
#pragma unroll
            for (int ks = 0; ks < kD / 16; ++ks)
              umma_bf16(tmem + col_s(x), dmove(dq, ks * 32), dmove(dk, ks * 32), idS, ks > 0);
            if (masked) umma_bf16(tmem + col_s(x), dOnes, db, idS, 1u);  // + bias of each key column
            umma_commit(s_full(x));
            ++gx;
          }
          if (!ok) break;
          umma_commit(k_empty + st);
        }
        if (!ok) break;
        umma_commit(q_empty + qb);  // Q_A, Q_B of this item no longer read
        ++W;
      }
      umma_commit(drain);
      mbar_wait<set_status_f64>(drain, 0, abort_flag, false);
    } else if (warp == 2 && lane == 0) {
      // ---------------------------------------------------------- issuer of O_x += P_x V
      constexpr uint32_t idO = idesc_bf16(128, kD, 1);
      const uint64_t dV0 = sw128_desc(smem_u32(smem + C::kV), 16384, 1024);  // MN-major (K = keys)
      uint32_t G = 0, GX0 = 0, GX1 = 0, WX0 = 0, WX1 = 0;
      bool ok = true;
      for (int w = blockIdx.x; w < n_items && ok; w += gridDim.x) {
        Item it;
        if (!resolve<RAGGED>(a, &tq, &tk, &tv, w, it)) continue;
        TileBlocks tbk;
        tile_blocks(*it.g, it.tile, tbk);
        const int qa = 2 * it.pair;
        if (qa >= tbk.NB) continue;
        const int nact = qa + 1 < tbk.NB ? 2 : 1;
        for (int j = 0; j < tbk.NB && ok; ++j, ++G) {
          const uint32_t st = G % kStages;
          if (!(ok = WAIT(v_full + st, (G / kStages) & 1))) break;
          const uint64_t dv = dmove(dV0, st * kBox);
#pragma unroll
          for (int x = 0; x < 2; ++x) {
            if (x >= nact) break;
            uint32_t& gx = x == 0 ? GX0 : GX1;
            const uint32_t wx = x == 0 ? WX0 : WX1;
            if (!(ok = WAIT(p_full(x), gx & 1))) break;
            if (j == 0 && !(ok = WAIT(o_empty(x), (wx & 1) ^ 1))) break;
            tc_fence_after();
#pragma unroll
            for (int ks = 0; ks < 8; ++ks)
              umma_bf16_ts(tmem + col_o(x), tmem + col_p(x) + ks * 8, dmove(dv, ks * 2048), idO,
                           (j > 0 || ks > 0) ? 1u : 0u);
            umma_commit(p_empty(x));
            if (j == tbk.NB - 1) umma_commit(o_full(x));
            ++gx;
          }
          if (!ok) break;
          umma_commit(v_empty + st);
        }
        ++WX0;
        if (nact > 1) ++WX1;
      }
      umma_commit(drain + 1);
      mbar_wait<set_status_f64>(drain + 1, 0, abort_flag, false);
    } else if (warp == 3) {
      // ---------------------------------------------------------- key-mask writer
      // One arrival on k_full per stage use (the stage's second arrival), in
      // the producer's order.  It first waits until the stage is free again,
      // which also guarantees that the previous phase of k_full completed.
      const uint32_t neg = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(-1e30f));
      uint32_t G = 0;
      bool ok = true;
      for (int w = blockIdx.x; w < n_items && ok; w += gridDim.x) {
        Item it;
        if (!resolve<RAGGED>(a, &tq, &tk, &tv, w, it)) continue;
        const Geom& g = *it.g;
        TileBlocks tbk;
        tile_blocks(g, it.tile, tbk);
        if (2 * it.pair >= tbk.NB) continue;
        for (int j = 0; j < tbk.NB; ++j, ++G) {
          const uint32_t st = G % kStages, n = G / kStages;
          int ko[3];
          block_origin(g, tbk, j, ko);
          if (lane == 0) ok = WAIT(k_empty + st, (n & 1) ^ 1);
          ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
          if (!ok) break;
          if (!block_full(g, tbk, ko)) {
            for (int r = lane; r < 128; r += 32) {
              int kl[3];
              block_row(g, ko, r, kl);
              *reinterpret_cast<uint4*>(smem + C::kBias + st * 4096 + r * 16) =
                  make_uint4(inside(tbk, kl) ? 0u : neg, 0u, 0u, 0u);
            }
            fence_proxy_async_smem();  // the tensor core reads what these lanes wrote
          }
          __syncwarp();
          if (lane == 0) mbar_arrive(k_full + st);
        }
      }
    }
  } else {
    setmaxnreg_inc<kRegsHigh>();
    // ------------------------------------------------------------ softmax + epilogue of box x
    const int x = (warp - kSoft0) >> 2;
    const int quad = warp & 3;
    const int row = quad * 32 + lane;  // TMEM lane = query row of the box
    const uint32_t tl = tmem + ((uint32_t)(quad * 32) << 16);
    const uint32_t tS = tl + col_s(x), tP = tl + col_p(x), tO = tl + col_o(x);
    uint32_t GX = 0, WX = 0;
    bool ok = true;
    for (int w = blockIdx.x; w < n_items && ok; w += gridDim.x) {
      Item it;
      if (!resolve<RAGGED>(a, &tq, &tk, &tv, w, it)) continue;
      const Geom& g = *it.g;
      const int bh = it.bh, tile = it.tile;
      const float sl2 = g.scale_log2;
      const uint64_t s2 = f2pack(sl2, sl2);
      TileBlocks tbk;
      tile_blocks(g, tile, tbk);
      const int qa = 2 * it.pair;
      if (qa + x >= tbk.NB) continue;
      const int qb = qa + x;
      int qo[3], ql[3];
      block_origin(g, tbk, qb, qo);
      block_row(g, qo, row, ql);
      const bool qvalid = inside(tbk, ql);
      float m = -INFINITY, l = 0.f, lc = 0.f;  // lc: Kahan compensation of the row sum l
      for (int j = 0; j < tbk.NB; ++j, ++GX) {
        if (!(ok = WAIT(s_full(x), GX & 1))) break;
        tc_fence_after();
        // the row's 128 scores into registers, then S_x is released
        uint32_t s0[32], s1[32], s2r[32], s3[32];
        tmem_ld32(tS, s0);
        tmem_ld32(tS + 32, s1);
        tmem_ld32(tS + 64, s2r);
        tmem_ld32(tS + 96, s3);
        tmem_wait_ld(s0);
        tmem_wait_ld(s1);
        tmem_wait_ld(s2r);
        tmem_wait_ld(s3);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(s_empty(x));
        float mx[4] = {-INFINITY, -INFINITY, -INFINITY, -INFINITY};
        // masked keys carry -1e30 from the extension step: no mask here
        chunk_max(s0, mx);
        chunk_max(s1, mx);
        chunk_max(s2r, mx);
        chunk_max(s3, mx);
        const float mblk = fmaxf(fmaxf(mx[0], mx[1]), fmaxf(mx[2], mx[3])) * sl2;
        float f = 1.f;
        bool any_grow = false;
        if (j == 0) {
          m = mblk;
        } else {
          const bool grow = mblk > m + kRescaleLog2;
          any_grow = __any_sync(0xffffffffu, grow);
          if (grow) {
            f = ex2(m - mblk);
            m = mblk;
          }
        }
        // the exponentials depend only on the scores and the new reference max:
        // they are computed into registers before P_x is known to be free
        const uint64_t nm2 = f2pack(-m, -m);
        uint64_t acc[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[i] = f2pack(0.f, 0.f);
        uint32_t pk0[16], pk1[16], pk2[16], pk3[16];
        exp_chunk(s0, s2, nm2, acc, pk0);
        exp_chunk(s1, s2, nm2, acc, pk1);
        exp_chunk(s2r, s2, nm2, acc, pk2);
        exp_chunk(s3, s2, nm2, acc, pk3);
        float lsum = 0.f;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          float u, v;
          f2unpack(acc[i], u, v);
          lsum += u + v;
        }
        // P_x and O_x are free once the previous P V of this box completed
        if (GX > 0 && !(ok = WAIT(p_empty(x), (GX - 1) & 1))) break;
        tc_fence_after();
        if (any_grow) {
          rescale_o(tO, f);
          l *= f;
          lc *= f;
        }
        {  // compensated sum over the tile's key blocks
          const float y = lsum - lc;
          const float t = l + y;
          lc = (t - l) - y;
          l = t;
        }
        tmem_st16(tP, pk0);
        tmem_st16(tP + 16, pk1);
        tmem_st16(tP + 32, pk2);
        tmem_st16(tP + 48, pk3);
        tmem_wait_st();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(p_full(x));
      }
      if (!ok) break;
      // ---- epilogue: wait for the last P V, O / l
      if (!(ok = WAIT(o_full(x), WX & 1))) break;
      tc_fence_after();
      ++WX;
      const float inv = 1.f / l;
      const int64_t slot = tile_slot0(g, bh, tile) + qb * 128 + row;
      if (qvalid && it.lse2) it.lse2[slot] = m + __log2f(l);
      const int p[3] = {tbk.tb.lo[0] + ql[0], tbk.tb.lo[1] + ql[1], tbk.tb.lo[2] + ql[2]};
      const int64_t tok = qvalid ? ((int64_t)p[0] * g.G[1] + p[1]) * g.G[2] + p[2] : 0;
      const bool single = qvalid && single_cover(g, p);
      OutT* dst_out = static_cast<OutT*>(it.out) + ((int64_t)bh * g.N + tok) * kD;
      float* dst_scr = it.ot + slot * kD;
      // the whole O row into registers, then O_x is released at once: the next
      // item's first P V may overwrite it while this row is scaled and stored
      uint32_t r0[32], r1[32];
      tmem_ld32(tO, r0);
      tmem_ld32(tO + 32, r1);
      tmem_wait_ld(r0);
      tmem_wait_ld(r1);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(o_empty(x));
      if (qvalid) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const uint32_t* r = c == 0 ? r0 : r1;
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
  memset(&a, 0, sizeof(a));
  a.g = g;
  a.out = out;
  a.lse2 = lse2;
  a.ot = ot;
  a.flags = flags;
  a.pad_R = g.R;
  const int64_t items = (int64_t)g.B * g.nh * g.ntiles * box_pairs(g);
  if (items >= (1LL << 31)) return cudaErrorNotSupported;
  a.items = (int)items;
  const int BH = g.B * g.nh;
  CUtensorMap mq, mk, mv;
  if (!make_tmap_5d(&mq, q, kD, g.G[2], g.G[1], g.G[0], BH, g.bx, g.by, g.bt) ||
      !make_tmap_5d(&mk, k, kD, g.G[2], g.G[1], g.G[0], BH, g.bx, g.by, g.bt) ||
      !make_tmap_5d(&mv, v, kD, g.G[2], g.G[1], g.G[0], BH, g.bx, g.by, g.bt))
    return cudaErrorInvalidValue;
  auto kern = fwd64_kernel<OutT, false>;
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

int fwd64_ragged_items(const Geom& g) { return g.nh * g.ntiles * box_pairs(g); }

cudaError_t launch_sm103_fwd64_ragged(const ReqDesc* reqs, const int64_t* counts, int box_rows, cudaStream_t st) {
  Fwd64Args a;
  memset(&a, 0, sizeof(a));
  a.reqs = reqs;
  a.counts = counts;
  a.pad_R = box_rows;
  CUtensorMap dummy;
  memset(&dummy, 0, sizeof(dummy));
  auto kern = fwd64_kernel<__nv_bfloat16, true>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::kSmem);
  if (e != cudaSuccess) return e;
  kern<<<num_sms(), kThreadsF, Cfg::kSmem, st>>>(dummy, dummy, dummy, a);
  return cudaGetLastError();
}

}  // namespace gattn
