// serve.cu -- continuous-batching serving engine for diffusion posterior
// sampling with STORM-GPA (arXiv 2604.16590): every request runs `steps`
// denoising steps z <- z + c (GPA(z, z, z) - z) on its own token grid, the
// Hann-weighted merge being the per-step propagation of Sec. III-C.
//
// Host side (C++): FIFO admission under a slot limit and an HBM budget,
// per-request device memory from a stream-ordered pool kept across steps, one
// descriptor table per engine iteration, retirement that keeps the final state
// in device memory until its client takes it (at once, or on a copy stream
// while the engine keeps stepping) or releases it, latency statistics.  Device
// side: one persistent ragged tcgen05 attention launch over the work items of
// all active requests (sm103_fwd64.cu / sm103_fwd.cu, RAGGED mode) and one
// merge-and-update launch over all their (head, token) rows (below), both
// captured once in a CUDA graph that reads the active set from device memory.
#include <algorithm>
#include <chrono>
#include <deque>
#include <unordered_map>
#include <vector>

#include "internal.cuh"
#include "merge_common.cuh"
#include "sm103_common.cuh"

GATTN_DEFINE_STATUS(serve)

namespace gattn {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ int find_request(const ReqDesc* reqs, int n, int64_t row) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (reqs[mid].tok0 <= row) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// For every (request, head, token) row and 4-column group: the GPA output a
// (the tile kernel's output for single-cover tokens, else the Hann-weighted
// merge of the per-tile outputs, ascending tile order) and the state update
// z <- z + c (a - z), rounded to BF16.
__global__ void __launch_bounds__(kThreads) serve_update_kernel(const ReqDesc* __restrict__ reqs,
                                                                const int64_t* __restrict__ counts, int d, float c) {
  const int nreq = (int)counts[0];
  const int64_t rows = counts[2];
  const int F4 = d / 4;
  const int64_t total = rows * F4;
  for (int64_t idx = (int64_t)blockIdx.x * kThreads + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * kThreads) {
    const int f = (int)(idx % F4);
    const int64_t grow = idx / F4;
    const int r = find_request(reqs, nreq, grow);
    const ReqDesc& rq = reqs[r];
    const Geom& g = rq.g;
    const int64_t local = grow - rq.tok0;  // head * N + token
    if (nreq < 1 || local < 0 || local >= (int64_t)g.nh * g.N) {
      set_status(kStatusBounds);
      continue;
    }
    const int h = (int)(local / g.N);
    const int64_t i = local % g.N;
    int p[3], k0[3], k1[3];
    token_pos(g, i, p);
    bool multi = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      cover_dim(g, a, p[a], k0[a], k1[a]);
      multi = multi || (k1[a] > k0[a]);
    }
    float4 att;
    if (!multi) {
      att = load4<__nv_bfloat16>(static_cast<const __nv_bfloat16*>(rq.out) + local * d + 4 * f);
    } else {
      float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
      float wsum = 0.f;
      int k[3];
      for (k[0] = k0[0]; k[0] <= k1[0]; ++k[0])
        for (k[1] = k0[1]; k[1] <= k1[1]; ++k[1])
          for (k[2] = k0[2]; k[2] <= k1[2]; ++k[2]) {
            int e[3], l[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
              int lo = k[a] * g.c[a] - g.h[a];
              int hi = (k[a] + 1) * g.c[a] + g.h[a];
              lo = lo < 0 ? 0 : lo;
              hi = hi > g.G[a] ? g.G[a] : hi;
              e[a] = hi - lo;
              l[a] = p[a] - lo;
            }
            const int tile = (k[0] * g.n[1] + k[1]) * g.n[2] + k[2];
            const float w = tile_weight(g, p, k);
            const float4 o = __ldg(reinterpret_cast<const float4*>(rq.ot + slot_of(g, h, tile, e, l) * d) + f);
            acc.x = fmaf(w, o.x, acc.x);
            acc.y = fmaf(w, o.y, acc.y);
            acc.z = fmaf(w, o.z, acc.z);
            acc.w = fmaf(w, o.w, acc.w);
            wsum += w;
          }
      const float inv = 1.f / wsum;
      att = make_float4(acc.x * inv, acc.y * inv, acc.z * inv, acc.w * inv);
    }
    __nv_bfloat16* zp = rq.z + local * d + 4 * f;
    const float4 z = load4<__nv_bfloat16>(zp);
    store4<__nv_bfloat16>(zp, make_float4(fmaf(c, att.x - z.x, z.x), fmaf(c, att.y - z.y, z.y),
                                          fmaf(c, att.z - z.z, z.z), fmaf(c, att.w - z.w, z.w)));
  }
}

// The same update, a warp per 32 consecutive rows, organised like the forward
// merge of merge.cu but with a quarter-warp per row: each lane resolves its
// row's request, head and token and lists what the row needs, in order -- its
// covering tiles' FP32 rows with their window weights (or, for a token covered
// by one tile, the tile kernel's BF16 output row with weight 1), then its BF16
// state row, whose entry carries 1 / sum of weights -- into one of four
// shared-memory lists (group_offset): quarter-warp q works through the rows of
// the tokens of lanes q, q + 4, ..., R rows at a time with all R loads issued
// first, lane f of the quarter holding columns [8 f, 8 f + 8) (32 bytes of an
// FP32 row, 16 of a BF16 row; and [8 f + 64, 8 f + 72) at d = 128, U = 2).
// Eight lanes per row instead of sixteen halve the list reads, address and
// flag work per byte moved, which bound the half-warp form.  At a state row it
// forms a = (weighted sum) / (sum of weights) and writes z + c (a - z) back.
// The window table is built from the first request's geometry; a row whose
// request differs in core, halo, window or tiled dimensions evaluates its
// window directly.
template <int MAXC, int U>
__global__ void __launch_bounds__(kThreads, 2)
    serve_update_warp_kernel(const ReqDesc* __restrict__ reqs, const int64_t* __restrict__ counts, int d, float c) {
  constexpr int R = 4 / U;
  constexpr int W = kThreads / 32;
  constexpr int NE = MAXC + 1;  // rows listed per token
  __shared__ float win[kWinMax];
  __shared__ RowRef rows[W][4][8 * NE];
  const int nreq = (int)counts[0];
  if (nreq < 1) return;  // uniform over the grid: no request, no table
  const int64_t nrows = counts[2];
  const Geom& g0 = reqs[0].g;
  const WinTable tbl = build_win_table(g0, win);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int f8 = lane & 7;
  const int F8 = d / 8;  // 8-column units of a row: 4, 8 or 16
  const int64_t stride = (int64_t)gridDim.x * W * 32;
  const RowRef* list = rows[wid][lane >> 3];
  for (int64_t base = ((int64_t)blockIdx.x * W + wid) * 32; base < nrows; base += stride) {
    const int64_t idx = base + lane;
    int r = -1, n = 0;
    int64_t local = 0;
    int64_t slot[MAXC];
    float w[MAXC];
    float wsum = 0.f;
    if (idx < nrows) {
      r = find_request(reqs, nreq, idx);
      const Geom& g = reqs[r].g;
      local = idx - reqs[r].tok0;  // head * N + token
      if (local < 0 || local >= (int64_t)g.nh * g.N) {
        set_status(kStatusBounds);
        r = -1;
      } else {
        bool same = g.window == g0.window;
#pragma unroll
        for (int a = 0; a < 3; ++a) same = same && g.c[a] == g0.c[a] && g.h[a] == g0.h[a] && g.tiled[a] == g0.tiled[a];
        WinTable t = tbl;
        t.direct = t.direct || !same;
        n = token_covers(g, t, (int)(local / g.N), local % g.N, slot, w);
        if (n > MAXC) {  // the host chose MAXC from the largest cover count
          set_status(kStatusBounds);
          r = -1;
          n = 0;
        }
#pragma unroll
        for (int k = 0; k < MAXC; ++k)
          if (k < n) wsum += w[k];
      }
    }
    const int cnt = r < 0 ? 0 : n == 0 ? 2 : n + 1;
    int len;
    RowRef* mine = rows[wid][lane & 3] + group_offset(cnt, lane, len);
    if (r >= 0) {
      const ReqDesc& rq = reqs[r];
      RowRef e;
      if (n == 0) {
        e.p = reinterpret_cast<const char*>(static_cast<const __nv_bfloat16*>(rq.out) + local * d) + 1;
        e.w = 1.f;
        e.flags = lane | kRowBf16;
        mine[0] = e;
      }
#pragma unroll
      for (int k = 0; k < MAXC; ++k)
        if (k < n) {
          e.p = rq.ot + slot[k] * d;
          e.w = w[k];
          e.flags = lane;
          mine[k] = e;
        }
      e.p = reinterpret_cast<const char*>(rq.z + local * d) + 1;
      e.w = n == 0 ? 1.f : 1.f / wsum;
      e.flags = lane | kRowBf16 | kRowState;
      mine[cnt - 1] = e;
    }
    __syncwarp();
    int lmax = max(len, __shfl_xor_sync(0xffffffffu, len, 8));
    lmax = max(lmax, __shfl_xor_sync(0xffffffffu, lmax, 16));
    float acc[U][8];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int e = 0; e < 8; ++e) acc[u][e] = 0.f;
#pragma unroll 1
    for (int e0 = 0; e0 < lmax; e0 += R) {
      const int nv = len - e0;  // rows of this quarter's list from e0 on
      uint4 v[R][U][2];
#pragma unroll
      for (int j = 0; j < R; ++j)
        if (j < nv) {
          const uint64_t a = row_addr(list + e0 + j);
          const bool bf = a & 1;  // BF16 rows are listed with the low address bit set
          const void* p = reinterpret_cast<const void*>(a & ~(uint64_t)1);
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int col8 = f8 + 8 * u;
            if (col8 >= F8) continue;
            if (bf) {
              v[j][u][0] = __ldg(static_cast<const uint4*>(p) + col8);
            } else {
              v[j][u][0] = __ldg(static_cast<const uint4*>(p) + 2 * col8);
              v[j][u][1] = __ldg(static_cast<const uint4*>(p) + 2 * col8 + 1);
            }
          }
        }
#pragma unroll
      for (int j = 0; j < R; ++j) {
        if (j >= nv) break;
        float wr;
        int fl;
        row_weight_flags(list + e0 + j, wr, fl);
        __nv_bfloat16* zrow =
            (fl & kRowState) ? reinterpret_cast<__nv_bfloat16*>(row_addr(list + e0 + j) & ~(uint64_t)1) : nullptr;
#pragma unroll
        for (int u = 0; u < U; ++u) {
          float x[8];
          if (fl & kRowBf16) {
            const uint32_t q[4] = {v[j][u][0].x, v[j][u][0].y, v[j][u][0].z, v[j][u][0].w};
#pragma unroll
            for (int h = 0; h < 4; ++h) {
              const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&q[h]));
              x[2 * h] = f.x;
              x[2 * h + 1] = f.y;
            }
          } else {
            x[0] = __uint_as_float(v[j][u][0].x);
            x[1] = __uint_as_float(v[j][u][0].y);
            x[2] = __uint_as_float(v[j][u][0].z);
            x[3] = __uint_as_float(v[j][u][0].w);
            x[4] = __uint_as_float(v[j][u][1].x);
            x[5] = __uint_as_float(v[j][u][1].y);
            x[6] = __uint_as_float(v[j][u][1].z);
            x[7] = __uint_as_float(v[j][u][1].w);
          }
          if (fl & kRowState) {  // wr = 1 / sum of weights
            const int col8 = f8 + 8 * u;
            uint32_t o[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
              const float a0 = acc[u][2 * h] * wr, a1 = acc[u][2 * h + 1] * wr;
              const __nv_bfloat162 b =
                  __floats2bfloat162_rn(fmaf(c, a0 - x[2 * h], x[2 * h]), fmaf(c, a1 - x[2 * h + 1], x[2 * h + 1]));
              o[h] = *reinterpret_cast<const uint32_t*>(&b);
            }
            if (col8 < F8) *(reinterpret_cast<uint4*>(zrow) + col8) = make_uint4(o[0], o[1], o[2], o[3]);
#pragma unroll
            for (int e = 0; e < 8; ++e) acc[u][e] = 0.f;
          } else {
#pragma unroll
            for (int e = 0; e < 8; ++e) acc[u][e] = fmaf(wr, x[e], acc[u][e]);
          }
        }
      }
    }
    __syncwarp();  // the lists are rewritten for the next 32 rows
  }
}

using Clock = std::chrono::steady_clock;
double seconds_since(Clock::time_point t0) {
  return std::chrono::duration<double>(Clock::now() - t0).count();
}

}  // namespace

cudaError_t launch_serve_update(const ReqDesc* reqs, const int64_t* counts, int d, float c, int warp_covers,
                                cudaStream_t st) {
  const unsigned grid = num_sms() * 8;
  if (warp_covers > 0 && warp_covers <= 4 && d == 64)
    serve_update_warp_kernel<4, 1><<<grid, kThreads, 0, st>>>(reqs, counts, d, c);
  else if (warp_covers > 0 && warp_covers <= 4)
    serve_update_warp_kernel<4, 2><<<grid, kThreads, 0, st>>>(reqs, counts, d, c);
  else if (warp_covers > 0 && d == 64)
    serve_update_warp_kernel<kMaxCover, 1><<<grid, kThreads, 0, st>>>(reqs, counts, d, c);
  else if (warp_covers > 0)
    serve_update_warp_kernel<kMaxCover, 2><<<grid, kThreads, 0, st>>>(reqs, counts, d, c);
  else
    serve_update_kernel<<<grid, kThreads, 0, st>>>(reqs, counts, d, c);
  return cudaGetLastError();
}

}  // namespace gattn

using namespace gattn;

struct ServeRequest {
  uint64_t id;
  int T, nh;
  Geom g;
  size_t bytes;
  const void* z0_dev = nullptr;
  std::vector<uint16_t> z0_host;  // copied at submit for host inputs
  __nv_bfloat16* z = nullptr;
  void* out = nullptr;
  float* ot = nullptr;
  CUtensorMap tmap;
  int steps_done = 0;
  double t_submit = 0.0;
  double latency = -1.0;
  size_t held = 0;                // bytes of this request counted in hbm_in_use
  bool taken = false;             // the result was fetched or released
  cudaEvent_t copied = nullptr;   // end of the result's asynchronous copy, while it is in flight
  std::vector<uint16_t> result;   // the result, once spilled to host memory
};

struct gattn_server {
  gattn_serve_cfg cfg;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  Clock::time_point t0;
  bool started = false;
  uint64_t next_id = 1;
  std::deque<ServeRequest*> waiting;
  std::vector<ServeRequest*> active;
  std::deque<ServeRequest*> finished;  // retired, result possibly still in device memory
  cudaMemPool_t pool = nullptr;        // request memory (kept by the pool between requests)
  cudaStream_t copy_stream = nullptr;  // asynchronous result copies (gattn_serve_take_async)
  std::vector<ServeRequest*> copying;  // results whose asynchronous copy may still be in flight
  std::unordered_map<uint64_t, ServeRequest*> all;
  ReqDesc* d_reqs = nullptr;
  int64_t* d_counts = nullptr;
  ReqDesc* h_reqs = nullptr;  // pinned staging
  int64_t* h_counts = nullptr;
  cudaGraphExec_t graph = nullptr;
  int warp_covers = 0;  // most tiles covering a token (<= kMaxCover: the warp-per-32-rows update), else 0
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  size_t hbm_in_use = 0, hbm_peak = 0;
  int64_t submitted = 0, admitted = 0, completed = 0, rejected = 0, iterations = 0;
  double gpu_busy = 0.0, token_steps = 0.0, t_first = -1.0, t_last = 0.0;
  std::vector<double> latencies;
};

// Geometry of a request with T frames and nh heads.  All requests of a server
// share one box shape (the one chosen for a single temporal tile of one head),
// because the ragged launch zeroes the padding rows of its operand blocks once.
static bool serve_geom(const gattn_serve_cfg* cfg, int T, int nh, Geom* g, bool probe = false) {
  if (!probe) {
    Geom p;
    if (!serve_geom(cfg, cfg->core[0], 1, &p, true)) return false;
    const int box[3] = {p.bt, p.by, p.bx};
    return serve_geom(cfg, T, nh, g, true) && apply_box(g, box);
  }
  gattn_desc d;
  memset(&d, 0, sizeof(d));
  d.B = 1;
  d.nh = nh;
  d.d = cfg->d;
  d.T = T;
  d.Y = cfg->Y;
  d.X = cfg->X;
  for (int a = 0; a < 3; ++a) {
    d.core[a] = cfg->core[a];
    d.halo[a] = cfg->halo[a];
  }
  d.window = cfg->window;
  d.in_dtype = GATTN_BF16;
  d.out_dtype = GATTN_BF16;
  return make_geom(&d, g);
}

// rows of the box shape every request of this server uses
static int probe_rows(const gattn_server* s) {
  Geom p;
  return serve_geom(&s->cfg, s->cfg.core[0], 1, &p, true) ? p.R : 128;
}

static size_t request_bytes(const Geom& g) {
  const size_t nd = (size_t)g.nh * g.N * g.d;
  const size_t slots = (size_t)g.nh * g.ntiles * g.per_tile;
  return align_up(nd * 2) + align_up(nd * 2) + align_up(slots * g.d * 4);
}

// Device memory of a request goes back to the server's pool (stream-ordered,
// after the request's last use on the server's stream).
static void free_dev(gattn_server* s, void*& p) {
  if (p) cudaFreeAsync(p, s->stream);
  p = nullptr;
}

static void release(gattn_server* s, ServeRequest* r) {
  void* z = r->z;
  free_dev(s, z);
  free_dev(s, r->out);
  void* ot = r->ot;
  free_dev(s, ot);
  r->z = nullptr;
  r->ot = nullptr;
  s->hbm_in_use -= r->held;
  r->held = 0;
}

// Results whose asynchronous copy has completed give their device memory
// back to the pool; with `wait`, every copy in flight is waited for first.
static void reap(gattn_server* s, bool wait = false) {
  std::vector<ServeRequest*> still;
  for (ServeRequest* r : s->copying) {
    const cudaError_t e = wait ? cudaEventSynchronize(r->copied) : cudaEventQuery(r->copied);
    if (e == cudaErrorNotReady) {
      still.push_back(r);
      continue;
    }
    if (e != cudaSuccess) cudaGetLastError();  // a failed copy still ends: nothing is in flight
    cudaEventDestroy(r->copied);
    r->copied = nullptr;
    release(s, r);
  }
  s->copying.swap(still);
}

// Moves the result of a retired request from device to host memory (when
// waiting requests need the budget and its client has not fetched it yet).
static bool spill(gattn_server* s, ServeRequest* r) {
  const size_t nd = (size_t)r->g.nh * r->g.N * r->g.d;
  r->result.resize(nd);
  if (cudaMemcpyAsync(r->result.data(), r->z, nd * 2, cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
      cudaStreamSynchronize(s->stream) != cudaSuccess)
    return false;
  release(s, r);
  return true;
}

extern "C" {

size_t gattn_serve_request_bytes(const gattn_serve_cfg* cfg, int32_t T, int32_t nh) {
  Geom g;
  if (!cfg || !serve_geom(cfg, T, nh, &g)) return 0;
  return request_bytes(g);
}

gattn_status gattn_serve_create(const gattn_serve_cfg* cfg, gattn_stream_t stream, gattn_server** out) {
  if (!cfg || !out || cfg->steps < 1 || cfg->max_active < 1 || cfg->max_active > 4096 || cfg->hbm_budget == 0)
    return GATTN_ERR_INVALID_ARG;
  Geom probe;
  if (!serve_geom(cfg, cfg->core[0], 1, &probe, true)) return GATTN_ERR_INVALID_ARG;
  gattn_server* s = new gattn_server();
  s->cfg = *cfg;
  {
    // covering tiles per token: temporal extents of 3 c + 2 h frames show the maximum
    Geom span;
    if (serve_geom(cfg, 3 * cfg->core[0] + 2 * cfg->halo[0], 1, &span, true) && max_covers(span) <= kMaxCover)
      s->warp_covers = max_covers(span);
  }
  s->stream = reinterpret_cast<cudaStream_t>(stream);
  if (!s->stream) {
    // the legacy default stream cannot be captured into a graph: use an own
    // blocking stream (ordered with the legacy stream, so inputs produced there
    // are complete before admission copies them)
    if (cudaStreamCreate(&s->stream) != cudaSuccess) {
      delete s;
      return GATTN_ERR_CUDA;
    }
    s->own_stream = true;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  cudaMemPoolProps props;
  memset(&props, 0, sizeof(props));
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  const uint64_t keep_all = ~0ull;  // the pool keeps freed request memory for the next admissions
  bool ok = cudaMemPoolCreate(&s->pool, &props) == cudaSuccess &&
            cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, (void*)&keep_all) == cudaSuccess &&
            cudaMalloc(&s->d_reqs, sizeof(ReqDesc) * cfg->max_active) == cudaSuccess &&
            cudaMalloc(&s->d_counts, 4 * sizeof(int64_t)) == cudaSuccess &&
            cudaMallocHost(&s->h_reqs, sizeof(ReqDesc) * cfg->max_active) == cudaSuccess &&
            cudaMallocHost(&s->h_counts, 4 * sizeof(int64_t)) == cudaSuccess &&
            cudaEventCreate(&s->ev0) == cudaSuccess && cudaEventCreate(&s->ev1) == cudaSuccess &&
            cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking) == cudaSuccess;
  if (!ok) {
    gattn_serve_destroy(s);
    return GATTN_ERR_CUDA;
  }
  *out = s;
  return GATTN_OK;
}

gattn_status gattn_serve_submit(gattn_server* s, const gattn_request* req, uint64_t* id) {
  if (!s || !req || !id || !req->z0 || req->T < 1 || req->nh < 1) return GATTN_ERR_INVALID_ARG;
  Geom g;
  if (!serve_geom(&s->cfg, req->T, req->nh, &g)) return GATTN_ERR_INVALID_ARG;
  ServeRequest* r = new ServeRequest();
  r->id = s->next_id++;
  r->T = req->T;
  r->nh = req->nh;
  r->g = g;
  r->bytes = request_bytes(g);
  if (!s->started) {
    s->t0 = Clock::now();
    s->started = true;
  }
  r->t_submit = seconds_since(s->t0);
  if (s->t_first < 0) s->t_first = r->t_submit;
  ++s->submitted;
  *id = r->id;
  s->all[r->id] = r;
  if (r->bytes > s->cfg.hbm_budget) {
    ++s->rejected;
    r->latency = -2.0;  // marks a rejected request
    return GATTN_ERR_OOM;
  }
  const size_t elems = (size_t)g.nh * g.N * g.d;
  if (req->z0_on_device) {
    r->z0_dev = req->z0;
  } else {
    r->z0_host.resize(elems);
    memcpy(r->z0_host.data(), req->z0, elems * 2);
  }
  s->waiting.push_back(r);
  return GATTN_OK;
}

gattn_status gattn_serve_step(gattn_server* s, int32_t* n_active, int32_t* n_waiting) {
  if (!s) return GATTN_ERR_INVALID_ARG;
  reap(s);  // results copied out since the last iteration free their memory
  // ---- admission: arrival order, slot limit, HBM budget (head of line waits)
  while (!s->waiting.empty() && (int)s->active.size() < s->cfg.max_active) {
    ServeRequest* r = s->waiting.front();
    // results that their clients have not fetched yet move to host memory
    // (oldest first) while the head of the queue does not fit the budget
    while (s->hbm_in_use + r->bytes > s->cfg.hbm_budget && !s->finished.empty()) {
      ServeRequest* f = s->finished.front();
      s->finished.pop_front();
      if (f->z && !f->taken && !spill(s, f)) return GATTN_ERR_CUDA;
    }
    if (s->hbm_in_use + r->bytes > s->cfg.hbm_budget) break;
    const Geom& g = r->g;
    const size_t nd = (size_t)g.nh * g.N * g.d;
    const size_t slots = (size_t)g.nh * g.ntiles * g.per_tile;
    r->held = r->bytes;
    s->hbm_in_use += r->bytes;
    void *z = nullptr, *ot = nullptr;
    if (cudaMallocFromPoolAsync(&z, nd * 2, s->pool, s->stream) != cudaSuccess ||
        cudaMallocFromPoolAsync(&r->out, nd * 2, s->pool, s->stream) != cudaSuccess ||
        cudaMallocFromPoolAsync(&ot, slots * g.d * 4, s->pool, s->stream) != cudaSuccess) {
      r->z = static_cast<__nv_bfloat16*>(z);
      r->ot = static_cast<float*>(ot);
      release(s, r);
      cudaGetLastError();
      break;  // the device is fuller than the budget says: retry next iteration
    }
    r->z = static_cast<__nv_bfloat16*>(z);
    r->ot = static_cast<float*>(ot);
    const void* src = r->z0_dev ? r->z0_dev : (const void*)r->z0_host.data();
    if (cudaMemcpyAsync(r->z, src, nd * 2, cudaMemcpyDefault, s->stream) != cudaSuccess) return GATTN_ERR_CUDA;
    if (!make_tmap_5d(&r->tmap, r->z, g.d, g.G[2], g.G[1], g.G[0], g.nh, g.bx, g.by, g.bt)) return GATTN_ERR_CUDA;
    s->waiting.pop_front();
    s->active.push_back(r);
    s->hbm_peak = std::max(s->hbm_peak, s->hbm_in_use);
    ++s->admitted;
  }
  if (!s->active.empty()) {
    // ---- descriptor table of the active set
    int64_t item = 0;
    int64_t rows = 0;
    for (size_t i = 0; i < s->active.size(); ++i) {
      ServeRequest* r = s->active[i];
      ReqDesc& d = s->h_reqs[i];
      d.tmap = r->tmap;
      d.g = r->g;
      d.z = r->z;
      d.out = r->out;
      d.ot = r->ot;
      d.tok0 = rows;
      d.item0 = (int)item;
      // work items as the ragged forward counts them (box pairs for d = 64, boxes otherwise)
      d.items = s->cfg.d == 64 ? fwd64_ragged_items(r->g) : r->g.nh * r->g.ntiles * r->g.nbmax_tot;
      item += d.items;
      rows += (int64_t)r->g.nh * r->g.N;
    }
    if (item >= (1LL << 31)) return GATTN_ERR_UNSUPPORTED;
    s->h_counts[0] = (int64_t)s->active.size();
    s->h_counts[1] = item;
    s->h_counts[2] = rows;
    s->h_counts[3] = 0;
    if (cudaMemcpyAsync(s->d_reqs, s->h_reqs, sizeof(ReqDesc) * s->active.size(), cudaMemcpyHostToDevice,
                        s->stream) != cudaSuccess ||
        cudaMemcpyAsync(s->d_counts, s->h_counts, 4 * sizeof(int64_t), cudaMemcpyHostToDevice, s->stream) != cudaSuccess)
      return GATTN_ERR_CUDA;
    // ---- the iteration's two launches (graph-captured once)
    cudaEventRecord(s->ev0, s->stream);
    if (s->cfg.use_graph) {
      if (!s->graph) {
        // the first iteration runs its two launches directly (which also sets the
        // kernels' attributes outside capture), then records the same two
        // launches into the graph that every later iteration replays
        if (launch_sm103_fwd_ragged(s->d_reqs, s->d_counts, s->cfg.d, probe_rows(s), s->stream) != cudaSuccess ||
            launch_serve_update(s->d_reqs, s->d_counts, s->cfg.d, s->cfg.c, s->warp_covers, s->stream) != cudaSuccess)
          return GATTN_ERR_CUDA;
        cudaGraph_t gr;
        if (cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return GATTN_ERR_CUDA;
        cudaError_t e1 = launch_sm103_fwd_ragged(s->d_reqs, s->d_counts, s->cfg.d, probe_rows(s), s->stream);
        cudaError_t e2 = launch_serve_update(s->d_reqs, s->d_counts, s->cfg.d, s->cfg.c, s->warp_covers, s->stream);
        cudaError_t e3 = cudaStreamEndCapture(s->stream, &gr);
        if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) return GATTN_ERR_CUDA;
        if (cudaGraphInstantiate(&s->graph, gr, 0) != cudaSuccess) return GATTN_ERR_CUDA;
        cudaGraphDestroy(gr);
      } else if (cudaGraphLaunch(s->graph, s->stream) != cudaSuccess) {
        return GATTN_ERR_CUDA;
      }
    } else {
      if (launch_sm103_fwd_ragged(s->d_reqs, s->d_counts, s->cfg.d, probe_rows(s), s->stream) != cudaSuccess ||
          launch_serve_update(s->d_reqs, s->d_counts, s->cfg.d, s->cfg.c, s->warp_covers, s->stream) != cudaSuccess)
        return GATTN_ERR_CUDA;
    }
    cudaEventRecord(s->ev1, s->stream);
    gattn_status st = gattn_stream_status(reinterpret_cast<gattn_stream_t>(s->stream));
    if (st != GATTN_OK) return st;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, s->ev0, s->ev1);
    s->gpu_busy += ms * 1e-3;
    ++s->iterations;
    // ---- retirement
    std::vector<ServeRequest*> still;
    for (ServeRequest* r : s->active) {
      if (++r->steps_done < s->cfg.steps) {
        still.push_back(r);
        continue;
      }
      // the final state stays in device memory until its client fetches it
      // (gattn_serve_poll) or releases it; the scratch goes back to the pool
      free_dev(s, r->out);
      void* ot = r->ot;
      free_dev(s, ot);
      r->ot = nullptr;
      const size_t zb = align_up((size_t)r->g.nh * r->g.N * r->g.d * 2);
      s->hbm_in_use -= r->held - zb;
      r->held = zb;
      s->finished.push_back(r);
      r->z0_host.clear();
      r->z0_host.shrink_to_fit();
      const double now = seconds_since(s->t0);
      r->latency = now - r->t_submit;
      s->latencies.push_back(r->latency);
      s->token_steps += (double)r->g.nh * r->g.N * s->cfg.steps;
      s->t_last = now;
      ++s->completed;
    }
    s->active.swap(still);
  }
  if (n_active) *n_active = (int32_t)s->active.size();
  if (n_waiting) *n_waiting = (int32_t)s->waiting.size();
  return GATTN_OK;
}

gattn_status gattn_serve_poll(gattn_server* s, uint64_t id, int32_t* done, double* latency_s, void* result_host) {
  if (!s || !done) return GATTN_ERR_INVALID_ARG;
  auto it = s->all.find(id);
  if (it == s->all.end()) return GATTN_ERR_NOT_FOUND;
  ServeRequest* r = it->second;
  if (r->latency == -2.0) return GATTN_ERR_OOM;
  *done = r->latency >= 0.0 ? 1 : 0;
  if (*done) {
    if (latency_s) *latency_s = r->latency;
    if (result_host) {
      if (r->taken) return GATTN_ERR_NOT_FOUND;
      const size_t nd = (size_t)r->g.nh * r->g.N * r->g.d;
      if (r->z) {
        if (cudaMemcpyAsync(result_host, r->z, nd * 2, cudaMemcpyDefault, s->stream) != cudaSuccess ||
            cudaStreamSynchronize(s->stream) != cudaSuccess)
          return GATTN_ERR_CUDA;
        release(s, r);
      } else {
        memcpy(result_host, r->result.data(), nd * 2);
        r->result.clear();
        r->result.shrink_to_fit();
      }
      r->taken = true;
    }
  }
  return GATTN_OK;
}

gattn_status gattn_serve_release(gattn_server* s, uint64_t id) {
  if (!s) return GATTN_ERR_INVALID_ARG;
  auto it = s->all.find(id);
  if (it == s->all.end()) return GATTN_ERR_NOT_FOUND;
  ServeRequest* r = it->second;
  if (r->latency < 0.0) return GATTN_ERR_INVALID_ARG;  // not finished (or rejected)
  if (r->taken) return GATTN_ERR_NOT_FOUND;             // taken or released already
  if (r->z) release(s, r);
  r->result.clear();
  r->result.shrink_to_fit();
  r->taken = true;
  return GATTN_OK;
}

gattn_status gattn_serve_take_async(gattn_server* s, uint64_t id, void* dst) {
  if (!s || !dst) return GATTN_ERR_INVALID_ARG;
  auto it = s->all.find(id);
  if (it == s->all.end()) return GATTN_ERR_NOT_FOUND;
  ServeRequest* r = it->second;
  if (r->latency < 0.0) return GATTN_ERR_INVALID_ARG;  // not finished (or rejected)
  if (r->taken) return GATTN_ERR_NOT_FOUND;
  const size_t nd = (size_t)r->g.nh * r->g.N * r->g.d;
  if (!r->z) {  // spilled to host memory: copied at once
    memcpy(dst, r->result.data(), nd * 2);
    r->result.clear();
    r->result.shrink_to_fit();
    r->taken = true;
    return GATTN_OK;
  }
  // the copy stream starts after everything the server's stream holds so far
  // (the iteration that wrote the final state included)
  if (cudaEventCreateWithFlags(&r->copied, cudaEventDisableTiming) != cudaSuccess) return GATTN_ERR_CUDA;
  if (cudaEventRecord(r->copied, s->stream) != cudaSuccess ||
      cudaStreamWaitEvent(s->copy_stream, r->copied, 0) != cudaSuccess ||
      cudaMemcpyAsync(dst, r->z, nd * 2, cudaMemcpyDefault, s->copy_stream) != cudaSuccess ||
      cudaEventRecord(r->copied, s->copy_stream) != cudaSuccess) {
    cudaStreamSynchronize(s->copy_stream);
    cudaEventDestroy(r->copied);
    r->copied = nullptr;
    return GATTN_ERR_CUDA;
  }
  r->taken = true;
  s->copying.push_back(r);
  return GATTN_OK;
}

gattn_status gattn_serve_copied(gattn_server* s, uint64_t id, int32_t* copied) {
  if (!s || !copied) return GATTN_ERR_INVALID_ARG;
  auto it = s->all.find(id);
  if (it == s->all.end()) return GATTN_ERR_NOT_FOUND;
  reap(s);
  *copied = it->second->taken && !it->second->copied ? 1 : 0;
  return GATTN_OK;
}

gattn_status gattn_serve_stats(gattn_server* s, gattn_serve_stats_t* out) {
  if (!s || !out) return GATTN_ERR_INVALID_ARG;
  memset(out, 0, sizeof(*out));
  out->submitted = s->submitted;
  out->admitted = s->admitted;
  out->completed = s->completed;
  out->rejected = s->rejected;
  out->active = (int64_t)s->active.size();
  out->waiting = (int64_t)s->waiting.size();
  out->iterations = s->iterations;
  out->token_steps = s->token_steps;
  out->gpu_busy_s = s->gpu_busy;
  out->wall_s = s->t_first >= 0 ? s->t_last - s->t_first : 0.0;
  out->hbm_in_use = s->hbm_in_use;
  out->hbm_peak = s->hbm_peak;
  if (!s->latencies.empty()) {
    std::vector<double> v = s->latencies;
    std::sort(v.begin(), v.end());
    auto pct = [&](double q) {
      const double pos = q * (v.size() - 1);
      const size_t i = (size_t)pos;
      const double f = pos - i;
      return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
    };
    out->p50_latency_s = pct(0.50);
    out->p99_latency_s = pct(0.99);
    double sum = 0;
    for (double x : v) sum += x;
    out->mean_latency_s = sum / v.size();
    out->max_latency_s = v.back();
  }
  return GATTN_OK;
}

void gattn_serve_destroy(gattn_server* s) {
  if (!s) return;
  if (s->stream) cudaStreamSynchronize(s->stream);
  reap(s, true);
  for (auto& kv : s->all) {
    release(s, kv.second);
    delete kv.second;
  }
  if (s->stream) cudaStreamSynchronize(s->stream);
  if (s->pool) cudaMemPoolDestroy(s->pool);
  if (s->graph) cudaGraphExecDestroy(s->graph);
  if (s->d_reqs) cudaFree(s->d_reqs);
  if (s->d_counts) cudaFree(s->d_counts);
  if (s->h_reqs) cudaFreeHost(s->h_reqs);
  if (s->h_counts) cudaFreeHost(s->h_counts);
  if (s->ev0) cudaEventDestroy(s->ev0);
  if (s->ev1) cudaEventDestroy(s->ev1);
  if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
  if (s->own_stream) cudaStreamDestroy(s->stream);
  delete s;
}

}  // extern "C"
