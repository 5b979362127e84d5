// gattn_abi.cu -- the C ABI of libgattn (declared in include/gattn.h):
// descriptor validation, buffer sizing and the launch sequence of the
// forward and backward of STORM-GPA (arXiv 2604.16590, Sec. III-C).
#include <math.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "internal.cuh"

namespace gattn {

// ------------------------------------------------------------ kernel timing
namespace {
const char* const kKernelNames[kKCount] = {"fwd_tiles", "merge_fwd", "bwd_prep", "bwd_dkdv", "bwd_dq", "merge_bwd",
                                           "compress", "compress_combine", "gated_mix", "dps_residual",
                                           "dps_update", "linear_summary", "linear_combine", "linear_query",
                                           "linear_bwd_query", "linear_bwd_combine", "linear_bwd_key"};
struct ProfRecord {
  int kernel;
  cudaEvent_t start, stop;
};
struct ProfState {
  std::mutex mu;
  bool on = false;
  std::vector<ProfRecord> recs;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t open_start[kKCount] = {};
};
ProfState& prof() {
  static ProfState s;
  return s;
}
cudaEvent_t take_event(ProfState& p) {
  if (!p.pool.empty()) {
    cudaEvent_t e = p.pool.back();
    p.pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}
}  // namespace

void prof_begin(int kernel, cudaStream_t st) {
  ProfState& p = prof();
  std::lock_guard<std::mutex> lk(p.mu);
  if (!p.on || p.recs.size() >= 65536) return;
  cudaEvent_t e = take_event(p);
  if (e && cudaEventRecord(e, st) == cudaSuccess) p.open_start[kernel] = e;
}

void prof_end(int kernel, cudaStream_t st) {
  ProfState& p = prof();
  std::lock_guard<std::mutex> lk(p.mu);
  if (!p.on || !p.open_start[kernel]) return;
  cudaEvent_t e = take_event(p);
  if (e && cudaEventRecord(e, st) == cudaSuccess) p.recs.push_back({kernel, p.open_start[kernel], e});
  p.open_start[kernel] = nullptr;
}

static bool dtype_ok(int32_t t) { return t == GATTN_BF16 || t == GATTN_FP32; }

static int clipped_extent(const Geom& g, int a, int k) {
  int64_t lo = (int64_t)k * g.c[a] - g.h[a], hi = (int64_t)(k + 1) * g.c[a] + g.h[a];
  lo = lo < 0 ? 0 : lo;
  hi = hi > g.G[a] ? g.G[a] : hi;
  return (int)(hi - lo);
}

bool apply_box(Geom* g, const int b[3]);

// Box shape (bt, by, bx) with R = bt*by*bx <= 128 rows.  Every box is one
// 128-row MMA block, so the attention work of a tile grows with the square of
// its box count and the shape minimising sum_tiles NB_t^2 =
// prod_a sum_k ceil(e_a(k)/b_a)^2 (the sum factorises over dimensions) wins;
// ties go to the fewest rows (least over-fetch), then to the longest
// contiguous x run.  Non-power-of-two shapes matter for small tiles: a 24 x 24
// extended tile takes five 5 x 24 boxes instead of six 4 x 32 boxes of which
// a quarter is outside the tile.
static bool choose_box(Geom* g) {
  // per dimension: the distinct clipped extents and how many tiles have each
  double cost[3][129];
  for (int a = 0; a < 3; ++a) {
    int ext[8], cnt[8], nd = 0;
    for (int k = 0; k < g->n[a]; ++k) {
      const int e = clipped_extent(*g, a, k);
      int i = 0;
      while (i < nd && ext[i] != e) ++i;
      if (i == nd) {
        if (nd == 8) {  // cannot happen (at most first, interior, last two); be safe
          ext[7] = e;
          cnt[7] = 0;
          i = 7;
        } else {
          ext[nd] = e;
          cnt[nd++] = 0;
        }
      }
      ++cnt[i];
    }
    for (int b = 1; b <= 128; ++b) {
      double sum = 0.0;
      for (int i = 0; i < nd; ++i) {
        const double nb = (double)(((int64_t)ext[i] + b - 1) / b);
        sum += cnt[i] * nb * nb;
      }
      cost[a][b] = sum;
    }
  }
  double best_cost = -1.0;
  int best[3] = {1, 1, 128};
  for (int bt = 1; bt <= 128; ++bt)
    for (int by = 1; bt * by <= 128; ++by)
      for (int bx = 1; bt * by * bx <= 128; ++bx) {
        const double c = cost[0][bt] * cost[1][by] * cost[2][bx];
        const int R = bt * by * bx, Rb = best[0] * best[1] * best[2];
        const bool tie = best_cost >= 0 && c <= best_cost * (1 + 1e-12) && c >= best_cost * (1 - 1e-12);
        if (best_cost < 0 || c < best_cost * (1 - 1e-12) || (tie && (R < Rb || (R == Rb && bx > best[2])))) {
          best_cost = c;
          best[0] = bt;
          best[1] = by;
          best[2] = bx;
        }
      }
  return apply_box(g, best);
}

bool apply_box(Geom* g, const int b[3]) {
  if (b[0] < 1 || b[1] < 1 || b[2] < 1 || b[0] * b[1] * b[2] > 128) return false;
  g->bt = b[0];
  g->by = b[1];
  g->bx = b[2];
  g->R = b[0] * b[1] * b[2];
  g->mdx = (65536u + (uint32_t)g->bx - 1) / (uint32_t)g->bx;
  g->mdxy = (65536u + (uint32_t)(g->bx * g->by) - 1) / (uint32_t)(g->bx * g->by);
  int64_t tot = 1;
  for (int a = 0; a < 3; ++a) {
    g->nbmax[a] = (g->emax[a] + b[a] - 1) / b[a];
    tot *= g->nbmax[a];
  }
  if (tot * 128 >= (1LL << 31)) return false;
  g->nbmax_tot = (int32_t)tot;
  g->per_tile = g->nbmax_tot * 128;
  return true;
}

bool make_geom(const gattn_desc* desc, Geom* g) {
  if (!desc || !g) return false;
  memset(g, 0, sizeof(*g));
  const gattn_desc& d = *desc;
  if (d.B < 1 || d.nh < 1 || d.T < 1 || d.Y < 1 || d.X < 1) return false;
  if (!dtype_ok(d.in_dtype) || !dtype_ok(d.out_dtype)) return false;
  if (d.window != GATTN_WINDOW_HANN && d.window != GATTN_WINDOW_FLAT) return false;
  if (d.in_dtype == GATTN_FP32 && d.d != 32 && d.d != 64 && d.d != 128) return false;
  if (d.in_dtype == GATTN_BF16 && d.d != 64 && d.d != 128) return false;
  if (!(d.scale >= 0.f) || !isfinite(d.scale)) return false;
  const int64_t N = (int64_t)d.T * d.Y * d.X;
  if (N >= (1LL << 31)) return false;
  g->B = d.B;
  g->nh = d.nh;
  g->d = d.d;
  g->G[0] = d.T;
  g->G[1] = d.Y;
  g->G[2] = d.X;
  g->N = N;
  int64_t ntiles = 1, Lmax = 1;
  for (int a = 0; a < 3; ++a) {
    if (d.core[a] < 1 || d.halo[a] < 0 || d.halo[a] > (1 << 24)) return false;
    ntiles *= ((int64_t)g->G[a] + d.core[a] - 1) / d.core[a];
  }
  if (ntiles > 65535) return false;  // before the per-tile loops below
  ntiles = 1;
  for (int a = 0; a < 3; ++a) {
    g->c[a] = d.core[a];
    g->h[a] = d.halo[a];
    g->n[a] = (int32_t)(((int64_t)g->G[a] + g->c[a] - 1) / g->c[a]);
    int emax = 0;
    for (int k = 0; k < g->n[a]; ++k) {
      const int e = clipped_extent(*g, a, k);
      emax = e > emax ? e : emax;
    }
    g->emax[a] = emax;
    g->tiled[a] = (g->n[a] > 1 || g->h[a] > 0) ? 1 : 0;
    ntiles *= g->n[a];
    Lmax *= emax;
  }
  if (ntiles > 65535 || Lmax >= (1LL << 31)) return false;
  if ((int64_t)d.B * d.nh > 65535) return false;
  g->ntiles = (int32_t)ntiles;
  g->Lmax = (int32_t)Lmax;
  g->window = d.window;
  g->scale = d.scale > 0.f ? d.scale : 1.0f / sqrtf((float)d.d);
  g->scale_log2 = g->scale * 1.4426950408889634f;
  // a box shape whose per-tile slot count does not fit 32 bits is refused
  if (!choose_box(g)) return false;
  if (g->R < 1 || g->nbmax_tot < 1 || (int64_t)g->nbmax_tot * 128 >= (1LL << 31)) return false;
  return true;
}

// Some token is covered by more than one tile (a tiled dimension with a halo).
static bool has_overlap(const Geom& g) {
  for (int a = 0; a < 3; ++a)
    if (g.n[a] > 1 && g.h[a] > 0) return true;
  return false;
}

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

static gattn_status from_cuda(cudaError_t e) { return e == cudaSuccess ? GATTN_OK : GATTN_ERR_CUDA; }

}  // namespace gattn

using namespace gattn;

extern "C" {

int32_t gattn_abi_version(void) { return 1; }

const char* gattn_status_string(gattn_status s) {
  switch (s) {
    case GATTN_OK: return "ok";
    case GATTN_ERR_INVALID_ARG: return "invalid argument";
    case GATTN_ERR_UNSUPPORTED: return "unsupported";
    case GATTN_ERR_WORKSPACE: return "saved/workspace buffer too small";
    case GATTN_ERR_CUDA: return "CUDA error";
    case GATTN_ERR_TIMEOUT: return "device wait timed out";
    case GATTN_ERR_OOM: return "request exceeds the HBM budget";
    case GATTN_ERR_BUSY: return "no free slot";
    case GATTN_ERR_DEVICE_BOUNDS: return "device bounds check failed";
    case GATTN_ERR_NOT_FOUND: return "unknown request";
  }
  return "unknown status";
}

gattn_status gattn_validate(const gattn_desc* desc) {
  Geom g;
  return make_geom(desc, &g) ? GATTN_OK : GATTN_ERR_INVALID_ARG;
}

int64_t gattn_num_tiles(const gattn_desc* desc) {
  Geom g;
  return make_geom(desc, &g) ? (int64_t)g.ntiles : -1;
}

gattn_status gattn_block_shape(const gattn_desc* desc, int32_t shape[3]) {
  Geom g;
  if (!shape || !make_geom(desc, &g)) return GATTN_ERR_INVALID_ARG;
  shape[0] = g.bt;
  shape[1] = g.by;
  shape[2] = g.bx;
  return GATTN_OK;
}

size_t gattn_saved_bytes(const gattn_desc* desc) {
  Geom g;
  return make_geom(desc, &g) ? saved_layout(g).bytes : 0;
}

size_t gattn_bwd_workspace_bytes(const gattn_desc* desc) {
  Geom g;
  return make_geom(desc, &g) ? bwd_layout(g).bytes : 0;
}

gattn_status gattn_fwd(const gattn_desc* desc, const void* q, const void* k, const void* v, void* out,
                       void* saved, size_t saved_bytes, gattn_stream_t stream) {
  Geom g;
  if (!make_geom(desc, &g)) return GATTN_ERR_INVALID_ARG;
  if (!q || !k || !v || !out || !saved) return GATTN_ERR_INVALID_ARG;
  if (!aligned16(q) || !aligned16(k) || !aligned16(v) || !aligned16(out) || !aligned16(saved))
    return GATTN_ERR_INVALID_ARG;
  const SavedLayout sl = saved_layout(g);
  if (saved_bytes < sl.bytes) return GATTN_ERR_WORKSPACE;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  float* lse2 = reinterpret_cast<float*>(static_cast<char*>(saved) + sl.lse_off);
  float* ot = reinterpret_cast<float*>(static_cast<char*>(saved) + sl.ot_off);
  cudaError_t e;
  prof_begin(kKFwdTiles, st);
  if (desc->in_dtype == GATTN_FP32)
    e = launch_simt_fwd(g, (const float*)q, (const float*)k, (const float*)v, out, desc->out_dtype, lse2, ot, st);
  else
    e = launch_sm103_fwd(g, (const __nv_bfloat16*)q, (const __nv_bfloat16*)k, (const __nv_bfloat16*)v, out,
                         desc->out_dtype, lse2, ot, desc->flags, st);
  prof_end(kKFwdTiles, st);
  if (e == cudaErrorNotSupported) return GATTN_ERR_UNSUPPORTED;
  if (e != cudaSuccess) return GATTN_ERR_CUDA;
  if (has_overlap(g)) {
    prof_begin(kKMergeFwd, st);
    e = launch_merge_fwd(g, ot, out, desc->out_dtype, st);
    prof_end(kKMergeFwd, st);
  }
  return from_cuda(e);
}

gattn_status gattn_bwd(const gattn_desc* desc, const void* q, const void* k, const void* v, const void* out,
                       const void* dout, const void* saved, size_t saved_bytes, void* dq, void* dk, void* dv,
                       void* ws, size_t ws_bytes, gattn_stream_t stream) {
  Geom g;
  if (!make_geom(desc, &g)) return GATTN_ERR_INVALID_ARG;
  const void* ptrs[] = {q, k, v, out, dout, saved, dq, dk, dv, ws};
  for (const void* p : ptrs)
    if (!p || !aligned16(p)) return GATTN_ERR_INVALID_ARG;
  const SavedLayout sl = saved_layout(g);
  const BwdLayout bl = bwd_layout(g);
  if (saved_bytes < sl.bytes || ws_bytes < bl.bytes) return GATTN_ERR_WORKSPACE;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const float* lse2 = reinterpret_cast<const float*>(static_cast<const char*>(saved) + sl.lse_off);
  const float* ot = reinterpret_cast<const float*>(static_cast<const char*>(saved) + sl.ot_off);
  char* w = static_cast<char*>(ws);
  float* lse2c = reinterpret_cast<float*>(w + bl.lse_off);
  float* dd = reinterpret_cast<float*>(w + bl.dd_off);
  // the statistics rows are read only by the tensor-core dK/dV kernels
  void* ext = desc->in_dtype == GATTN_BF16 ? static_cast<void*>(w + bl.ext_off) : nullptr;
  float* dq_s = reinterpret_cast<float*>(w + bl.dq_off);
  float* dk_s = reinterpret_cast<float*>(w + bl.dk_off);
  float* dv_s = reinterpret_cast<float*>(w + bl.dv_off);
  prof_begin(kKBwdPrep, st);
  cudaError_t e = launch_bwd_prep(g, out, desc->out_dtype, dout, desc->in_dtype, lse2, ot, lse2c, dd, ext, st);
  prof_end(kKBwdPrep, st);
  if (e != cudaSuccess) return GATTN_ERR_CUDA;
  if (desc->in_dtype == GATTN_FP32)
    e = launch_simt_bwd(g, (const float*)q, (const float*)k, (const float*)v, (const float*)dout, lse2c, dd, dq, dk,
                        dv, desc->out_dtype, dq_s, dk_s, dv_s, st);
  else
    e = launch_sm103_bwd(g, (const __nv_bfloat16*)q, (const __nv_bfloat16*)k, (const __nv_bfloat16*)v,
                         (const __nv_bfloat16*)dout, lse2c, dd, ext, dq, dk, dv, desc->out_dtype, dq_s, dk_s, dv_s,
                         desc->flags, st);
  if (e == cudaErrorNotSupported) return GATTN_ERR_UNSUPPORTED;
  if (e != cudaSuccess) return GATTN_ERR_CUDA;
  if (has_overlap(g)) {
    prof_begin(kKMergeBwd, st);
    e = launch_merge_bwd(g, dq_s, dk_s, dv_s, dq, dk, dv, desc->out_dtype, st);
    prof_end(kKMergeBwd, st);
  }
  return from_cuda(e);
}

// Factorised linear attention (not an operator of the paper; see linear.cu).
static bool linear_desc_ok(const gattn_linear_desc* l) {
  return l && l->B >= 1 && l->nh >= 1 && l->d == 64 && l->N >= 1 && l->N < (1LL << 31) &&
         l->in_dtype == GATTN_BF16 && l->out_dtype == GATTN_BF16 && (double)l->B * l->nh < 65536.0;
}

size_t gattn_linear_workspace_bytes(const gattn_linear_desc* l) {
  if (!linear_desc_ok(l)) return 0;
  return linear_ws_bytes(l->B, l->nh, l->N);
}

gattn_status gattn_linear_fwd(const gattn_linear_desc* l, const void* q, const void* k, const void* v, void* out,
                              void* ws, size_t ws_bytes, gattn_stream_t stream) {
  if (!linear_desc_ok(l)) return GATTN_ERR_INVALID_ARG;
  const void* ptrs[] = {q, k, v, out, ws};
  for (const void* p : ptrs)
    if (!p || !aligned16(p)) return GATTN_ERR_INVALID_ARG;
  if (ws_bytes < linear_ws_bytes(l->B, l->nh, l->N)) return GATTN_ERR_WORKSPACE;
  return from_cuda(launch_linear(q, k, v, out, ws, l->B, l->nh, l->N, reinterpret_cast<cudaStream_t>(stream)));
}

size_t gattn_linear_bwd_workspace_bytes(const gattn_linear_desc* l) {
  if (!linear_desc_ok(l)) return 0;
  return linear_bwd_layout(l->B, l->nh, l->N).bytes;
}

gattn_status gattn_linear_bwd(const gattn_linear_desc* l, const void* q, const void* k, const void* v,
                              const void* dout, const void* saved, size_t saved_bytes, void* dq, void* dk, void* dv,
                              void* ws, size_t ws_bytes, gattn_stream_t stream) {
  if (!linear_desc_ok(l)) return GATTN_ERR_INVALID_ARG;
  const void* ptrs[] = {q, k, v, dout, saved, dq, dk, dv, ws};
  for (const void* p : ptrs)
    if (!p || !aligned16(p)) return GATTN_ERR_INVALID_ARG;
  if (saved_bytes < linear_ws_bytes(l->B, l->nh, l->N) || ws_bytes < linear_bwd_layout(l->B, l->nh, l->N).bytes)
    return GATTN_ERR_WORKSPACE;
  return from_cuda(launch_linear_bwd(q, k, v, dout, saved, dq, dk, dv, ws, l->B, l->nh, l->N,
                                     reinterpret_cast<cudaStream_t>(stream)));
}

// Posterior-sampling step (Sec. III-A).  Workspace: attention saved state,
// backward workspace, then D, dq, dk, dv (FP32) and the residual r (in_dtype).
struct DpsLayout {
  size_t saved, bws, D, dq, dk, dv, r, bytes;
};
static DpsLayout dps_layout(const gattn_desc* desc, const Geom& g) {
  DpsLayout l;
  const size_t nd = (size_t)g.B * g.nh * g.N * g.d;
  l.saved = 0;
  l.bws = align_up(saved_layout(g).bytes);
  l.D = l.bws + align_up(bwd_layout(g).bytes);
  l.dq = l.D + align_up(nd * 4);
  l.dk = l.dq + align_up(nd * 4);
  l.dv = l.dk + align_up(nd * 4);
  l.r = l.dv + align_up(nd * 4);
  l.bytes = l.r + align_up(nd * (desc->in_dtype == GATTN_BF16 ? 2 : 4));
  return l;
}

size_t gattn_dps_workspace_bytes(const gattn_desc* desc) {
  Geom g;
  if (!make_geom(desc, &g) || desc->out_dtype != GATTN_FP32) return 0;
  return dps_layout(desc, g).bytes;
}

gattn_status gattn_dps_step(const gattn_desc* desc, const gattn_dps_params* p, float* z, void* zb, const float* y,
                            const uint8_t* mask, const float* eps, void* ws, size_t ws_bytes,
                            gattn_stream_t stream) {
  Geom g;
  if (!make_geom(desc, &g) || desc->out_dtype != GATTN_FP32 || !p) return GATTN_ERR_INVALID_ARG;
  const bool bf16 = desc->in_dtype == GATTN_BF16;
  const void* ptrs[] = {z, y, eps, ws};
  for (const void* q : ptrs)
    if (!q || !aligned16(q)) return GATTN_ERR_INVALID_ARG;
  if (!mask || (bf16 && (!zb || !aligned16(zb)))) return GATTN_ERR_INVALID_ARG;
  if (!(p->sigma > 0.f) || !(p->sigma_next >= 0.f) || !(p->sigma_next <= p->sigma) || !isfinite(p->sigma) ||
      !isfinite(p->lam))
    return GATTN_ERR_INVALID_ARG;
  const DpsLayout l = dps_layout(desc, g);
  if (ws_bytes < l.bytes) return GATTN_ERR_WORKSPACE;
  char* w = static_cast<char*>(ws);
  float* D = reinterpret_cast<float*>(w + l.D);
  float* dq = reinterpret_cast<float*>(w + l.dq);
  float* dk = reinterpret_cast<float*>(w + l.dk);
  float* dv = reinterpret_cast<float*>(w + l.dv);
  void* r = w + l.r;
  const void* a = bf16 ? static_cast<const void*>(zb) : static_cast<const void*>(z);
  const size_t sb = saved_layout(g).bytes, bb = bwd_layout(g).bytes;
  gattn_status s = gattn_fwd(desc, a, a, a, D, w + l.saved, sb, stream);
  if (s != GATTN_OK) return s;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  prof_begin(kKDpsResidual, st);
  cudaError_t e = launch_dps_residual(g, D, y, mask, r, bf16, st);
  prof_end(kKDpsResidual, st);
  if (e != cudaSuccess) return GATTN_ERR_CUDA;
  s = gattn_bwd(desc, a, a, a, D, r, w + l.saved, sb, dq, dk, dv, w + l.bws, bb, stream);
  if (s != GATTN_OK) return s;
  prof_begin(kKDpsUpdate, st);
  e = launch_dps_update(g, z, bf16 ? zb : nullptr, D, dq, dk, dv, eps, p->sigma, p->sigma_next, p->lam, st);
  prof_end(kKDpsUpdate, st);
  return from_cuda(e);
}

// Noise-gated self + cross attention (Sec. III-B): the workspace holds the
// saved state (reused by both attentions; forward only) and the cross output.
static size_t gated_cross_off(const Geom& g) { return align_up(saved_layout(g).bytes); }
static size_t out_elem_bytes(int32_t t) { return t == GATTN_BF16 ? 2 : 4; }

size_t gattn_gated_workspace_bytes(const gattn_desc* desc) {
  Geom g;
  if (!make_geom(desc, &g)) return 0;
  return gated_cross_off(g) + align_up((size_t)g.B * g.nh * g.N * g.d * out_elem_bytes(desc->out_dtype));
}

gattn_status gattn_gated_fwd(const gattn_desc* desc, const void* q, const void* k, const void* v, const void* kc,
                             const void* vc, const float* gate, void* out, void* ws, size_t ws_bytes,
                             gattn_stream_t stream) {
  Geom g;
  if (!make_geom(desc, &g)) return GATTN_ERR_INVALID_ARG;
  const void* ptrs[] = {q, k, v, kc, vc, gate, out, ws};
  for (const void* p : ptrs)
    if (!p || !aligned16(p)) return GATTN_ERR_INVALID_ARG;
  if (ws_bytes < gattn_gated_workspace_bytes(desc)) return GATTN_ERR_WORKSPACE;
  const SavedLayout sl = saved_layout(g);
  void* cross = static_cast<char*>(ws) + gated_cross_off(g);
  gattn_status s = gattn_fwd(desc, q, k, v, out, ws, sl.bytes, stream);
  if (s != GATTN_OK) return s;
  s = gattn_fwd(desc, q, kc, vc, cross, ws, sl.bytes, stream);
  if (s != GATTN_OK) return s;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  prof_begin(kKGatedMix, st);
  const cudaError_t e = launch_gated_mix(g, out, cross, gate, desc->out_dtype, st);
  prof_end(kKGatedMix, st);
  return from_cuda(e);
}

static bool compress_desc_ok(const gattn_compress_desc* c) {
  if (!c) return false;
  if (c->B < 1 || c->nh < 1 || c->S < 1 || c->M < 1) return false;
  if (!dtype_ok(c->in_dtype) || !dtype_ok(c->out_dtype)) return false;
  if (c->in_dtype == GATTN_BF16 && c->d != 64 && c->d != 128) return false;
  if (c->in_dtype == GATTN_FP32 && c->d != 32 && c->d != 64 && c->d != 128) return false;
  if (!(c->scale >= 0.f) || !isfinite(c->scale)) return false;
  // element offsets of k/v stay below 2^62 and grid sizes below 2^31
  const double kv = (double)c->B * c->nh * c->S * c->M * c->d;
  const double items = (double)c->B * c->nh * ((c->M + 31) / 32) * 64.0;
  return kv < 4.0e18 && items < 2.0e9;
}

size_t gattn_compress_workspace_bytes(const gattn_compress_desc* c) {
  if (!compress_desc_ok(c)) return 0;
  return compress_ws_bytes(c->B, c->nh, c->S, c->M, c->d);
}

gattn_status gattn_compress_fwd(const gattn_compress_desc* c, const float* q, const void* k, const void* v, void* out,
                                float* lse, void* ws, size_t ws_bytes, gattn_stream_t stream) {
  if (!compress_desc_ok(c)) return GATTN_ERR_INVALID_ARG;
  if (!q || !k || !v || !out) return GATTN_ERR_INVALID_ARG;
  if (!aligned16(q) || !aligned16(k) || !aligned16(v) || !aligned16(out)) return GATTN_ERR_INVALID_ARG;
  if (lse && ((uintptr_t)lse & 3u)) return GATTN_ERR_INVALID_ARG;
  const size_t need = compress_ws_bytes(c->B, c->nh, c->S, c->M, c->d);
  if (need && (!ws || ws_bytes < need || !aligned16(ws))) return GATTN_ERR_WORKSPACE;
  const float scale = c->scale > 0.f ? c->scale : 1.f / sqrtf((float)c->d);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  return from_cuda(launch_compress(q, k, v, out, lse, need ? static_cast<float*>(ws) : nullptr, c->B, c->nh, c->S,
                                   c->M, c->d, c->in_dtype == GATTN_BF16, c->out_dtype == GATTN_BF16, scale, st));
}

gattn_status gattn_profile_enable(int32_t enable) {
  ProfState& p = prof();
  std::lock_guard<std::mutex> lk(p.mu);
  if (enable) {
    for (auto& r : p.recs) {
      p.pool.push_back(r.start);
      p.pool.push_back(r.stop);
    }
    p.recs.clear();
  }
  p.on = enable != 0;
  return GATTN_OK;
}

int32_t gattn_profile_read(gattn_kernel_stat* out, int32_t max) {
  ProfState& p = prof();
  std::lock_guard<std::mutex> lk(p.mu);
  int64_t n[kKCount] = {};
  double ms[kKCount] = {};
  for (auto& r : p.recs) {
    float t = 0.f;
    if (cudaEventSynchronize(r.stop) != cudaSuccess || cudaEventElapsedTime(&t, r.start, r.stop) != cudaSuccess)
      return -(int32_t)GATTN_ERR_CUDA;
    n[r.kernel] += 1;
    ms[r.kernel] += t;
  }
  int32_t count = 0;
  for (int k = 0; k < kKCount; ++k) {
    if (!n[k]) continue;
    if (out && count < max) {
      memset(out[count].name, 0, sizeof(out[count].name));
      strncpy(out[count].name, kKernelNames[k], sizeof(out[count].name) - 1);
      out[count].launches = n[k];
      out[count].total_ms = ms[k];
    }
    ++count;
  }
  return count;
}

gattn_status gattn_stream_status(gattn_stream_t stream) {
  if (cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess) return GATTN_ERR_CUDA;
  uint32_t words[] = {fetch_status_simt(), fetch_status_merge(), fetch_status_sm103_fwd(), fetch_status_sm103_fwd64(), fetch_status_sm103_bwd(),
                      fetch_status_sm103_bwd64(),
                      fetch_status_serve(), fetch_status_compress(), fetch_status_linear()};
  for (uint32_t w : words)
    if (w == ~0u) return GATTN_ERR_CUDA;
  for (uint32_t w : words)
    if (w) return (gattn_status)w;
  return GATTN_OK;
}

}  // extern "C"
