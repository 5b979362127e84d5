/*
 * gpa_oracle.c -- plain FP64 CPU oracle of STORM Global Propagation Attention
 * (STORM-GPA), arXiv 2604.16590, Sec. III-C and Fig. 3(a).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * definition the CUDA library is checked against.  Only the test suite, the
 * smoke check and the benchmark's CPU-baseline leg may load it; the library
 * never links, calls or includes it, and it includes nothing of the library.
 *
 * What it computes (the paper's steps, in the paper's order):
 *   1. Partition the (T, Y, X) token grid into tiles (Sec. III-C, first
 *      paragraph: "partition the spatiotemporal volume into tiles").
 *   2. Extend every tile by spatiotemporal halos that overlap its neighbours
 *      (Sec. III-C, same paragraph; Fig. 3(a) ii-iii).
 *   3. Run ordinary softmax attention independently inside every extended
 *      tile; interior tokens attend to halo tokens (Sec. III-C, "This shared
 *      context information is then propagated within each tile through
 *      attention"; Sec. III-D Level 5 names FlashAttention, i.e. exact softmax
 *      attention).
 *   4. Average the per-tile outputs where tiles overlap (Sec. III-C, "average
 *      denoised outputs in overlapping halos"; Fig. 3(a) iv), weighting every
 *      contribution by a Hanning window that trusts tile centres more than
 *      tile edges (Sec. III-C last sentence; Fig. 3(a) vi).
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - tile shape, halo width and whether time is tiled are free parameters
 *     (core[3], halo[3]); the last tile of a dimension may be short;
 *   - extended intervals are clipped to the grid (no periodic longitude);
 *   - every token of an extended tile is a query (all of them get an output);
 *   - window: per dimension a, with nominal extended length M = c + 2h and
 *     offset n from the nominal (unclipped) start k*c - h,
 *         win(n) = sin^2(pi * (n + 1/2) / M)
 *     (a Hann window sampled at half-integer points: strictly positive and
 *     symmetric).  A dimension that is not tiled (one tile, no halo) has
 *     weight 1.  The tile weight is the product over the three dimensions.
 *     window == 1 selects a flat window (plain average);
 *   - the average is normalised: Out(i) = sum_t w_t(i) O_t(i) / sum_t w_t(i),
 *     summed in ascending tile order;
 *   - softmax scale s (1/sqrt(d) by default), no mask, heads independent;
 *   - memory layout [B, heads, N, d], token i = (t*Y + y)*X + x.
 *
 * The backward is the analytic gradient of that forward for the scalar
 * loss sum(Out * dOut): with c_t(i) = w_t(i) / sum_t' w_t'(i),
 *   dO_t(i) = c_t(i) dOut(i),  D_t(i) = dO_t(i) . O_t(i),
 *   P = softmax(s Q K^T) inside the tile,  dP = dO_t V^T,
 *   dS = P * (dP - D),  dQ_t = s dS K,  dK_t = s dS^T Q,  dV_t = P^T dO_t,
 * and every input gradient is the ascending-tile sum of the per-tile ones.
 * The paper needs this gradient because diffusion training and the
 * likelihood score of posterior sampling (Sec. III-A, Eq. 8) differentiate
 * through the denoiser.
 *
 * Geometry array g[12] = {B, nh, d, T, Y, X, ct, cy, cx, ht, hy, hx}.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define G_B 0
#define G_NH 1
#define G_D 2
#define G_T 3
#define G_Y 4
#define G_X 5
#define G_C 6 /* core[0..2] at 6,7,8 */
#define G_H 9 /* halo[0..2] at 9,10,11 */

static const double ORACLE_PI = 3.14159265358979323846;

/* number of tiles along one dimension of extent G with core c */
static int ntiles_dim(int G, int c) { return (G + c - 1) / c; }

int gpa_oracle_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

int gpa_num_tiles(const int32_t *g) {
  return ntiles_dim(g[G_T], g[G_C + 0]) * ntiles_dim(g[G_Y], g[G_C + 1]) *
         ntiles_dim(g[G_X], g[G_C + 2]);
}

/* Step 1+2: the clipped extended interval [lo, hi) of tile k along one
 * dimension, and its nominal start k*c - h. */
static void ext_interval(int G, int c, int h, int k, int *lo, int *hi, int *nominal_lo) {
  int a = k * c - h, b = (k + 1) * c + h;
  *nominal_lo = a;
  *lo = a < 0 ? 0 : a;
  *hi = b > G ? G : b;
}

/* Step 4 window along one dimension, offset n from the nominal start. */
double gpa_window_1d(int n, int M) {
  double s = sin(ORACLE_PI * ((double)n + 0.5) / (double)M);
  return s * s;
}

typedef struct {
  int lo[3], hi[3], nlo[3], ext[3];
  int L;
} tile_box;

static void tile_of(const int32_t *g, int tile, tile_box *tb) {
  int n[3], kk[3];
  const int Gs[3] = {g[G_T], g[G_Y], g[G_X]};
  for (int a = 0; a < 3; ++a) n[a] = ntiles_dim(Gs[a], g[G_C + a]);
  kk[2] = tile % n[2];
  kk[1] = (tile / n[2]) % n[1];
  kk[0] = tile / (n[2] * n[1]);
  tb->L = 1;
  for (int a = 0; a < 3; ++a) {
    ext_interval(Gs[a], g[G_C + a], g[G_H + a], kk[a], &tb->lo[a], &tb->hi[a], &tb->nlo[a]);
    tb->ext[a] = tb->hi[a] - tb->lo[a];
    tb->L *= tb->ext[a];
  }
}

/* Hann (or flat) weight of tile tb for the token at grid position p[3]. */
static double tile_weight(const int32_t *g, int window, const tile_box *tb, const int p[3]) {
  if (window == 1) return 1.0;
  const int Gs[3] = {g[G_T], g[G_Y], g[G_X]};
  double w = 1.0;
  for (int a = 0; a < 3; ++a) {
    int c = g[G_C + a], h = g[G_H + a];
    if (ntiles_dim(Gs[a], c) == 1 && h == 0) continue; /* untiled dimension */
    w *= gpa_window_1d(p[a] - tb->nlo[a], c + 2 * h);
  }
  return w;
}

/* grid index of local row r of tile tb */
static int64_t token_of_row(const int32_t *g, const tile_box *tb, int r) {
  int lx = r % tb->ext[2];
  int ly = (r / tb->ext[2]) % tb->ext[1];
  int lt = r / (tb->ext[2] * tb->ext[1]);
  int t = tb->lo[0] + lt, y = tb->lo[1] + ly, x = tb->lo[2] + lx;
  return ((int64_t)t * g[G_Y] + y) * g[G_X] + x;
}

static int contains(const tile_box *tb, const int p[3]) {
  for (int a = 0; a < 3; ++a)
    if (p[a] < tb->lo[a] || p[a] >= tb->hi[a]) return 0;
  return 1;
}

static int row_of_token(const tile_box *tb, const int p[3]) {
  return ((p[0] - tb->lo[0]) * tb->ext[1] + (p[1] - tb->lo[1])) * tb->ext[2] + (p[2] - tb->lo[2]);
}

static void pos_of_token(const int32_t *g, int64_t i, int p[3]) {
  p[2] = (int)(i % g[G_X]);
  p[1] = (int)((i / g[G_X]) % g[G_Y]);
  p[0] = (int)(i / ((int64_t)g[G_X] * g[G_Y]));
}

static double dot(const double *a, const double *b, int d) {
  double s = 0.0;
  for (int e = 0; e < d; ++e) s += a[e] * b[e];
  return s;
}

/* Step 3 for one (batch*head, tile) unit, query rows [r0, r1):
 *   O_t[r] = softmax_j(s q_r . k_j) v_j over all j in the extended tile,
 *   lse[r] = log sum_j exp(s q_r . k_j).
 * q,k,v point at the [N, d] slice of this batch*head.  O_t and lse hold the
 * rows r0..r1-1 only (row r at index r - r0); lse may be NULL. */
static void tile_attention(const int32_t *g, double scale, const tile_box *tb, const double *q,
                           const double *k, const double *v, int r0, int r1, double *O_t,
                           double *lse) {
  const int d = g[G_D], L = tb->L;
  double *srow = (double *)malloc(sizeof(double) * (size_t)L);
  int64_t *tok = (int64_t *)malloc(sizeof(int64_t) * (size_t)L);
  for (int j = 0; j < L; ++j) tok[j] = token_of_row(g, tb, j);
  for (int r = r0; r < r1; ++r) {
    const double *qr = q + tok[r] * d;
    double m = -INFINITY;
    for (int j = 0; j < L; ++j) {
      srow[j] = scale * dot(qr, k + tok[j] * d, d);
      if (srow[j] > m) m = srow[j];
    }
    double l = 0.0;
    for (int j = 0; j < L; ++j) {
      srow[j] = exp(srow[j] - m);
      l += srow[j];
    }
    double *o = O_t + (size_t)(r - r0) * d;
    for (int e = 0; e < d; ++e) o[e] = 0.0;
    for (int j = 0; j < L; ++j) {
      const double *vj = v + tok[j] * d;
      double p = srow[j] / l;
      for (int e = 0; e < d; ++e) o[e] += p * vj[e];
    }
    if (lse) lse[r - r0] = m + log(l);
  }
  free(srow);
  free(tok);
}

/* Forward of the whole operator.  out is [B, nh, N, d]. */
void gpa_forward(const int32_t *g, int window, double scale, const double *q, const double *k,
                 const double *v, double *out) {
  const int BH = g[G_B] * g[G_NH], d = g[G_D], nt = gpa_num_tiles(g);
  const int64_t N = (int64_t)g[G_T] * g[G_Y] * g[G_X];
  const int64_t units = (int64_t)BH * nt;
  double **Ot = (double **)calloc((size_t)units, sizeof(double *));
  /* step 3: every (batch*head, tile) independently */
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t u = 0; u < units; ++u) {
    int bh = (int)(u / nt), t = (int)(u % nt);
    tile_box tb;
    tile_of(g, t, &tb);
    Ot[u] = (double *)malloc(sizeof(double) * (size_t)tb.L * d);
    const size_t off = (size_t)bh * N * d;
    tile_attention(g, scale, &tb, q + off, k + off, v + off, 0, tb.L, Ot[u], NULL);
  }
  /* step 4: Hann-weighted average over the tiles that cover each token */
#pragma omp parallel for schedule(static)
  for (int64_t bi = 0; bi < (int64_t)BH * N; ++bi) {
    int bh = (int)(bi / N);
    int64_t i = bi % N;
    int p[3];
    pos_of_token(g, i, p);
    double *o = out + bi * d;
    for (int e = 0; e < d; ++e) o[e] = 0.0;
    double wsum = 0.0;
    for (int t = 0; t < nt; ++t) {
      tile_box tb;
      tile_of(g, t, &tb);
      if (!contains(&tb, p)) continue;
      double w = tile_weight(g, window, &tb, p);
      const double *ot = Ot[(int64_t)bh * nt + t] + (size_t)row_of_token(&tb, p) * d;
      for (int e = 0; e < d; ++e) o[e] += w * ot[e];
      wsum += w;
    }
    for (int e = 0; e < d; ++e) o[e] /= wsum;
  }
  for (int64_t u = 0; u < units; ++u) free(Ot[u]);
  free(Ot);
}

/* sum_t w_t(i) over the tiles covering grid position p */
static double weight_sum(const int32_t *g, int window, const int p[3]) {
  const int nt = gpa_num_tiles(g);
  double ws = 0.0;
  for (int t = 0; t < nt; ++t) {
    tile_box tb;
    tile_of(g, t, &tb);
    if (contains(&tb, p)) ws += tile_weight(g, window, &tb, p);
  }
  return ws;
}

/* Backward for one (batch*head, tile) unit, query rows [r0, r1).  Writes the
 * per-tile gradients dQ_t (rows r0..r1) and accumulates dK_t, dV_t over those
 * rows (all L rows of dK_t, dV_t are touched). */
static void tile_backward(const int32_t *g, int window, double scale, const tile_box *tb,
                          const double *q, const double *k, const double *v, const double *dout,
                          int r0, int r1, double *dQt, double *dKt, double *dVt) {
  const int d = g[G_D], L = tb->L;
  const int R = r1 > r0 ? r1 - r0 : 1;
  double *O = (double *)malloc(sizeof(double) * (size_t)R * d);
  double *lse = (double *)malloc(sizeof(double) * (size_t)R);
  double *dOt = (double *)malloc(sizeof(double) * (size_t)d);
  int64_t *tok = (int64_t *)malloc(sizeof(int64_t) * (size_t)L);
  for (int j = 0; j < L; ++j) tok[j] = token_of_row(g, tb, j);
  /* recompute the forward of this tile for the rows needed */
  tile_attention(g, scale, tb, q, k, v, r0, r1, O, lse);
  for (int r = r0; r < r1; ++r) {
    int p[3];
    pos_of_token(g, tok[r], p);
    double c = tile_weight(g, window, tb, p) / weight_sum(g, window, p);
    const double *qr = q + tok[r] * d;
    const double *dor = dout + tok[r] * d;
    for (int e = 0; e < d; ++e) dOt[e] = c * dor[e];
    double D = dot(dOt, O + (size_t)(r - r0) * d, d);
    double *dq = dQt + (size_t)r * d;
    for (int e = 0; e < d; ++e) dq[e] = 0.0;
    for (int j = 0; j < L; ++j) {
      const double *kj = k + tok[j] * d, *vj = v + tok[j] * d;
      double P = exp(scale * dot(qr, kj, d) - lse[r - r0]);
      double dP = dot(dOt, vj, d);
      double dS = P * (dP - D);
      double *dk = dKt + (size_t)j * d, *dv = dVt + (size_t)j * d;
      for (int e = 0; e < d; ++e) {
        dq[e] += scale * dS * kj[e];
        dk[e] += scale * dS * qr[e];
        dv[e] += P * dOt[e];
      }
    }
  }
  free(O);
  free(lse);
  free(dOt);
  free(tok);
}

/* Backward of the whole operator for the loss sum(Out * dout). */
void gpa_backward(const int32_t *g, int window, double scale, const double *q, const double *k,
                  const double *v, const double *dout, double *dq, double *dk, double *dv) {
  const int BH = g[G_B] * g[G_NH], d = g[G_D], nt = gpa_num_tiles(g);
  const int64_t N = (int64_t)g[G_T] * g[G_Y] * g[G_X];
  const int64_t units = (int64_t)BH * nt;
  double **buf = (double **)calloc((size_t)units, sizeof(double *));
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t u = 0; u < units; ++u) {
    int bh = (int)(u / nt), t = (int)(u % nt);
    tile_box tb;
    tile_of(g, t, &tb);
    buf[u] = (double *)calloc((size_t)3 * tb.L * d, sizeof(double));
    const size_t off = (size_t)bh * N * d;
    double *dQt = buf[u], *dKt = buf[u] + (size_t)tb.L * d, *dVt = buf[u] + (size_t)2 * tb.L * d;
    tile_backward(g, window, scale, &tb, q + off, k + off, v + off, dout + off, 0, tb.L, dQt, dKt,
                  dVt);
  }
  /* every input gradient is the ascending-tile sum of the per-tile ones */
#pragma omp parallel for schedule(static)
  for (int64_t bi = 0; bi < (int64_t)BH * N; ++bi) {
    int bh = (int)(bi / N);
    int64_t i = bi % N;
    int p[3];
    pos_of_token(g, i, p);
    double *a = dq + bi * d, *b = dk + bi * d, *c = dv + bi * d;
    for (int e = 0; e < d; ++e) a[e] = b[e] = c[e] = 0.0;
    for (int t = 0; t < nt; ++t) {
      tile_box tb;
      tile_of(g, t, &tb);
      if (!contains(&tb, p)) continue;
      const double *base = buf[(int64_t)bh * nt + t];
      size_t r = (size_t)row_of_token(&tb, p) * d;
      for (int e = 0; e < d; ++e) {
        a[e] += base[r + e];
        b[e] += base[(size_t)tb.L * d + r + e];
        c[e] += base[(size_t)2 * tb.L * d + r + e];
      }
    }
  }
  for (int64_t u = 0; u < units; ++u) free(buf[u]);
  free(buf);
}

/* Forward and dQ for a list of sampled outputs.  rows[n] holds (b*nh + h) * N
 * + i.  Both are row-local: they need only the sampled query and the keys and
 * values of the tiles that cover it.  out_rows and dq_rows are [n, d];
 * dq_rows may be NULL (then dout is not read). */
void gpa_rows(const int32_t *g, int window, double scale, const double *q, const double *k,
              const double *v, const double *dout, int64_t n, const int64_t *rows, double *out_rows,
              double *dq_rows) {
  const int d = g[G_D], nt = gpa_num_tiles(g);
  const int64_t N = (int64_t)g[G_T] * g[G_Y] * g[G_X];
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t s = 0; s < n; ++s) {
    int64_t bh = rows[s] / N, i = rows[s] % N;
    const size_t off = (size_t)bh * N * d;
    int p[3];
    pos_of_token(g, i, p);
    double wsum = weight_sum(g, window, p);
    double *o = out_rows + s * d;
    double *dq = dq_rows ? dq_rows + s * d : NULL;
    double *Ot = (double *)malloc(sizeof(double) * (size_t)d);
    double *dOt = (double *)malloc(sizeof(double) * (size_t)d);
    for (int e = 0; e < d; ++e) o[e] = 0.0;
    if (dq)
      for (int e = 0; e < d; ++e) dq[e] = 0.0;
    for (int t = 0; t < nt; ++t) {
      tile_box tb;
      tile_of(g, t, &tb);
      if (!contains(&tb, p)) continue;
      double w = tile_weight(g, window, &tb, p);
      int r = row_of_token(&tb, p);
      double lse;
      tile_attention(g, scale, &tb, q + off, k + off, v + off, r, r + 1, Ot, &lse);
      for (int e = 0; e < d; ++e) o[e] += w * Ot[e];
      if (dq) {
        const double *qr = q + off + i * d;
        double c = w / wsum;
        for (int e = 0; e < d; ++e) dOt[e] = c * dout[off + i * d + e];
        double D = dot(dOt, Ot, d);
        for (int j = 0; j < tb.L; ++j) {
          int64_t tj = token_of_row(g, &tb, j);
          const double *kj = k + off + tj * d, *vj = v + off + tj * d;
          double P = exp(scale * dot(qr, kj, d) - lse);
          double dS = P * (dot(dOt, vj, d) - D);
          for (int e = 0; e < d; ++e) dq[e] += scale * dS * kj[e];
        }
      }
    }
    for (int e = 0; e < d; ++e) o[e] /= wsum;
    free(Ot);
    free(dOt);
  }
}

/* dK and dV for sampled keys.  keys[n] holds (b*nh + h) * N + j.  A key's
 * gradient needs every query row of every tile that covers it, so this runs
 * the full per-tile backward of those tiles (rows parallelised) and reads the
 * sampled rows out of it.  dk_rows, dv_rows are [n, d]. */
void gpa_key_rows(const int32_t *g, int window, double scale, const double *q, const double *k,
                  const double *v, const double *dout, int64_t n, const int64_t *keys,
                  double *dk_rows, double *dv_rows) {
  const int d = g[G_D], nt = gpa_num_tiles(g);
  const int64_t N = (int64_t)g[G_T] * g[G_Y] * g[G_X];
  memset(dk_rows, 0, sizeof(double) * (size_t)n * d);
  memset(dv_rows, 0, sizeof(double) * (size_t)n * d);
  /* group by (bh, tile): for each pair that covers at least one sampled key,
   * run the tile backward once with rows split across threads */
  for (int64_t bh = 0; bh < (int64_t)g[G_B] * g[G_NH]; ++bh) {
    const size_t off = (size_t)bh * N * d;
    for (int t = 0; t < nt; ++t) {
      tile_box tb;
      tile_of(g, t, &tb);
      int needed = 0;
      for (int64_t s = 0; s < n && !needed; ++s) {
        if (keys[s] / N != bh) continue;
        int p[3];
        pos_of_token(g, keys[s] % N, p);
        needed = contains(&tb, p);
      }
      if (!needed) continue;
      int nth = gpa_oracle_threads();
      double **part = (double **)calloc((size_t)nth, sizeof(double *));
#pragma omp parallel num_threads(nth)
      {
        int id = 0, cnt = 1;
#ifdef _OPENMP
        id = omp_get_thread_num();
        cnt = omp_get_num_threads();
#endif
        int r0 = (int)((int64_t)tb.L * id / cnt), r1 = (int)((int64_t)tb.L * (id + 1) / cnt);
        double *b = (double *)calloc((size_t)3 * tb.L * d, sizeof(double));
        tile_backward(g, window, scale, &tb, q + off, k + off, v + off, dout + off, r0, r1, b,
                      b + (size_t)tb.L * d, b + (size_t)2 * tb.L * d);
        part[id] = b;
      }
      for (int64_t s = 0; s < n; ++s) {
        if (keys[s] / N != bh) continue;
        int p[3];
        pos_of_token(g, keys[s] % N, p);
        if (!contains(&tb, p)) continue;
        size_t r = (size_t)row_of_token(&tb, p) * d;
        for (int id = 0; id < nth; ++id) {
          if (!part[id]) continue;
          for (int e = 0; e < d; ++e) {
            dk_rows[s * d + e] += part[id][(size_t)tb.L * d + r + e];
            dv_rows[s * d + e] += part[id][(size_t)2 * tb.L * d + r + e];
          }
        }
      }
      for (int id = 0; id < nth; ++id) free(part[id]);
      free(part);
    }
  }
}

/* Work of one (batch*head, tile) unit restricted to query rows [r0, r1):
 * the per-tile forward of those rows and their backward (which recomputes the
 * forward, as gpa_backward does).  Used only to time the
 * oracle on a bounded sample of a large workload. */
void gpa_unit_fwd_bwd(const int32_t *g, int window, double scale, const double *q,
                      const double *k, const double *v, const double *dout, int bh, int tile,
                      int r0, int r1) {
  const int d = g[G_D];
  const int64_t N = (int64_t)g[G_T] * g[G_Y] * g[G_X];
  const size_t off = (size_t)bh * N * d;
  tile_box tb;
  tile_of(g, tile, &tb);
  if (r1 > tb.L) r1 = tb.L;
  int nth = gpa_oracle_threads();
#pragma omp parallel num_threads(nth)
  {
    int id = 0, cnt = 1;
#ifdef _OPENMP
    id = omp_get_thread_num();
    cnt = omp_get_num_threads();
#endif
    int a = r0 + (int)((int64_t)(r1 - r0) * id / cnt);
    int b = r0 + (int)((int64_t)(r1 - r0) * (id + 1) / cnt);
    double *buf = (double *)calloc((size_t)3 * tb.L * d, sizeof(double));
    double *O = (double *)malloc(sizeof(double) * (size_t)(b > a ? b - a : 1) * d);
    /* the forward of these rows, then their backward (which recomputes it) */
    tile_attention(g, scale, &tb, q + off, k + off, v + off, a, b, O, NULL);
    tile_backward(g, window, scale, &tb, q + off, k + off, v + off, dout + off, a, b, buf,
                  buf + (size_t)tb.L * d, buf + (size_t)2 * tb.L * d);
    free(O);
    free(buf);
  }
}

/* Length of the extended tile (rows of its unit). */
int gpa_tile_rows(const int32_t *g, int tile) {
  tile_box tb;
  tile_of(g, tile, &tb);
  return tb.L;
}
