/*
 * gattn.h -- C ABI of the GB300 (sm_103a) STORM global propagation attention
 * library (STORM-GPA, arXiv 2604.16590, Sec. III-C "STORM-GPA:
 * Linear-Complexity Global Attention", Fig. 3(a)).
 *
 * The operator.  Tokens live on a (T, Y, X) grid of frames x latitude x
 * longitude patches; N = T*Y*X and token i = (t*Y + y)*X + x.  The grid is
 * cut into tiles of core size core[3]; each tile is extended by halo[3]
 * tokens on both sides of every dimension (clipped to the grid), so that
 * neighbouring extended tiles overlap (Sec. III-C, first two paragraphs).
 * Softmax attention runs independently inside every extended tile, every
 * token of the tile being both a query and a key/value (Sec. III-C: interior
 * tokens attend to halo tokens; Sec. III-D Level 5: FlashAttention inside a
 * tile).  Where extended tiles overlap, the per-tile outputs are averaged
 * with Hanning weights that trust tile centres more than tile edges
 * (Sec. III-C, "average denoised outputs in overlapping halos" and the
 * closing sentence on the Hanning window):
 *
 *     O_t(i)  = sum_{j in E_t} softmax_j(s q_i.k_j) v_j          (i in E_t)
 *     Out(i)  = sum_{t : i in E_t} w_t(i) O_t(i) / sum_t w_t(i)
 *     w_t(i)  = prod_a sin^2(pi (n_a + 1/2) / (c_a + 2 h_a))
 *
 * with n_a the offset of i from the nominal (unclipped) start k_a c_a - h_a
 * of tile t in dimension a; a dimension with a single tile and no halo
 * contributes weight 1.  The paper does not print the window; this
 * half-sample Hann (strictly positive, symmetric) is the reading taken, and
 * window = GATTN_WINDOW_FLAT gives a plain mean.  One tile with no halo is
 * exact global softmax attention (Sec. IV-B: Tiles = 1 is STORM-DiT
 * without GPA).  The cost is linear in N for a fixed tile size.
 *
 * Memory layout: Q, K, V, Out, dOut, dQ, dK, dV are dense [B, nh, N, d]
 * row-major tensors (d contiguous), 16-byte aligned, in device memory owned
 * by the caller.  The library allocates nothing on the fwd/bwd path: the
 * caller passes the saved-state and workspace buffers, sized by the query
 * functions below.  Every call is asynchronous on the given CUDA stream.
 *
 * Errors.  Argument and shape errors are returned synchronously, before any
 * launch.  A failed launch returns GATTN_ERR_CUDA.  Device-side conditions
 * (a bounded wait that ran out, a debug bounds check) set a per-library
 * device status word and the kernel exits cleanly; gattn_stream_status()
 * synchronises the stream and reports and clears that word.
 */
#ifndef GATTN_H
#define GATTN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st *gattn_stream_t;

typedef enum {
  GATTN_OK = 0,
  GATTN_ERR_INVALID_ARG = 1,   /* NULL pointer, bad shape, misaligned pointer */
  GATTN_ERR_UNSUPPORTED = 2,   /* valid request this library does not implement */
  GATTN_ERR_WORKSPACE = 3,     /* saved/workspace buffer smaller than required */
  GATTN_ERR_CUDA = 4,          /* a CUDA runtime call or launch failed */
  GATTN_ERR_TIMEOUT = 5,       /* a bounded device-side wait ran out */
  GATTN_ERR_OOM = 6,           /* serving: request does not fit the HBM budget */
  GATTN_ERR_BUSY = 7,          /* serving: no free slot */
  GATTN_ERR_DEVICE_BOUNDS = 8, /* debug bounds check tripped on the device */
  GATTN_ERR_NOT_FOUND = 9      /* serving: unknown request id, or a result already taken */
} gattn_status;

typedef enum { GATTN_BF16 = 0, GATTN_FP32 = 1 } gattn_dtype;
typedef enum { GATTN_WINDOW_HANN = 0, GATTN_WINDOW_FLAT = 1 } gattn_window;

/* flags */
#define GATTN_FLAG_DEBUG_BOUNDS 0x1u /* device-side index checks on global accesses */
/* Test hook for failure detection (BF16 forward only): the MMA-issuing thread
 * of every CTA first waits on an mbarrier that nothing arrives on.  The
 * bounded wait gives up after ~20 ms, the CTA raises its abort flag, drains
 * the loads it issued, frees its tensor memory and exits; the call returns
 * GATTN_OK and gattn_stream_status() then reports GATTN_ERR_TIMEOUT.  The
 * output is not computed.  The context stays usable. */
#define GATTN_FLAG_TEST_STALL 0x2u

/*
 * Problem descriptor.
 *   B, nh, d      batch, heads, head dim.  d in {32, 64, 128} for FP32 inputs,
 *                 d in {64, 128} for BF16 inputs (tensor-core path).
 *   T, Y, X       token grid; N = T*Y*X < 2^31.
 *   core[3]       tile core size along (t, y, x), each >= 1; the last tile of a
 *                 dimension may be short when the grid is not a multiple.
 *   halo[3]       halo width along (t, y, x), each >= 0.
 *   window        gattn_window.
 *   in_dtype      dtype of Q, K, V and dOut.  GATTN_BF16 runs the tcgen05
 *                 tensor-core kernels (FP32 accumulation in TMEM);
 *                 GATTN_FP32 runs the plain FP32 SIMT kernels.
 *   out_dtype     dtype of Out, dQ, dK, dV (BF16 or FP32).
 *   scale         softmax scale s; 0 means 1/sqrt(d).
 *   flags         GATTN_FLAG_*.
 */
typedef struct {
  int32_t B, nh, d;
  int32_t T, Y, X;
  int32_t core[3];
  int32_t halo[3];
  int32_t window;
  int32_t in_dtype;
  int32_t out_dtype;
  float scale;
  uint32_t flags;
} gattn_desc;

/* Version of this ABI (bumped on any incompatible change). */
int32_t gattn_abi_version(void);

/* Human-readable name of a status code (static storage). */
const char *gattn_status_string(gattn_status s);

/* Checks a descriptor without touching the GPU. */
gattn_status gattn_validate(const gattn_desc *desc);

/* Number of tiles, prod_a ceil(G_a / core_a). Negative on an invalid desc. */
int64_t gattn_num_tiles(const gattn_desc *desc);

/* Shape (bt, by, bx) of the token boxes the tensor-core kernels cut every
 * extended tile into (bt * by * bx <= 128 tokens, one 128-row MMA block per
 * box; rows past bt * by * bx and rows outside the tile are padding).  The
 * attention work of a tile is (128 * boxes)^2 query-key pairs, so the padded
 * (executed) work of a call follows from it.  GATTN_OK, or
 * GATTN_ERR_INVALID_ARG on an invalid desc or a NULL shape. */
gattn_status gattn_block_shape(const gattn_desc *desc, int32_t shape[3]);

/*
 * Bytes of the saved-state buffer that gattn_fwd fills and gattn_bwd reads:
 * the per-(tile, row) log-sum-exp of every extended-tile row, and the FP32
 * per-tile outputs O_t of the rows covered by more than one tile (the
 * operands of the Hann-weighted merge).  Returns 0 on an invalid desc.
 */
size_t gattn_saved_bytes(const gattn_desc *desc);

/* Bytes of the backward workspace (per-row softmax statistics and the FP32
 * per-tile gradients of multiply-covered rows).  0 on an invalid desc. */
size_t gattn_bwd_workspace_bytes(const gattn_desc *desc);

/*
 * Forward: out = GPA(q, k, v).
 *   q, k, v   [B, nh, N, d] in in_dtype (device).
 *   out       [B, nh, N, d] in out_dtype (device), fully overwritten.
 *   saved     device buffer of at least gattn_saved_bytes(desc) bytes; its
 *             contents after the call are what gattn_bwd needs.
 * Launches: the tile-attention kernel (tcgen05 for BF16, SIMT for FP32),
 * then the deterministic merge of multiply-covered tokens (fixed ascending
 * tile order; no atomics, bitwise reproducible).
 */
gattn_status gattn_fwd(const gattn_desc *desc, const void *q, const void *k, const void *v,
                       void *out, void *saved, size_t saved_bytes, gattn_stream_t stream);

/*
 * Backward of the loss sum(out * dout):
 *   q, k, v   the forward's inputs (in_dtype);
 *   out       the forward's output (out_dtype);
 *   dout      upstream gradient [B, nh, N, d] in in_dtype;
 *   saved     the buffer the forward filled (unchanged since);
 *   dq,dk,dv  [B, nh, N, d] in out_dtype, fully overwritten;
 *   ws        device workspace of at least gattn_bwd_workspace_bytes(desc).
 * Per tile: dO_t = (w_t / sum w) dout, P recomputed from the saved
 * log-sum-exp (never stored), dV_t = P^T dO_t, dS = P (dO_t V^T - D),
 * dQ_t = s dS K, dK_t = s dS^T Q; each input gradient is the fixed-order sum
 * of its tiles' contributions (deterministic, no atomics).
 */
gattn_status gattn_bwd(const gattn_desc *desc, const void *q, const void *k, const void *v,
                       const void *out, const void *dout, const void *saved, size_t saved_bytes,
                       void *dq, void *dk, void *dv, void *ws, size_t ws_bytes,
                       gattn_stream_t stream);

/*
 * Serving: continuous batching of diffusion posterior-sampling requests.
 *
 * Every request carries a token state z ([nh, N, d] BF16 on a (T, Y, X) grid,
 * N = T*Y*X) and runs `steps` denoising steps
 *     z <- z + c * (GPA(z, z, z) - z)
 * (a one-layer synthetic denoiser whose output is the GPA attention of its
 * state; the per-step Hann-weighted merge is the propagation step of
 * Sec. III-C, which the paper runs once per diffusion step without extra
 * iterations).  The server keeps each active request's state on the device
 * across its steps.  An engine iteration (gattn_serve_step) admits waiting
 * requests in arrival order while the slot limit and the HBM budget allow,
 * then runs one step of every active request in one persistent ragged
 * attention launch (per-request descriptors and item offsets) followed by one
 * merge-and-update launch, both captured in a CUDA graph that is replayed
 * every iteration; requests that finish are retired: their scratch goes back
 * to the server's memory pool and their final state stays in device memory
 * until the client takes it (gattn_serve_poll with a buffer, or
 * gattn_serve_take_async) or drops it (gattn_serve_release).  Unclaimed results count against hbm_budget; when
 * the head of the queue does not fit, the oldest unclaimed results are moved
 * to host memory first.  Results do not depend on which other requests share
 * an iteration (deterministic kernels).
 * The server owns its device memory (within hbm_budget) and one internal
 * device buffer per slot of descriptors; calls on one server must not overlap.
 */
typedef struct gattn_server gattn_server;

typedef struct {
  int32_t d;                /* head dim: 64 or 128 */
  int32_t Y, X;             /* spatial grid shared by every request; T varies */
  int32_t core[3];          /* tile core (t, y, x) */
  int32_t halo[3];          /* tile halo (t, y, x) */
  int32_t window;           /* gattn_window */
  int32_t steps;            /* denoising steps per request, >= 1 */
  float c;                  /* step size of the state update */
  int32_t max_active;       /* slot limit, 1..4096 */
  int32_t use_graph;        /* 1: capture the iteration's two launches in a CUDA graph */
  size_t hbm_budget;        /* bytes of device memory the server may hold for request state */
} gattn_serve_cfg;

typedef struct {
  int32_t T;                /* frames: N = T * Y * X */
  int32_t nh;               /* heads */
  const void *z0;           /* initial state [nh, N, d] BF16 */
  int32_t z0_on_device;     /* 1: device pointer, read at admission (keep it valid until then);
                               0: host pointer, copied at submit */
} gattn_request;

typedef struct {
  int64_t submitted, admitted, completed, rejected, active, waiting;
  int64_t iterations;       /* engine iterations that ran GPU work */
  double p50_latency_s, p99_latency_s, mean_latency_s, max_latency_s;  /* submit -> final state complete */
  double token_steps;       /* sum over completed requests of nh * N * steps */
  double gpu_busy_s;        /* device time of the engine iterations */
  double wall_s;            /* host time from the first submit to the last completion */
  size_t hbm_in_use, hbm_peak;
} gattn_serve_stats_t;

/* Device memory one request holds while active (state, attention output,
 * merge scratch); 0 on an invalid request. */
size_t gattn_serve_request_bytes(const gattn_serve_cfg *cfg, int32_t T, int32_t nh);

/* `stream`: the stream engine iterations run on; NULL makes the server create
 * (and destroy) its own blocking stream (a graph cannot be captured on the
 * legacy default stream). */
gattn_status gattn_serve_create(const gattn_serve_cfg *cfg, gattn_stream_t stream, gattn_server **out);
/* Queues a request.  GATTN_ERR_OOM if it can never fit the budget,
 * GATTN_ERR_INVALID_ARG on a bad shape. */
gattn_status gattn_serve_submit(gattn_server *s, const gattn_request *req, uint64_t *id);
/* One engine iteration (admission, one step of every active request,
 * retirement); synchronises the server's stream.  *n_active receives the
 * number of active requests after the iteration, *n_waiting the queue length. */
gattn_status gattn_serve_step(gattn_server *s, int32_t *n_active, int32_t *n_waiting);
/* *done = 1 once the request finished, and then *latency_s its latency.  With
 * result_host (host or device memory, [nh, N, d] BF16; NULL: only poll) the
 * final state is copied there and released: a result can be taken once
 * (GATTN_ERR_NOT_FOUND when it was already taken or released, as for an
 * unknown id). */
gattn_status gattn_serve_poll(gattn_server *s, uint64_t id, int32_t *done, double *latency_s, void *result_host);
/* Drops the final state of a finished request without copying it (its device
 * memory returns to the pool).  GATTN_ERR_INVALID_ARG if the request has not
 * finished, GATTN_ERR_NOT_FOUND for an unknown id or a result already taken
 * or released. */
gattn_status gattn_serve_release(gattn_server *s, uint64_t id);
/* Takes the final state of a finished request without waiting for the copy:
 * starts copying its nh*N*d BF16 values to `dst` (host memory, pinned for
 * an asynchronous copy, or device memory) on a copy stream of the server and
 * returns, so that the engine's next iterations run while the result moves.
 * `dst` must stay valid and must not be read until gattn_serve_copied reports
 * the copy complete; the result's device memory returns to the pool at the
 * first gattn_serve_step or gattn_serve_copied after that.  A result can be
 * taken once, by this call or by gattn_serve_poll.  Errors:
 * GATTN_ERR_INVALID_ARG (NULL arguments, request not finished),
 * GATTN_ERR_NOT_FOUND (unknown id, result already taken or released),
 * GATTN_ERR_CUDA. */
gattn_status gattn_serve_take_async(gattn_server *s, uint64_t id, void *dst);
/* *copied = 1 once the result of `id` has been taken and its copy is complete
 * (immediately for gattn_serve_poll, which copies before returning), else 0.
 * GATTN_ERR_NOT_FOUND for an unknown id. */
gattn_status gattn_serve_copied(gattn_server *s, uint64_t id, int32_t *copied);
gattn_status gattn_serve_stats(gattn_server *s, gattn_serve_stats_t *out);
void gattn_serve_destroy(gattn_server *s);

/*
 * Forward without a caller-provided saved buffer, for callers that cannot
 * allocate device memory: code that runs under a memory manager which owns
 * all of HBM after start-up (a serving process that partitions the device up
 * front, or a host framework whose operator interface passes only input and
 * output tensors) has no way to obtain the scratch gattn_fwd needs.  This
 * entry point has no counterpart in the paper.
 *
 * Same computation and arguments as gattn_fwd minus `saved`: the forward's
 * scratch lives in a device array of GATTN_NOALLOC_SCRATCH_BYTES that every
 * GPU loading this library holds until the process exits.  Problems whose
 * gattn_saved_bytes(desc) exceeds that size are rejected with
 * GATTN_ERR_WORKSPACE before any launch.  The call itself allocates nothing
 * (no cudaMalloc / cudaFree or allocating library routine).
 *
 * The first call on a device looks up the array's device address on that
 * device (cudaGetSymbolAddress) and caches it; make that first call before
 * any stream capture.  With CUDA's default lazy module loading the driver
 * allocates the device copy of the array at that first lookup, not when the
 * library is loaded: a caller whose memory manager takes all of HBM makes
 * one call on each device before it does (a small problem is enough), or
 * runs with CUDA_MODULE_LOADING=EAGER so that the array is placed when the
 * context is created.  From then on calls allocate nothing.  The cached
 * address belongs to the device's primary context: after cudaDeviceReset on
 * that device it is stale, and this entry point must not be called again in
 * that process.  All calls share the one array and it keeps the last
 * call's contents (no call depends on them: everything read is written
 * first in the same call).  Calls whose work overlaps on the GPU -- on
 * different streams, or from different host threads -- race on the array:
 * serialise them.  The result cannot be passed to gattn_bwd (the saved state
 * is not the caller's).
 */
#define GATTN_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
gattn_status gattn_fwd_noalloc(const gattn_desc *desc, const void *q, const void *k, const void *v,
                               void *out, gattn_stream_t stream);

/*
 * Factorised linear attention.  Not an operator of the paper (its global
 * attention is the tiled operator above): the textbook linear-complexity
 * global attention in which keys and values over all N tokens are reduced
 * into a fixed-size per-head summary and normaliser that every query reads.
 * Feature map phi(x) = elu(x) + 1 (Katharopoulos et al., 2020):
 *
 *     S = sum_n phi(k_n) v_n^T,   z = sum_n phi(k_n),
 *     out_i = phi(q_i)^T S / (phi(q_i)^T z).
 *
 * q, k, v, out: [B, nh, N, d] BF16 (device), d = 64, N < 2^31.  ws: device
 * workspace of gattn_linear_workspace_bytes(desc) bytes (per-chunk FP32
 * partial summaries, the combined summary).  Launches: a split-N summary
 * kernel (TMA tiles, phi in shared memory, S accumulated by tcgen05 in TMEM,
 * z in FP32 registers), a fixed-order compensated combine of the chunk
 * partials, and a query pass (tcgen05 phi(Q) S with S split into BF16 high
 * and low parts, FP32 denominator).  Deterministic.  The workspace keeps the
 * combined summary (S^T as BF16 high and low parts, z) for the backward.
 */
typedef struct {
  int32_t B, nh, d;
  int64_t N;
  int32_t in_dtype, out_dtype;  /* GATTN_BF16 */
} gattn_linear_desc;

size_t gattn_linear_workspace_bytes(const gattn_linear_desc *desc);
gattn_status gattn_linear_fwd(const gattn_linear_desc *desc, const void *q, const void *k, const void *v,
                              void *out, void *ws, size_t ws_bytes, gattn_stream_t stream);

/*
 * Backward of the loss sum(out * dout) of the factorised linear attention,
 * with den_i = phi(q_i) . z and phi'(x) = 1 (x > 0), exp(x) (x <= 0):
 *
 *     dq_i = (S^T dout_i - z (dout_i . out_i)) / den_i * phi'(q_i)
 *     dS   = sum_i phi(q_i) (dout_i / den_i)^T       (query-side gradient summary)
 *     dz   = -sum_i phi(q_i) (dout_i . out_i) / den_i
 *     dk_n = (dS v_n + dz) * phi'(k_n),   dv_n = dS^T phi(k_n)
 *
 * (dout_i . out_i is recomputed as phi(q_i) . S^T dout_i / den_i; out is not
 * read).  Not an operator of the paper, like the forward.
 *   q, k, v, dout  [B, nh, N, d] BF16 (device), d = 64.
 *   saved          the workspace gattn_linear_fwd filled for these q, k, v,
 *                  unchanged since (its combined S and z are read);
 *                  saved_bytes >= gattn_linear_workspace_bytes(desc).
 *   dq, dk, dv     [B, nh, N, d] BF16 (device), fully overwritten.
 *   ws             device workspace of gattn_linear_bwd_workspace_bytes(desc)
 *                  bytes (per-chunk FP32 partials of dS and dz, the combined
 *                  dS as BF16 high and low parts).
 * Launches: a query pass (tcgen05 products S^T dout and phi(Q)^T (dout / den)
 * with BF16 high and low parts of both factors; dq; split-N partials of dS and
 * dz), a fixed-order compensated combine, and a key pass (tcgen05 products
 * V dS^T and phi(K) dS; dk, dv).  Deterministic.  All pointers 16-byte
 * aligned.  GATTN_ERR_INVALID_ARG on a bad desc or pointer,
 * GATTN_ERR_WORKSPACE when saved or ws is short, GATTN_ERR_CUDA when a launch
 * fails.
 */
size_t gattn_linear_bwd_workspace_bytes(const gattn_linear_desc *desc);
gattn_status gattn_linear_bwd(const gattn_linear_desc *desc, const void *q, const void *k, const void *v,
                              const void *dout, const void *saved, size_t saved_bytes, void *dq, void *dk,
                              void *dv, void *ws, size_t ws_bytes, gattn_stream_t stream);

/*
 * One diffusion posterior-sampling step with the GPA denoiser (arXiv
 * 2604.16590, Sec. III-A: the reverse SDE, the decomposition of the posterior
 * score into prior and likelihood scores, the DPS likelihood score, and the
 * prior score from the denoiser, Eq. denoise; Sec. III-C: the per-step merge
 * is what propagates context across tiles).  With D(z) = GPA(z, z, z) (a
 * synthetic one-layer denoiser; heads act as channels) and a token mask H:
 *
 *     S      = (D(z) - z) / sigma^2 - lam J_D(z)^T H^T (H D(z) - y)
 *     z_next = z + delta S + sqrt(delta) eps,   delta = sigma^2 - sigma_next^2
 *
 * (Euler-Maruyama step of the variance-exploding reverse SDE; lam folds the
 * guidance weight zeta_t, the factor 2 and the observation-error variance).
 *   desc      the GPA problem; out_dtype must be GATTN_FP32 (D and the
 *             gradients are kept in FP32); in_dtype BF16 runs the tensor-core
 *             attention on zb, FP32 the plain form on z.
 *   z         [B, nh, N, d] FP32 state (device), updated in place.
 *   zb        [B, nh, N, d] BF16 copy of z (device; BF16 form only, else
 *             ignored): read as the attention input, rewritten as bf16(z_next).
 *   y         [B, nh, N, d] FP32 observations (read where the mask is set).
 *   mask      [B, N] uint8, nonzero where a token is observed.
 *   eps       [B, nh, N, d] FP32 standard normal noise for this step.
 *   ws        device workspace of gattn_dps_workspace_bytes(desc) bytes.
 * Launches: the GPA forward, the residual kernel, the GPA backward with
 * dOut = the residual, the update kernel.
 */
typedef struct {
  float sigma;       /* current noise level (> 0) */
  float sigma_next;  /* next noise level (0 <= sigma_next <= sigma) */
  float lam;         /* likelihood guidance weight */
} gattn_dps_params;

size_t gattn_dps_workspace_bytes(const gattn_desc *desc);
gattn_status gattn_dps_step(const gattn_desc *desc, const gattn_dps_params *params, float *z, void *zb,
                            const float *y, const uint8_t *mask, const float *eps, void *ws, size_t ws_bytes,
                            gattn_stream_t stream);

/*
 * Noise-gated self + cross attention (arXiv 2604.16590, Sec. III-B, the
 * STORM-DiT layer and the noise-gated attention paragraph): each layer runs
 * spatial self-attention on the current state and cross-attention from the
 * current state to the compressed temporal representation, and blends them
 * with a gate set by the diffusion noise level (more weight on the temporal
 * branch at high noise).  With GPA tiling both branches are tile-local:
 *
 *     out = g_h GPA(q, k, v) + (1 - g_h) GPA(q, kc, vc)
 *
 * q, k, v from the current state and kc, vc from the temporal representation,
 * all [B, nh, N, d] in in_dtype on the same grid and tiling (desc); gate [nh]
 * FP32 on the device (the caller maps sigma_t to g; the paper does not give
 * the map).  out [B, nh, N, d] in out_dtype.  Forward only.
 * ws: device workspace of gattn_gated_workspace_bytes(desc) bytes (the
 * attention saved state, reused by both branches, and the cross branch's
 * output).  Launches: both GPA forwards, then one blend kernel.
 */
size_t gattn_gated_workspace_bytes(const gattn_desc *desc);
gattn_status gattn_gated_fwd(const gattn_desc *desc, const void *q, const void *k, const void *v,
                             const void *kc, const void *vc, const float *gate, void *out,
                             void *ws, size_t ws_bytes, gattn_stream_t stream);

/*
 * Temporal compression (arXiv 2604.16590, Sec. III-B, the STORM-DiT
 * architecture paragraph and Fig. 2(b)): history states are folded into one
 * global temporal representation by cross-attention across the temporal
 * dimension.  At every spatial location m a learned query per head attends
 * over the S history frames of that location and returns one token:
 *
 *     out[b,h,m] = sum_t softmax_t(scale q_h . k[b,h,t,m]) v[b,h,t,m]
 *     lse[b,h,m] = log sum_t exp(scale q_h . k[b,h,t,m])
 *
 * The same call aggregates the variable dimension (S = number of variables,
 * M = tokens per variable).  The cost is linear in S: every history token is
 * read once, and the pass is bound by HBM bandwidth.
 *
 *   B, nh, d   batch, heads, head dim: d in {64, 128} for BF16 inputs,
 *              {32, 64, 128} for FP32 inputs.
 *   S          frames pooled per location (>= 1).
 *   M          locations per frame (>= 1), e.g. Y * X.
 *   in_dtype   dtype of k and v; out_dtype the dtype of out.
 *   scale      softmax scale; 0 means 1/sqrt(d).
 */
typedef struct {
  int32_t B, nh, d;
  int32_t S, M;
  int32_t in_dtype;
  int32_t out_dtype;
  float scale;
} gattn_compress_desc;

/* Bytes of the workspace gattn_compress_fwd needs: nonzero when the frames
 * are split into ranges to fill the GPU (few locations, long histories);
 * then it holds FP32 per-range partials.  0 also on an invalid desc. */
size_t gattn_compress_workspace_bytes(const gattn_compress_desc *desc);

/*
 * Forward of the temporal compression.
 *   q     [nh, d] FP32 learned queries (device).
 *   k, v  [B, nh, S, M, d] in in_dtype (device), location m contiguous within
 *         a frame.
 *   out   [B, nh, M, d] in out_dtype (device), fully overwritten.
 *   lse   [B, nh, M] FP32 natural-log normaliser (device), or NULL.
 *   ws    device workspace of gattn_compress_workspace_bytes(desc) bytes
 *         (may be NULL when that is 0).
 * All pointers 16-byte aligned (lse 4-byte).  One streaming kernel (online
 * softmax, S-long sums compensated by 256-frame blocking); when the frames
 * are split, a second kernel merges the ranges in fixed order.  Deterministic.
 * GATTN_ERR_INVALID_ARG on a bad desc or pointer, GATTN_ERR_WORKSPACE when the
 * workspace is missing or short, GATTN_ERR_CUDA when a launch fails.
 */
gattn_status gattn_compress_fwd(const gattn_compress_desc *desc, const float *q, const void *k, const void *v,
                                void *out, float *lse, void *ws, size_t ws_bytes, gattn_stream_t stream);

/* Synchronises `stream`, then returns (and clears) the device status word of
 * this library on the current device: GATTN_OK, GATTN_ERR_TIMEOUT or
 * GATTN_ERR_DEVICE_BOUNDS; GATTN_ERR_CUDA if the stream reported an error. */
gattn_status gattn_stream_status(gattn_stream_t stream);

/*
 * Per-kernel device timing (diagnostics, used by the benchmark).  While
 * enabled, every kernel launch of this library is bracketed by a pair of CUDA
 * events recorded on its launch stream.  gattn_profile_read synchronises on
 * those events and returns, per kernel name, the number of launches and the
 * summed device time since the last enable.  Host-side state, process-wide,
 * guarded by a mutex; at most 65536 launches are recorded per enable.
 */
typedef struct {
  char name[24];    /* "fwd_tiles", "merge_fwd", "bwd_prep", "bwd_dkdv", "bwd_dq", "merge_bwd",
                       "compress", "compress_combine", "gated_mix", "dps_residual", "dps_update",
                       "linear_summary", "linear_combine", "linear_query", "linear_bwd_query",
                       "linear_bwd_combine", "linear_bwd_key" */
  int64_t launches;
  double total_ms;
} gattn_kernel_stat;

/* enable != 0 clears the record and starts recording; 0 stops. */
gattn_status gattn_profile_enable(int32_t enable);

/* Fills up to `max` entries; returns the number of kernel names recorded, or
 * a negative gattn_status on a CUDA error. */
int32_t gattn_profile_read(gattn_kernel_stat *out, int32_t max);

#ifdef __cplusplus
}
#endif

#endif /* GATTN_H */
