// simt_fp32.cu -- the plain FP32 form of STORM-GPA tile attention (CUDA cores,
// no tensor cores): forward (online softmax, Sec. III-C / III-D Level 5) and
// the two backward kernels (dQ per query row, dK/dV per key row).  This is
// the FP32 baseline the BF16 tensor-core form is measured against, and the
// path used when the inputs are FP32.
//
// Work decomposition: one CTA of 128 threads per (row block, tile, batch*head);
// each row of the extended tile is owned by TPR = D/DPT consecutive lanes,
// each lane holding DPT = 16 of the D head dimensions in registers; partial
// dot products are combined with warp shuffles.  Keys (or queries, for dK/dV)
// stream through shared memory in chunks of KC rows; every chunk is reduced
// locally before it is folded into the running sums (two-level summation,
// which keeps the FP32 error of L-long sums near eps * (sqrt(KC) + sqrt(L/KC))).
#include "internal.cuh"

GATTN_DEFINE_STATUS(simt)

namespace gattn {
namespace {

constexpr int kThreads = 128;
constexpr int kDPT = 16;  // head dims per lane
constexpr int kKC = 32;   // rows per shared-memory chunk

// Physical float4 slot of lane group `grp`'s f-th float4 in a staged row:
// spreads the groups of one quarter-warp over distinct shared-memory banks.
__device__ __forceinline__ int swz(int grp, int f) { return 4 * grp + (f ^ ((grp >> 1) & 3)); }

// Stage rows [j0, j0+KC) of the tile from two [N, D] tensors into shared memory.
template <int D>
__device__ __forceinline__ void stage_rows(const Geom& g, const TileBox& tb, int j0, const float* __restrict__ A,
                                           const float* __restrict__ Bm, float* As, float* Bs) {
  constexpr int F4 = D / 4;
  for (int idx = threadIdx.x; idx < kKC * F4; idx += kThreads) {
    int jj = idx / F4, F = idx % F4;
    int j = j0 + jj;
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
    if (j < tb.L) {
      int64_t tok = tile_token(g, tb, j);
      a = __ldg(reinterpret_cast<const float4*>(A + tok * D) + F);
      b = __ldg(reinterpret_cast<const float4*>(Bm + tok * D) + F);
    }
    int p = swz(F / 4, F % 4);
    reinterpret_cast<float4*>(As + jj * D)[p] = a;
    reinterpret_cast<float4*>(Bs + jj * D)[p] = b;
  }
}

template <int D>
__device__ __forceinline__ float dot_group(const float (&x)[kDPT], const float* row, int grp) {
  float s = 0.f;
#pragma unroll
  for (int f = 0; f < kDPT / 4; ++f) {
    float4 k4 = reinterpret_cast<const float4*>(row)[swz(grp, f)];
    s = fmaf(x[4 * f + 0], k4.x, s);
    s = fmaf(x[4 * f + 1], k4.y, s);
    s = fmaf(x[4 * f + 2], k4.z, s);
    s = fmaf(x[4 * f + 3], k4.w, s);
  }
  return s;
}

template <int TPR>
__device__ __forceinline__ float group_sum(float s) {
#pragma unroll
  for (int o = 1; o < TPR; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

template <int D>
__device__ __forceinline__ void axpy_group(float (&acc)[kDPT], float a, const float* row, int grp) {
#pragma unroll
  for (int f = 0; f < kDPT / 4; ++f) {
    float4 v4 = reinterpret_cast<const float4*>(row)[swz(grp, f)];
    acc[4 * f + 0] = fmaf(a, v4.x, acc[4 * f + 0]);
    acc[4 * f + 1] = fmaf(a, v4.y, acc[4 * f + 1]);
    acc[4 * f + 2] = fmaf(a, v4.z, acc[4 * f + 2]);
    acc[4 * f + 3] = fmaf(a, v4.w, acc[4 * f + 3]);
  }
}

__device__ __forceinline__ void load_group(float (&x)[kDPT], const float* __restrict__ src) {
#pragma unroll
  for (int f = 0; f < kDPT / 4; ++f) {
    float4 t = __ldg(reinterpret_cast<const float4*>(src) + f);
    x[4 * f + 0] = t.x;
    x[4 * f + 1] = t.y;
    x[4 * f + 2] = t.z;
    x[4 * f + 3] = t.w;
  }
}

template <typename T>
__device__ __forceinline__ void store_group(T* dst, const float (&x)[kDPT], float mul) {
#pragma unroll
  for (int f = 0; f < kDPT / 4; ++f)
    store4<T>(dst + 4 * f, make_float4(x[4 * f] * mul, x[4 * f + 1] * mul, x[4 * f + 2] * mul, x[4 * f + 3] * mul));
}

// ---------------------------------------------------------------- forward
template <int D, typename OutT>
__global__ void __launch_bounds__(kThreads) simt_fwd_kernel(Geom g, const float* __restrict__ Q,
                                                            const float* __restrict__ K,
                                                            const float* __restrict__ V, OutT* __restrict__ out,
                                                            float* __restrict__ lse2, float* __restrict__ ot) {
  constexpr int TPR = D / kDPT, RPC = kThreads / TPR;
  __shared__ __align__(16) float Ks[kKC * D];
  __shared__ __align__(16) float Vs[kKC * D];
  const int tile = blockIdx.y, bh = blockIdx.z;
  TileBox tb;
  tile_box(g, tile, tb);
  const int row0 = blockIdx.x * RPC;
  if (row0 >= tb.L) return;  // uniform over the CTA
  const int grp = threadIdx.x % TPR;
  const int r = row0 + threadIdx.x / TPR;
  const bool active = r < tb.L;
  const int64_t base = (int64_t)bh * g.N * D;
  const float* Qb = Q + base;
  const float* Kb = K + base;
  const float* Vb = V + base;
  int64_t tok = active ? tile_token(g, tb, r) : 0;

  float q[kDPT], o[kDPT], oc[kDPT];
  if (active) load_group(q, Qb + tok * D + grp * kDPT);
  else
#pragma unroll
    for (int e = 0; e < kDPT; ++e) q[e] = 0.f;
#pragma unroll
  for (int e = 0; e < kDPT; ++e) o[e] = 0.f;
  float m = -INFINITY, l = 0.f;

  for (int j0 = 0; j0 < tb.L; j0 += kKC) {
    __syncthreads();
    stage_rows<D>(g, tb, j0, Kb, Vb, Ks, Vs);
    __syncthreads();
    float s[kKC];
    float cmax = -INFINITY;
#pragma unroll
    for (int jj = 0; jj < kKC; ++jj) {
      float d = group_sum<TPR>(dot_group<D>(q, Ks + jj * D, grp));
      s[jj] = (j0 + jj < tb.L) ? d * g.scale_log2 : -INFINITY;
      cmax = fmaxf(cmax, s[jj]);
    }
    const float mnew = fmaxf(m, cmax);
    const float alpha = exp2f(m - mnew);  // 0 on the first chunk (m = -inf)
    float lc = 0.f;
#pragma unroll
    for (int e = 0; e < kDPT; ++e) oc[e] = 0.f;
#pragma unroll
    for (int jj = 0; jj < kKC; ++jj) {
      float p = exp2f(s[jj] - mnew);
      lc += p;
      axpy_group<D>(oc, p, Vs + jj * D, grp);
    }
    l = l * alpha + lc;
#pragma unroll
    for (int e = 0; e < kDPT; ++e) o[e] = o[e] * alpha + oc[e];
    m = mnew;
  }
  if (!active) return;
  const float inv = 1.f / l;
  int lr[3];
  tile_local(tb, r, lr);
  const int64_t slot = slot_of(g, bh, tile, tb.e, lr);
  if (grp == 0) lse2[slot] = m + log2f(l);
  int p[3];
  token_pos(g, tok, p);
  if (single_cover(g, p)) {
    store_group<OutT>(out + base + tok * D + grp * kDPT, o, inv);
  } else {
    store_group<float>(ot + slot * D + grp * kDPT, o, inv);
  }
}

// ---------------------------------------------------------------- backward: dQ
// P = exp2(s q.k log2e - lse') already carries the merge weight w_t / sum w,
// so dS = P (dOut.v - D) and dQ_t = s sum_j dS k_j (the workspace holds -lse'
// and -D).
template <int D, typename OutT>
__global__ void __launch_bounds__(kThreads) simt_dq_kernel(Geom g, const float* __restrict__ Q,
                                                           const float* __restrict__ K,
                                                           const float* __restrict__ V,
                                                           const float* __restrict__ dO,
                                                           const float* __restrict__ lse2c,
                                                           const float* __restrict__ dd, OutT* __restrict__ dq,
                                                           float* __restrict__ dq_s) {
  constexpr int TPR = D / kDPT, RPC = kThreads / TPR;
  __shared__ __align__(16) float Ks[kKC * D];
  __shared__ __align__(16) float Vs[kKC * D];
  const int tile = blockIdx.y, bh = blockIdx.z;
  TileBox tb;
  tile_box(g, tile, tb);
  const int row0 = blockIdx.x * RPC;
  if (row0 >= tb.L) return;
  const int grp = threadIdx.x % TPR;
  const int r = row0 + threadIdx.x / TPR;
  const bool active = r < tb.L;
  const int64_t base = (int64_t)bh * g.N * D;
  int64_t tok = active ? tile_token(g, tb, r) : 0;
  int lr[3];
  tile_local(tb, active ? r : 0, lr);
  const int64_t slot = slot_of(g, bh, tile, tb.e, lr);

  float q[kDPT], go[kDPT], acc[kDPT], accc[kDPT];
  if (active) {
    load_group(q, Q + base + tok * D + grp * kDPT);
    load_group(go, dO + base + tok * D + grp * kDPT);
  } else {
#pragma unroll
    for (int e = 0; e < kDPT; ++e) q[e] = go[e] = 0.f;
  }
  const float nL = active ? lse2c[slot] : -INFINITY;  // -lse' (negated in the workspace)
  const float nD = active ? dd[slot] : 0.f;           // -D
#pragma unroll
  for (int e = 0; e < kDPT; ++e) acc[e] = 0.f;

  for (int j0 = 0; j0 < tb.L; j0 += kKC) {
    __syncthreads();
    stage_rows<D>(g, tb, j0, K + base, V + base, Ks, Vs);
    __syncthreads();
#pragma unroll
    for (int e = 0; e < kDPT; ++e) accc[e] = 0.f;
#pragma unroll 8
    for (int jj = 0; jj < kKC; ++jj) {
      float sk = dot_group<D>(q, Ks + jj * D, grp);
      float dp = dot_group<D>(go, Vs + jj * D, grp);
      sk = group_sum<TPR>(sk);
      dp = group_sum<TPR>(dp);
      float p = (j0 + jj < tb.L) ? exp2f(fmaf(sk, g.scale_log2, nL)) : 0.f;
      float ds = p * (dp + nD);
      axpy_group<D>(accc, ds, Ks + jj * D, grp);
    }
#pragma unroll
    for (int e = 0; e < kDPT; ++e) acc[e] += accc[e];
  }
  if (!active) return;
  int p[3];
  token_pos(g, tok, p);
  if (single_cover(g, p)) store_group<OutT>(dq + base + tok * D + grp * kDPT, acc, g.scale);
  else store_group<float>(dq_s + slot * D + grp * kDPT, acc, g.scale);
}

// ---------------------------------------------------------------- backward: dK, dV
// One row per key j: dV_t(j) = sum_i P_ij dOut_i, dK_t(j) = s sum_i dS_ij q_i.
template <int D, typename OutT>
__global__ void __launch_bounds__(kThreads) simt_dkdv_kernel(Geom g, const float* __restrict__ Q,
                                                             const float* __restrict__ K,
                                                             const float* __restrict__ V,
                                                             const float* __restrict__ dO,
                                                             const float* __restrict__ lse2c,
                                                             const float* __restrict__ dd, OutT* __restrict__ dk,
                                                             OutT* __restrict__ dv, float* __restrict__ dk_s,
                                                             float* __restrict__ dv_s) {
  constexpr int TPR = D / kDPT, RPC = kThreads / TPR;
  __shared__ __align__(16) float Qs[kKC * D];
  __shared__ __align__(16) float Os[kKC * D];
  __shared__ float Ls[kKC];
  __shared__ float Ds[kKC];
  const int tile = blockIdx.y, bh = blockIdx.z;
  TileBox tb;
  tile_box(g, tile, tb);
  const int row0 = blockIdx.x * RPC;
  if (row0 >= tb.L) return;
  const int grp = threadIdx.x % TPR;
  const int r = row0 + threadIdx.x / TPR;
  const bool active = r < tb.L;
  const int64_t base = (int64_t)bh * g.N * D;
  int64_t tok = active ? tile_token(g, tb, r) : 0;

  float kr[kDPT], vr[kDPT], adk[kDPT], adv[kDPT], cdk[kDPT], cdv[kDPT];
  if (active) {
    load_group(kr, K + base + tok * D + grp * kDPT);
    load_group(vr, V + base + tok * D + grp * kDPT);
  } else {
#pragma unroll
    for (int e = 0; e < kDPT; ++e) kr[e] = vr[e] = 0.f;
  }
#pragma unroll
  for (int e = 0; e < kDPT; ++e) adk[e] = adv[e] = 0.f;

  for (int i0 = 0; i0 < tb.L; i0 += kKC) {
    __syncthreads();
    stage_rows<D>(g, tb, i0, Q + base, dO + base, Qs, Os);
    if (threadIdx.x < kKC) {
      int i = i0 + threadIdx.x;
      int li[3];
      tile_local(tb, i < tb.L ? i : 0, li);
      int64_t s = slot_of(g, bh, tile, tb.e, li);
      Ls[threadIdx.x] = i < tb.L ? lse2c[s] : -INFINITY;  // -lse'
      Ds[threadIdx.x] = i < tb.L ? dd[s] : 0.f;           // -D
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < kDPT; ++e) cdk[e] = cdv[e] = 0.f;
#pragma unroll 4
    for (int ii = 0; ii < kKC; ++ii) {
      float sk = dot_group<D>(kr, Qs + ii * D, grp);
      float dp = dot_group<D>(vr, Os + ii * D, grp);
      sk = group_sum<TPR>(sk);
      dp = group_sum<TPR>(dp);
      float p = exp2f(fmaf(sk, g.scale_log2, Ls[ii]));
      float ds = p * (dp + Ds[ii]);
      axpy_group<D>(cdv, p, Os + ii * D, grp);
      axpy_group<D>(cdk, ds, Qs + ii * D, grp);
    }
#pragma unroll
    for (int e = 0; e < kDPT; ++e) {
      adk[e] += cdk[e];
      adv[e] += cdv[e];
    }
  }
  if (!active) return;
  int lr[3];
  tile_local(tb, r, lr);
  const int64_t slot = slot_of(g, bh, tile, tb.e, lr);
  int p[3];
  token_pos(g, tok, p);
  if (single_cover(g, p)) {
    store_group<OutT>(dk + base + tok * D + grp * kDPT, adk, g.scale);
    store_group<OutT>(dv + base + tok * D + grp * kDPT, adv, 1.f);
  } else {
    store_group<float>(dk_s + slot * D + grp * kDPT, adk, g.scale);
    store_group<float>(dv_s + slot * D + grp * kDPT, adv, 1.f);
  }
}

template <int D, typename OutT>
cudaError_t simt_fwd_dispatch(const Geom& g, const float* q, const float* k, const float* v, void* out,
                              float* lse2, float* ot, cudaStream_t st) {
  constexpr int RPC = kThreads / (D / kDPT);
  dim3 grid((g.Lmax + RPC - 1) / RPC, g.ntiles, g.B * g.nh);
  simt_fwd_kernel<D, OutT><<<grid, kThreads, 0, st>>>(g, q, k, v, static_cast<OutT*>(out), lse2, ot);
  return cudaGetLastError();
}

template <int D, typename OutT>
cudaError_t simt_bwd_dispatch(const Geom& g, const float* q, const float* k, const float* v, const float* dout,
                              const float* lse2c, const float* dd, void* dq, void* dk, void* dv, float* dq_s,
                              float* dk_s, float* dv_s, cudaStream_t st) {
  constexpr int RPC = kThreads / (D / kDPT);
  dim3 grid((g.Lmax + RPC - 1) / RPC, g.ntiles, g.B * g.nh);
  prof_begin(kKBwdDq, st);
  simt_dq_kernel<D, OutT><<<grid, kThreads, 0, st>>>(g, q, k, v, dout, lse2c, dd, static_cast<OutT*>(dq), dq_s);
  prof_end(kKBwdDq, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  prof_begin(kKBwdDkdv, st);
  simt_dkdv_kernel<D, OutT><<<grid, kThreads, 0, st>>>(g, q, k, v, dout, lse2c, dd, static_cast<OutT*>(dk),
                                                       static_cast<OutT*>(dv), dk_s, dv_s);
  prof_end(kKBwdDkdv, st);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_simt_fwd(const Geom& g, const float* q, const float* k, const float* v, void* out,
                            int out_dtype, float* lse2, float* ot, cudaStream_t st) {
  const bool bf = out_dtype == GATTN_BF16;
  switch (g.d) {
    case 32:
      return bf ? simt_fwd_dispatch<32, __nv_bfloat16>(g, q, k, v, out, lse2, ot, st)
                : simt_fwd_dispatch<32, float>(g, q, k, v, out, lse2, ot, st);
    case 64:
      return bf ? simt_fwd_dispatch<64, __nv_bfloat16>(g, q, k, v, out, lse2, ot, st)
                : simt_fwd_dispatch<64, float>(g, q, k, v, out, lse2, ot, st);
    case 128:
      return bf ? simt_fwd_dispatch<128, __nv_bfloat16>(g, q, k, v, out, lse2, ot, st)
                : simt_fwd_dispatch<128, float>(g, q, k, v, out, lse2, ot, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_simt_bwd(const Geom& g, const float* q, const float* k, const float* v, const float* dout,
                            const float* lse2c, const float* dd, void* dq, void* dk, void* dv, int out_dtype,
                            float* dq_s, float* dk_s, float* dv_s, cudaStream_t st) {
  const bool bf = out_dtype == GATTN_BF16;
#define GATTN_SIMT_BWD(DD)                                                                                 \
  return bf ? simt_bwd_dispatch<DD, __nv_bfloat16>(g, q, k, v, dout, lse2c, dd, dq, dk, dv, dq_s, dk_s, dv_s, st) \
            : simt_bwd_dispatch<DD, float>(g, q, k, v, dout, lse2c, dd, dq, dk, dv, dq_s, dk_s, dv_s, st);
  switch (g.d) {
    case 32: GATTN_SIMT_BWD(32)
    case 64: GATTN_SIMT_BWD(64)
    case 128: GATTN_SIMT_BWD(128)
  }
#undef GATTN_SIMT_BWD
  return cudaErrorInvalidValue;
}

}  // namespace gattn
