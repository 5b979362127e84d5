"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the attention method: it only draws
random tensors and names the workloads.  Both the oracle-based tests and the
CUDA path take their inputs from here, so the two sides see the same bytes.

The paper measures on ERA5 and HRRR reanalysis tensors (Sec. IV, Datasets),
which are not available here; the synthetic stand-ins below keep the paper's
shapes (patch-token grids of frames x latitude x longitude, Tab. III(a) uses a
32 x 64 spatial grid with long temporal context) with iid Gaussian Q, K, V.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import torch


@dataclass(frozen=True)
class Workload:
    """One synthetic GPA workload: grid, tile spec, heads and input law."""

    name: str
    B: int
    nh: int
    d: int
    grid: tuple  # (T, Y, X)
    core: tuple  # (c_t, c_y, c_x)
    halo: tuple  # (h_t, h_y, h_x)
    std: float = 1.0
    seed: int = 0
    dtype: str = "fp32"  # input dtype: "fp32" or "bf16"
    notes: str = field(default="", compare=False)

    @property
    def N(self) -> int:
        T, Y, X = self.grid
        return T * Y * X

    @property
    def shape(self):
        return (self.B, self.nh, self.N, self.d)


# The workloads the library is measured and checked on.
WORKLOADS = {
    # plain method, forward: 64 x 64 single frame, 16 tiles of 16 x 16 with a 4-token halo
    "c1_4k": Workload("c1_4k", 1, 1, 64, (1, 64, 64), (1, 16, 16), (0, 4, 4), 1.0, 20261, "fp32"),
    # 32 frames x 64 x 128 patch grid, Tiles = 16 (paper regime): core 32 x 16 x 32, halo 0/4/8
    "c2_262k_p": Workload("c2_262k_p", 4, 16, 64, (32, 64, 128), (32, 16, 32), (0, 4, 8), 0.5, 20262, "bf16"),
    # the same geometry with 1 x 4 heads (1/16 of the units, each tensor still larger than L2): profiling case
    "c2_262k_p1": Workload("c2_262k_p1", 1, 4, 64, (32, 64, 128), (32, 16, 32), (0, 4, 8), 0.5, 20262, "bf16"),
    # same grid, small tiles near the HBM/tensor ridge: core 1 x 16 x 16, halo 0/4/4
    "c2_262k_s": Workload("c2_262k_s", 4, 16, 64, (32, 64, 128), (1, 16, 16), (0, 4, 4), 0.5, 20262, "bf16"),
    # the small-tile geometry with 1 x 4 heads (1/16 of the units, each tensor 134 MB > L2): profiling case
    "c2_262k_s1": Workload("c2_262k_s1", 1, 4, 64, (32, 64, 128), (1, 16, 16), (0, 4, 4), 0.5, 20262, "bf16"),
    # long temporal context: 2048 frames x 32 x 64, d = 128, Tiles = 16 along time, halo 8 frames
    "c3_4m_p": Workload("c3_4m_p", 1, 8, 128, (2048, 32, 64), (128, 32, 64), (8, 0, 0), 0.5, 20263, "bf16"),
    # the long-context geometry with 512 frames and one head (each tensor 268 MB > L2): profiling case
    "c3_512_p1": Workload("c3_512_p1", 1, 1, 128, (512, 32, 64), (128, 32, 64), (8, 0, 0), 0.5, 20263, "bf16"),
    # gradient check size: 32 x 32, 2 heads, d = 32
    "c4_grad": Workload("c4_grad", 1, 2, 32, (1, 32, 32), (1, 16, 16), (0, 4, 4), 1.0, 20264, "fp32"),
    # backward throughput: 16 x 256 x 256, 8 heads, Tiles = 16
    "c4_1m_p": Workload("c4_1m_p", 1, 8, 64, (16, 256, 256), (16, 64, 64), (0, 8, 8), 0.5, 20264, "bf16"),
}


@dataclass(frozen=True)
class HistoryWorkload:
    """One synthetic temporal-compression workload: S history frames of a Y x X
    patch grid (M = Y * X locations), keys/values iid N(0, std^2), and one
    learned query per head iid N(0, 1) in FP32."""

    name: str
    B: int
    nh: int
    d: int
    S: int
    Y: int
    X: int
    std: float = 0.5
    seed: int = 0
    dtype: str = "bf16"

    @property
    def M(self) -> int:
        return self.Y * self.X

    @property
    def shape(self):
        return (self.B, self.nh, self.S, self.M, self.d)


HISTORY_WORKLOADS = {
    # the long-temporal-context shape (2048 frames x 32 x 64, 8 heads, d = 128) as history to compress
    "h3_2k": HistoryWorkload("h3_2k", 1, 8, 128, 2048, 32, 64, 0.5, 20266, "bf16"),
    # the same locations and heads with 512 frames (4.3 GB of keys and values): profiling case
    "h3_512": HistoryWorkload("h3_512", 1, 8, 128, 512, 32, 64, 0.5, 20266, "bf16"),
    # a long history on a few locations: 131072 frames x 8 x 8, 2 heads, d = 64 (S-long sums)
    "h_128k": HistoryWorkload("h_128k", 1, 2, 64, 131072, 8, 8, 0.5, 20267, "bf16"),
}


def history_inputs(w: HistoryWorkload, device="cpu"):
    """(q [nh, d] FP32, k, v [B, nh, S, M, d] in w.dtype) for a history workload."""
    k, v = qkv(w.shape, w.seed, w.std, w.dtype, device, n=2)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(w.seed) + 104729)
    q = torch.randn((w.nh, w.d), generator=gen, device=device, dtype=torch.float32)
    return q, k, v


def qkv(shape, seed: int, std: float = 1.0, dtype: str = "fp32", device="cpu", n: int = 3):
    """n iid N(0, std^2) tensors of `shape` from one seeded generator.

    dtype "bf16" rounds the fp32 draws to bfloat16 (round to nearest even) and
    returns bfloat16 tensors; "fp32" returns the fp32 draws.
    """
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    out = []
    for _ in range(n):
        t = torch.randn(shape, generator=gen, device=device, dtype=torch.float32)
        if std != 1.0:
            t.mul_(std)
        if dtype == "bf16":
            t = t.to(torch.bfloat16)
        elif dtype != "fp32":
            raise ValueError(dtype)
        out.append(t)
    return out


def upstream_grad(shape, seed: int, dtype: str = "fp32", device="cpu"):
    """dOut ~ iid N(0, 1), seeded independently of Q, K, V."""
    (g,) = qkv(shape, seed + 7919, 1.0, dtype, device, n=1)
    return g


def workload_inputs(w: Workload, device="cpu", with_grad: bool = True):
    """(q, k, v[, dout]) for a named workload."""
    q, k, v = qkv(w.shape, w.seed, w.std, w.dtype, device)
    if not with_grad:
        return q, k, v
    return q, k, v, upstream_grad(w.shape, w.seed, w.dtype, device)


@dataclass(frozen=True)
class ServeRequestSpec:
    """One synthetic posterior-sampling request of the serving workload."""

    arrival_s: float
    T: int  # frames; N = T * Y * X
    nh: int
    seed: int


def poisson_requests(n=256, rate=40.0, n_min=16384, n_max=2097152, frame=2048, heads=(8, 16), seed=20265):
    """Serving workload: n requests, Poisson arrivals at `rate` per second
    (seeded exponential gaps), token count N log-uniform in [n_min, n_max]
    rounded to a multiple of `frame` (one 32 x 64 frame of patch tokens),
    heads uniform over `heads`."""
    import math
    import random

    rng = random.Random(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += rng.expovariate(rate)
        N = math.exp(rng.uniform(math.log(n_min), math.log(n_max)))
        T = max(1, int(round(N / frame)))
        out.append(ServeRequestSpec(t, T, rng.choice(heads), seed * 1000 + i))
    return out


def request_state(spec: ServeRequestSpec, Y=32, X=64, d=64, std=0.5, device="cpu"):
    """Initial state z0 [nh, T*Y*X, d] BF16 of a request, iid N(0, std^2)."""
    (z,) = qkv((spec.nh, spec.T * Y * X, d), spec.seed, std, "bf16", device, n=1)
    return z


def state_pool(elems=2 * 16 * 2097152 * 64 // 2 + 1024, seed=20265, std=0.5, device="cuda"):
    """One shared buffer of iid N(0, std^2) BF16 values; request states are
    seeded slices of it (see pooled_state), so a long serving run draws its
    inputs without one allocation per request.  Default size covers the
    largest serving request (16 heads x 2,097,152 tokens x d = 64)."""
    (z,) = qkv((elems,), seed, std, "bf16", device, n=1)
    return z


def pooled_state(spec: ServeRequestSpec, pool, Y=32, X=64, d=64):
    """View [nh, T*Y*X, d] of the pool at an offset drawn from the request's seed."""
    import random

    n = spec.nh * spec.T * Y * X * d
    if n > pool.numel():
        raise ValueError("state pool too small for this request")
    off = random.Random(spec.seed).randrange(0, pool.numel() - n + 1)
    off -= off % 8  # 16-byte aligned
    return pool[off : off + n].view(spec.nh, spec.T * Y * X, d)
