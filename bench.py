"""Benchmark of the STORM-GPA hot path (arXiv 2604.16590, Sec. III-C) on GB300.

One step = one forward + backward of the halo-tiled global propagation
attention over one batch of synthetic tokens, through the C ABI of libgattn
(gattn_fwd + gattn_bwd: tile kernels, Hann-weighted merge, backward prep,
dK/dV and dQ kernels, gradient merge).  Default workload: 32 frames x 64 x 128
lat-lon patch tokens (N = 262,144), batch 4, 16 heads, d = 64, BF16 inputs
iid N(0, 0.5), upstream gradient iid N(0, 1), Tiles = 16 (core 32x16x32,
halo 0/4/8).  Q, K, V are 6.4 GB (> L2), so no L2 flush is needed.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gattn|reference]

N > 1 runs under torchrun, one rank per GPU: every rank runs its own replica
of the workload (independent (batch, head) units; no collective on the data
path) -> weak scaling.  --impl reference times the FP64 CPU oracle on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "global-attn fwd+bwd Gtokens/s & HBM-roofline %, BF16 vs FP32; serve p50/p99"
UNIT = "Gtokens/s"
# dram__bytes_read.sum + dram__bytes_write.sum per launch of a leg's dominant
# kernel, from the ncu captures summarised in profiles/; None for a kernel
# that changed since its counters were taken.
TRAFFIC_PER_LAUNCH = {
    # dkdv64: 1539.3 MB in one ncu capture of the same geometry with 1/16 of the
    # (batch*head) units (c2_262k_p1), times 16 (the units are independent)
    ("c2_262k_p", "bwd_dkdv"): 24.63e9,
}
# MUFU ex2 results per clock per SM (measured on GB300 with a micro-benchmark:
# 32 per clock, i.e. 8 per SM sub-partition), the exponential-unit peak of the
# attainable-time bound.
EX2_PER_CLK_SM = 32


def _extents(G, c, h):
    return [min((k + 1) * c + h, G) - max(k * c - h, 0) for k in range(-(-G // c))]


def sum_L2(w):
    """sum over tiles of L_t^2 (separable over the three dimensions)."""
    out = 1
    for a in range(3):
        out *= sum(e * e for e in _extents(w.grid[a], w.core[a], w.halo[a]))
    return out


def sum_L(w):
    out = 1
    for a in range(3):
        out *= sum(_extents(w.grid[a], w.core[a], w.halo[a]))
    return out


def padded_pairs(w, box):
    """Query-key pairs the tensor-core kernels execute per (batch, head): every
    tile is cut into prod_a ceil(e_a / b_a) boxes of one 128-row MMA block
    each, and all (query block, key block) pairs of a tile are computed."""
    out = 128 * 128
    for a in range(3):
        out *= sum((-(-e // box[a])) ** 2 for e in _extents(w.grid[a], w.core[a], w.halo[a]))
    return out


def gpa_work(w, box):
    """Algorithmic and executed work of one fwd+bwd step, whole batch.

    Algorithmic (the method's own work): forward 4 d sum L^2 FLOP (S = Q K^T,
    P V); backward 8 d sum L^2 (dV = P^T dO, dP = dO V^T, dK = dS^T Q in the
    dK/dV kernel, dQ = dS K in the dQ kernel).  Executed: the MMA FLOPs the
    kernels issue over padded 128-row blocks, including the recomputed S (dK/dV
    kernel) and S, dP (dQ kernel) and, at d = 64, the K = 16 statistics step
    of each score chain of the dK/dV kernel.  Exponentials: sum L^2 forward, 2
    sum L^2 backward (P and its recompute)."""
    bh, d = w.B * w.nh, w.d
    L2, P = sum_L2(w) * bh, padded_pairs(w, box) * bh
    stats = 2 * 2 * 16 * P if d == 64 else 0
    alg = {"fwd_tiles": 4 * d * L2, "bwd_dkdv": 6 * d * L2, "bwd_dq": 2 * d * L2}
    exe = {"fwd_tiles": 4 * d * P, "bwd_dkdv": 8 * d * P + stats, "bwd_dq": 6 * d * P}
    return {"alg_flops": alg, "exec_flops": exe, "step_alg_flops": 12 * d * L2, "step_exps": 3 * L2,
            "sum_L2": L2, "padded_pairs": P}


def algorithmic_bytes(w, in_bytes=2, out_bytes=2):
    """Unique HBM bytes of one fwd+bwd step: forward reads Q, K, V and writes
    Out and the per-row log-sum-exp; backward reads Q, K, V, Out, dOut and the
    log-sum-exp and writes dQ, dK, dV.  Halo re-reads and merge scratch are
    overhead, not counted."""
    nd = w.B * w.N * w.nh * w.d
    lse = 4 * sum_L(w) * w.B * w.nh
    fwd = 3 * nd * in_bytes + nd * out_bytes + lse
    bwd = 4 * nd * in_bytes + nd * out_bytes + lse + 3 * nd * out_bytes
    return fwd + bwd


def workload_config(w, world):
    """The `config` object of both arms' JSON lines for a GPA workload."""
    tiles = 1
    for a in range(3):
        tiles *= -(-w.grid[a] // w.core[a])
    gb = w.B * w.nh * w.N * w.d * 2 / 1e9
    return {"workload": w.name, "B": w.B, "heads": w.nh, "d": w.d, "grid": list(w.grid), "core": list(w.core),
            "halo": list(w.halo), "tiles": tiles, "tokens_per_step": w.B * w.N * world, "in_dtype": "bf16",
            "out_dtype": "bf16", "l2": f"inputs {3 * gb:.1f} GB per rank > L2, no flush",
            "parallelism": f"replicas x{world} (independent batch*head units, no collective)"}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return p["hbm_gbs"], p["bf16_tflops"], p["bf16_tflops_sustained"], "measured"
    except Exception:
        return 6800.0, 1900.0, 1700.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""

    FIELDS = (
        "clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
        "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
        "clocks_event_reasons.sw_power_cap"
    )

    def __init__(self, gpu_index):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(gpu_index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True,
            )
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        hi = max(sm)
        loaded = [x for x in sm if x >= 0.5 * hi] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_sample(w, q, k, v, go, target_s=12.0):
    """Time the FP64 oracle (as it stands) on a bounded sample of one
    (batch*head) slice, forward + backward: query rows of the largest tile, or
    whole tiles in turn when one tile is quicker than the target.  Returns
    (Gtokens/s extrapolated to the whole step by (query, key) pairs, threads,
    description, seconds)."""
    import numpy as np

    import oracle

    geo = oracle.Geometry(1, 1, w.d, *w.grid, w.core, w.halo)
    f64 = [np.ascontiguousarray(t[0, 0].double().cpu().numpy())[None, None] for t in (q, k, v, go)]
    nt = geo.num_tiles()
    tile = max(range(nt), key=geo.tile_rows)
    L = geo.tile_rows(tile)
    t0 = time.perf_counter()
    oracle.unit_fwd_bwd(geo, *f64, 0, tile, 0, min(64, L))
    t64 = time.perf_counter() - t0
    if L > 64 and t64 * L / 64 > target_s:
        # part of the largest tile: R query rows against all its L keys
        R = int(min(L, max(64, 64 * target_s / max(t64, 1e-6))))
        t0 = time.perf_counter()
        oracle.unit_fwd_bwd(geo, *f64, 0, tile, 0, R)
        tR = time.perf_counter() - t0
        pairs, what = R * L, f"{R} query rows x {L} keys of one (batch*head, tile) unit"
    else:
        # whole tiles, in index order, until the target time is spent
        pairs, n, tR = 0, 0, 0.0
        while tR < target_s and n < nt:
            Lt = geo.tile_rows(n)
            t0 = time.perf_counter()
            oracle.unit_fwd_bwd(geo, *f64, 0, n, 0, Lt)
            tR += time.perf_counter() - t0
            pairs += Lt * Lt
            n += 1
        what = f"{n} whole tiles ({pairs:.3e} query-key pairs) of one batch*head slice"
    pairs_total = sum_L2(w) * w.B * w.nh
    step_s = tR * pairs_total / pairs
    gtok = w.B * w.N / step_s / 1e9
    desc = (f"{what}, forward + backward, {tR:.1f} s; scaled by (query, key) pairs to the full step "
            f"({pairs_total:.3e} pairs)")
    return gtok, oracle.threads(), desc, tR


def run_serving(n_requests, rank=0):
    """Serving workload: n posterior-sampling requests with Poisson arrivals at
    40 req/s, N log-uniform in [16384, 2097152] (multiples of one 32 x 64
    frame), 8 or 16 heads, d = 64, BF16 states N(0, 0.5), 20 denoising steps
    each, small tiles (core 1x16x16, halo 0/4/4), 150 GB HBM budget."""
    import torch

    from paper_2604_16590_gb300 import gattn, serving
    from paper_2604_16590_gb300.inputs import poisson_requests, state_pool

    from paper_2604_16590_gb300.replicas import replica_seed

    specs = poisson_requests(n=n_requests, seed=replica_seed(20265, rank))
    pool = state_pool(seed=replica_seed(20265, rank))
    cfg = gattn.serve_cfg(d=64, Y=32, X=64, core=(1, 16, 16), halo=(0, 4, 4), steps=20, c=0.5, max_active=256,
                          use_graph=True, hbm_budget=150 * 10**9)
    # every client takes its final state to host memory as soon as it is
    # done: an asynchronous take into one of two pinned buffers of the largest
    # request, used in turn (a buffer is reused once its previous copy is
    # complete), so the copies run beside the next iterations
    shapes = [(sp.nh, sp.T * 32 * 64, 64) for sp in specs]
    biggest = max(a * b * c for a, b, c in shapes)
    ring = [torch.empty(biggest, dtype=torch.bfloat16, pin_memory=True) for _ in range(2)]
    ring_rid = [None, None]
    turn = [0]
    with gattn.Server(cfg) as srv:
        def wait_copied(rid):
            while not srv.copied(rid):
                time.sleep(0.0002)

        def take(i, rid):
            nh, n, d = shapes[i]
            slot = turn[0] % 2
            turn[0] += 1
            if ring_rid[slot] is not None:
                wait_copied(ring_rid[slot])
            srv.take_async(rid, ring[slot][: nh * n * d].view(nh, n, d))
            ring_rid[slot] = rid

        lat = serving.run(srv, specs, 32, 64, 64, device="cuda", realtime=True, pool=pool, on_done=take)
        for rid in ring_rid:
            if rid is not None:
                wait_copied(rid)
        st = srv.stats()
    del pool, ring
    torch.cuda.empty_cache()
    return {
        "workload": f"{n_requests} requests, Poisson 40/s, N log-uniform [16384, 2097152], heads 8|16, d=64, "
                    "20 steps, core 1x16x16 halo 0/4/4, 150 GB budget; each result copied to pinned host memory "
                    "when done (asynchronous takes into two pinned buffers used in turn)",
        "requests": int(st.completed), "rejected": int(st.rejected), "iterations": int(st.iterations),
        "p50_latency_s": st.p50_latency_s, "p99_latency_s": st.p99_latency_s, "mean_latency_s": st.mean_latency_s,
        "max_latency_s": st.max_latency_s, "token_steps": st.token_steps, "wall_s": st.wall_s,
        "gpu_busy_s": st.gpu_busy_s, "token_steps_per_s": st.token_steps / st.wall_s if st.wall_s > 0 else None,
        "hbm_peak_gb": st.hbm_peak / 1e9, "graph": True, "n_latencies": len(lat),
    }


# DRAM bytes (read + write) per launch of the compression kernel from one ncu
# capture of the 512-frame case (h3_512, 4.295 GB read, 69.5 MB written), reads
# scaled by frames to the 2048-frame case and writes = its 10 ranges' partials;
# None once the kernel changes.
COMPRESS_TRAFFIC_PER_LAUNCH = {"h3_2k": 17.27e9, "h3_512": 4.365e9}


def run_compress(steps, warmup, dev, rank=0, cpu=True, peaks=None, workload="h3_2k"):
    """Temporal compression (learned query per head over S history frames per
    location) on the long-temporal-context shape: 2048 frames x 32 x 64
    locations, 8 heads, d = 128, BF16 keys/values (17.2 GB read per call, > L2,
    no flush).  Device time from CUDA events on the launching stream."""
    import torch

    from paper_2604_16590_gb300 import gattn
    from paper_2604_16590_gb300.inputs import HISTORY_WORKLOADS, history_inputs
    from paper_2604_16590_gb300.replicas import replica_seed

    w = HISTORY_WORKLOADS[workload]
    w = type(w)(**{**w.__dict__, "seed": replica_seed(w.seed, rank)})
    q, k, v = history_inputs(w, dev)
    desc = gattn.compress_desc(k)
    out = torch.empty((w.B, w.nh, w.M, w.d), dtype=torch.bfloat16, device=dev)
    lse = torch.empty((w.B, w.nh, w.M), dtype=torch.float32, device=dev)
    nws = gattn.gattn_compress_workspace_bytes(desc)
    ws = torch.empty(max(nws, 16), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def call():
        gattn.check(gattn.gattn_compress_fwd(desc, q, k, v, out, lse, ws if nws else None, stream=stream),
                    "gattn_compress_fwd")

    for _ in range(warmup):
        call()
    torch.cuda.synchronize()
    gattn.gattn_profile_enable(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        call()
    e1.record(stream)
    torch.cuda.synchronize()
    prof = gattn.gattn_profile_read()
    gattn.gattn_profile_enable(False)
    gattn.check(gattn.gattn_stream_status(), "compress status")
    ms = e0.elapsed_time(e1) / steps
    kv_bytes = 2 * k.numel() * k.element_size()
    alg = kv_bytes + q.numel() * 4 + out.numel() * 2 + lse.numel() * 4
    main_ms = prof.get("compress", (steps, ms * steps))[1] / steps
    peak, src = (peaks[0], peaks[3]) if peaks else (6800.0, "fallback")
    res = {
        "workload": f"{w.name}: {w.S} history frames x {w.Y}x{w.X} locations, B={w.B}, {w.nh} heads, d={w.d}, "
                    "BF16 k/v N(0,0.5), FP32 learned query",
        "ms_per_call": ms, "calls": steps, "warmup": warmup,
        "frames_per_s": w.B * w.nh * w.S * w.M / (ms * 1e-3),
        "kernels": {n: {"launches": c, "ms_per_launch": t / c} for n, (c, t) in prof.items()},
        "workspace_bytes": nws,
        "roofline": {"kernel": "compress", "bound": "hbm", "achieved": alg / (main_ms * 1e-3) / 1e9, "peak": peak,
                     "unit": "GB/s", "frac": alg / (main_ms * 1e-3) / 1e9 / peak,
                     "peak_source": f"hbm_gbs of {src}", "algorithmic_bytes": alg,
                     "traffic": COMPRESS_TRAFFIC_PER_LAUNCH.get(workload)},
        "call_gbs": alg / (ms * 1e-3) / 1e9,
    }
    if cpu:
        import numpy as np

        from oracle import compress as oc

        # the oracle as it stands on whole locations (all S frames), ~5-10 s
        rng = np.random.default_rng(1)
        n_loc, spent, done = 0, 0.0, 0
        while spent < 5.0 and n_loc < 4096:
            h, m = int(rng.integers(0, w.nh)), int(rng.integers(0, w.M))
            kl = k[0, h, :, m].double().cpu().numpy()[None, None, :, None, :]
            vl = v[0, h, :, m].double().cpu().numpy()[None, None, :, None, :]
            qh = q[h:h + 1].double().cpu().numpy()
            t0 = time.perf_counter()
            oc.forward(qh, kl, vl)
            spent += time.perf_counter() - t0
            n_loc += 1
        per_call_s = spent / n_loc * w.B * w.nh * w.M
        res["cpu_baseline"] = {"value": w.B * w.nh * w.S * w.M / per_call_s, "unit": "frames/s", "cores": 1,
                               "kind": "oracle",
                               "sample": f"{n_loc} (head, location) units of {w.S} frames, {spent:.1f} s; "
                                         f"scaled by units to the whole call"}
    del q, k, v, out, lse, ws
    torch.cuda.empty_cache()
    return res


def run_gated(steps, warmup, dev, w, rank=0):
    """Noise-gated self + cross attention on the bench workload's grid and
    tiling: two GPA forwards (the cross branch with a separate key/value
    source, standing in for the compressed temporal representation) and the
    per-head blend.  Device time from CUDA events on the launching stream."""
    import torch

    from paper_2604_16590_gb300 import gattn
    from paper_2604_16590_gb300.inputs import qkv
    from paper_2604_16590_gb300.replicas import replica_seed

    q, k, v, kc, vc = qkv(w.shape, replica_seed(w.seed + 31, rank), w.std, "bf16", device=dev, n=5)
    gate = torch.linspace(0.1, 0.9, w.nh, device=dev, dtype=torch.float32)
    tiling = gattn.Tiling(w.grid, w.core, w.halo)
    desc = gattn.desc_for(q, tiling, torch.bfloat16)
    out = torch.empty_like(q)
    ws = torch.empty(gattn.gattn_gated_workspace_bytes(desc), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def call():
        gattn.check(gattn.gattn_gated_fwd(desc, q, k, v, kc, vc, gate, out, ws, stream=stream), "gattn_gated_fwd")

    for _ in range(warmup):
        call()
    torch.cuda.synchronize()
    gattn.gattn_profile_enable(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        call()
    e1.record(stream)
    torch.cuda.synchronize()
    prof = gattn.gattn_profile_read()
    gattn.gattn_profile_enable(False)
    gattn.check(gattn.gattn_stream_status(), "gated status")
    ms = e0.elapsed_time(e1) / steps
    mix_ms = prof.get("gated_mix", (steps, 0.0))[1] / steps
    mix_bytes = 3 * q.numel() * 2 + w.nh * 4
    res = {
        "workload": f"{w.name} grid and tiling, self + cross branch (separate BF16 K/V source), per-head gate",
        "ms_per_call": ms, "calls": steps, "warmup": warmup,
        "tokens_per_s": w.B * w.N / (ms * 1e-3),
        "kernels": {n: {"launches": c, "ms_per_launch": t / c} for n, (c, t) in prof.items()},
        "mix_gbs": mix_bytes / (mix_ms * 1e-3) / 1e9 if mix_ms > 0 else None,
    }
    del q, k, v, kc, vc, out, ws
    torch.cuda.empty_cache()
    return res


def run_dps(steps, warmup, dev, w, rank=0, n_prop=20):
    """Diffusion posterior sampling with the GPA denoiser (gattn_dps_step).

    (1) Step time on the bench workload's grid and tiling (BF16 attention, FP32
        state, 25 % of the tokens observed).
    The synthetic denoiser is GPA(z, z, z) with attention scale 1/d: at
    1/sqrt(d) a unit-variance state attends almost only to itself and the
    likelihood gradient through the softmax makes the sampler diverge.
    (2) Context propagation (Sec. III-C): a 64 x 256 frame cut into 4 x 8 tiles
        of 16 x 32 with a 4/8-token halo; only the first tile's core is
        observed.  Two runs share the noise, one with the likelihood term and
        one without; after every step the farthest tile (Chebyshev distance in
        tiles) whose state moved by more than 1e-3 of the state's scale is the
        propagation front.
    (3) The same sampling with Tiles = 1 (global attention): relative L2
        distance of the final states of the tiled run with halos, and of a
        tiled run without halos, to the global run."""
    import torch

    from paper_2604_16590_gb300 import gattn
    from paper_2604_16590_gb300.replicas import replica_seed

    # (1) step time at the bench size
    g = torch.Generator(device=dev)
    g.manual_seed(replica_seed(w.seed + 57, rank))
    z = torch.randn(w.shape, generator=g, device=dev) * 0.5
    y = torch.randn(w.shape, generator=g, device=dev) * 0.5
    eps = torch.randn(w.shape, generator=g, device=dev)
    mask = (torch.rand((w.B, w.N), generator=g, device=dev) < 0.25).to(torch.uint8)
    smp = gattn.PosteriorSampler(z, gattn.Tiling(w.grid, w.core, w.halo, scale=1.0 / w.d), "bf16")
    sig = gattn.sigma_schedule(steps + warmup, 2.0, 0.05)
    stream = torch.cuda.current_stream()
    for i in range(warmup):
        smp.step(y, mask, eps, sig[i], sig[i + 1], 0.5)
    torch.cuda.synchronize()
    gattn.gattn_profile_enable(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(warmup, warmup + steps):
        smp.step(y, mask, eps, sig[i], sig[i + 1], 0.5)
    e1.record(stream)
    torch.cuda.synchronize()
    prof = gattn.gattn_profile_read()
    gattn.gattn_profile_enable(False)
    gattn.check(gattn.gattn_stream_status(), "dps status")
    ms = e0.elapsed_time(e1) / steps
    del smp, z, y, eps, mask
    torch.cuda.empty_cache()

    # (2)-(3) propagation on a 64 x 256 frame, 2 heads, d = 64
    grid, d, nh = (1, 64, 256), 64, 2
    N = grid[1] * grid[2]
    g.manual_seed(replica_seed(20270, rank))
    z0 = torch.randn((1, nh, N, d), generator=g, device=dev)
    y = torch.randn((1, nh, N, d), generator=g, device=dev) * 0.5
    tok = torch.arange(N, device=dev)
    mask = (((tok // grid[2]) < 16) & ((tok % grid[2]) < 32)).to(torch.uint8)[None]
    noise = [torch.randn((1, nh, N, d), generator=g, device=dev) for _ in range(n_prop)]
    sig = gattn.sigma_schedule(n_prop, 2.0, 0.05)

    def run(core, halo, lam, keep=False):
        smp = gattn.PosteriorSampler(z0.clone(), gattn.Tiling(grid, core, halo, scale=1.0 / d), "bf16")
        states = []
        for i in range(n_prop):
            smp.step(y, mask, noise[i], sig[i], sig[i + 1], lam)
            if keep:
                states.append(smp.z.clone())
        return smp.z.clone(), states

    tiled, halo = (1, 16, 32), (0, 4, 8)
    _, with_obs = run(tiled, halo, 0.5, keep=True)
    _, without = run(tiled, halo, 0.0, keep=True)
    front = []
    for a, b in zip(with_obs, without):
        diff = (a - b).abs().amax(dim=(0, 1, 3)).reshape(grid[1] // 16, 16, grid[2] // 32, 32).amax(dim=(1, 3))
        scale = b.abs().amax()
        moved = (diff > 1e-3 * scale).nonzero()
        front.append(int(moved.max(dim=0).values.max()) if moved.numel() else -1)
    z_glob, _ = run(grid, (0, 0, 0), 0.5)
    z_halo = with_obs[-1]
    z_nohalo, _ = run(tiled, (0, 0, 0), 0.5)
    ref = (z_glob - z0).norm()
    res = {
        "workload": f"{w.name} grid and tiling, attention scale 1/d, FP32 state, BF16 attention, 25 % of tokens "
                    "observed, lam 0.5",
        "ms_per_step": ms, "steps": steps, "warmup": warmup,
        "kernels": {n: {"launches": c, "ms_per_launch": t / c} for n, (c, t) in prof.items()},
        "propagation": {
            "setup": "64 x 256 frame, 4 x 8 tiles of 16 x 32, halo 4/8, 2 heads, d 64, attention scale 1/d, lam 0.5; "
                     f"observations in tile (0,0) only; {n_prop} steps, sigma 2.0 -> 0.05",
            "front_tiles_per_step": front,
            "rel_dist_to_tiles1_with_halo": float((z_halo - z_glob).norm() / ref),
            "rel_dist_to_tiles1_without_halo": float((z_nohalo - z_glob).norm() / ref),
        },
    }
    torch.cuda.empty_cache()
    return res


def run_linear(steps, warmup, dev, w, rank=0, peaks=None):
    """Factorised linear attention (phi = elu + 1; not an operator of the paper)
    on the bench workload's shape: B x heads x N tokens x d = 64, BF16 Q, K, V
    N(0, 0.5), upstream gradient N(0, 1).  Forward: 4 x 2.15 GB moved per call
    (q, k, v read, out written); backward: 7 x 2.15 GB (q, k, v, dout read;
    dq, dk, dv written); both > L2, no flush.  Device time from CUDA events on
    the launching stream."""
    import torch

    from paper_2604_16590_gb300 import gattn
    from paper_2604_16590_gb300.inputs import qkv
    from paper_2604_16590_gb300.replicas import replica_seed

    q, k, v = qkv(w.shape, replica_seed(w.seed + 91, rank), w.std, "bf16", device=dev)
    (g,) = qkv(w.shape, replica_seed(w.seed + 93, rank), 1.0, "bf16", device=dev, n=1)
    desc = gattn.linear_desc(q)
    out = torch.empty_like(q)
    dq, dk, dv = torch.empty_like(q), torch.empty_like(q), torch.empty_like(q)
    ws = torch.empty(gattn.gattn_linear_workspace_bytes(desc), dtype=torch.uint8, device=dev)
    wsb = torch.empty(gattn.gattn_linear_bwd_workspace_bytes(desc), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def fwd():
        gattn.check(gattn.gattn_linear_fwd(desc, q, k, v, out, ws, stream=stream), "gattn_linear_fwd")

    def bwd():
        gattn.check(gattn.gattn_linear_bwd(desc, q, k, v, g, ws, dq, dk, dv, wsb, stream=stream), "gattn_linear_bwd")

    def timed(fn):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        gattn.gattn_profile_enable(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        prof = gattn.gattn_profile_read()
        gattn.gattn_profile_enable(False)
        gattn.check(gattn.gattn_stream_status(), "linear status")
        return e0.elapsed_time(e1) / steps, prof

    ms_f, prof_f = timed(fwd)
    ms_b, prof_b = timed(bwd)
    nd2 = q.numel() * 2
    peak, src = (peaks[0], peaks[3]) if peaks else (6800.0, "fallback")
    gbs_f, gbs_b = 4 * nd2 / (ms_f * 1e-3) / 1e9, 7 * nd2 / (ms_b * 1e-3) / 1e9
    gbs_fb = 11 * nd2 / ((ms_f + ms_b) * 1e-3) / 1e9
    kernels = {n: {"launches": c, "ms_per_launch": t / c} for n, (c, t) in {**prof_f, **prof_b}.items()}
    res = {
        "workload": f"{w.name} shape: B={w.B}, {w.nh} heads, N={w.N}, d={w.d}, BF16, phi = elu + 1",
        "ms_per_call": ms_f, "ms_backward": ms_b, "calls": steps, "warmup": warmup,
        "tokens_per_s": w.B * w.N / (ms_f * 1e-3), "fwd_bwd_tokens_per_s": w.B * w.N / ((ms_f + ms_b) * 1e-3),
        "kernels": kernels,
        "roofline": {"kernel": "linear forward (summary + combine + query)", "bound": "hbm", "achieved": gbs_f,
                     "peak": peak, "unit": "GB/s", "frac": gbs_f / peak, "peak_source": f"hbm_gbs of {src}",
                     "algorithmic_bytes": 4 * nd2, "traffic": None},
        "roofline_backward": {"kernel": "linear backward (query pass + combine + key pass)", "bound": "hbm",
                              "achieved": gbs_b, "peak": peak, "unit": "GB/s", "frac": gbs_b / peak,
                              "peak_source": f"hbm_gbs of {src}", "algorithmic_bytes": 7 * nd2, "traffic": None},
        "fwd_bwd_gbs": gbs_fb, "fwd_bwd_frac": gbs_fb / peak,
    }
    del q, k, v, g, out, dq, dk, dv, ws, wsb
    torch.cuda.empty_cache()
    return res


def run_gpa(w, steps, warmup, dev, rank, world, peaks, cpu=True, e2e_steps=1, fp32_steps=0, clocks=False,
            barrier=None):
    """One GPA workload: `steps` timed fwd+bwd steps (gattn_fwd + gattn_bwd
    through the C ABI) after `warmup` untimed ones, inputs device-resident
    (larger than L2, no flush).  Reports the step time (max over ranks), the
    per-kernel device times (CUDA events on the launch stream), the roofline of
    the dominant kernel on its algorithmic FLOPs, the step's fraction of its
    attainable time max(bytes / HBM, FLOPs / tensor peak, exps / exp-unit
    peak), an end-to-end time with pinned host buffers (H2D of Q, K, V, dOut
    and D2H of Out, dQ, dK, dV inside the timed region), the plain FP32 form
    on the same values (fp32_steps > 0) and the oracle on a bounded sample."""
    import torch

    from paper_2604_16590_gb300 import gattn, replicas
    from paper_2604_16590_gb300.inputs import qkv, upstream_grad

    barrier = barrier or (lambda: None)
    q, k, v = qkv(w.shape, replicas.replica_seed(w.seed, rank), w.std, "bf16", device=dev)
    go = upstream_grad(w.shape, replicas.replica_seed(w.seed, rank), "bf16", device=dev)
    tiling = gattn.Tiling(w.grid, w.core, w.halo)
    desc = gattn.desc_for(q, tiling, torch.bfloat16)
    st_box, box = gattn.gattn_block_shape(desc)
    gattn.check(st_box, "gattn_block_shape")
    out = torch.empty_like(q)
    dq, dk, dv = torch.empty_like(q), torch.empty_like(q), torch.empty_like(q)
    saved = torch.empty(gattn.gattn_saved_bytes(desc), dtype=torch.uint8, device=dev)
    ws = torch.empty(gattn.gattn_bwd_workspace_bytes(desc), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step(qq=q, kk=k, vv=v, gg=go, d=desc, o=out, a=dq, b=dk, c=dv, sv=saved, wsp=ws):
        gattn.check(gattn.gattn_fwd(d, qq, kk, vv, o, sv, stream=stream), "gattn_fwd")
        gattn.check(gattn.gattn_bwd(d, qq, kk, vv, o, gg, sv, a, b, c, wsp, stream=stream), "gattn_bwd")

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    st = gattn.gattn_stream_status(stream)
    if st != 0:
        raise RuntimeError(f"{w.name}: device status after warm-up: {gattn.STATUS.get(st, st)}")

    # ---- timed region (device-resident inputs)
    sampler = ClockSampler(dev.index or 0) if clocks else None
    if sampler:
        time.sleep(0.3)
    gattn.gattn_profile_enable(True)
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = sampler.stop() if sampler else None
    kstats = gattn.gattn_profile_read()
    gattn.gattn_profile_enable(False)
    st = gattn.gattn_stream_status(stream)
    if st != 0:
        raise RuntimeError(f"{w.name}: device status after timed steps: {gattn.STATUS.get(st, st)}")
    ms = replicas.max_over_ranks(e0.elapsed_time(e1) / steps, device=dev)
    value = replicas.weak_scaling_value(w.B * w.N, world, ms * 1e-3) / 1e9

    # ---- roofline: dominant kernel on its algorithmic FLOPs; the step against its attainable time
    hbm_peak, tc_peak, tc_sust, peak_src = peaks
    n_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_mhz = measured_sm_max_mhz()
    ex2_peak = EX2_PER_CLK_SM * n_sms * sm_mhz * 1e6
    work = gpa_work(w, box)
    kernels = {}
    for name, (n, tot) in kstats.items():
        per = tot / n
        ent = {"launches": n, "ms_per_launch": per, "share": tot / (ms * steps)}
        if name in work["alg_flops"]:
            ent["alg_tflops"] = work["alg_flops"][name] / (per * 1e-3) / 1e12
            ent["exec_tflops"] = work["exec_flops"][name] / (per * 1e-3) / 1e12
            ent["frac_of_sustained"] = ent["alg_tflops"] / tc_sust
        kernels[name] = ent
    dom = max(kstats, key=lambda nm: kstats[nm][1])
    dom_ms = kstats[dom][1] / kstats[dom][0]
    achieved = work["alg_flops"].get(dom, 0) / (dom_ms * 1e-3) / 1e12
    roofline = {
        "kernel": dom, "bound": "tensor", "achieved": achieved, "peak": tc_sust, "unit": "TFLOP/s",
        "frac": achieved / tc_sust, "peak_source": f"bf16_tflops_sustained of {peak_src}",
        "traffic": TRAFFIC_PER_LAUNCH.get((w.name, dom)),
        "algorithmic_flops": work["alg_flops"].get(dom), "executed_flops": work["exec_flops"].get(dom),
        "executed_tflops": work["exec_flops"].get(dom, 0) / (dom_ms * 1e-3) / 1e12,
    }
    alg_bytes = algorithmic_bytes(w)
    t_bytes = alg_bytes / (hbm_peak * 1e9)
    t_flops = work["step_alg_flops"] / (tc_sust * 1e12)
    t_exps = work["step_exps"] / ex2_peak
    t_att = max(t_bytes, t_flops, t_exps)
    attainable = {
        "ms": 1e3 * t_att, "bound": ("hbm", "tensor", "exp")[[t_bytes, t_flops, t_exps].index(t_att)],
        "ms_hbm": 1e3 * t_bytes, "ms_tensor": 1e3 * t_flops, "ms_exp": 1e3 * t_exps,
        "frac_of_attainable": t_att / (ms * 1e-3),
        "step_alg_flops": work["step_alg_flops"], "step_exec_flops": sum(work["exec_flops"].values()),
        "executed_over_algorithmic": sum(work["exec_flops"].values()) / work["step_alg_flops"],
        "padding": work["padded_pairs"] / work["sum_L2"], "block_shape": list(box),
        "exp_peak": f"{EX2_PER_CLK_SM} ex2/clk/SM x {n_sms} SMs x {sm_mhz:.0f} MHz",
    }
    hbm = {"algorithmic_bytes_per_step": alg_bytes, "gbs": alg_bytes / (ms * 1e-3) / 1e9,
           "frac_of_hbm": alg_bytes / (ms * 1e-3) / 1e9 / hbm_peak, "peak_gbs": hbm_peak, "peak_source": peak_src}

    # ---- e2e through the public API with host buffers: every step copies its
    # inputs (Q, K, V, dOut) from pinned host memory and its results (Out, dQ,
    # dK, dV) back, on a copy-in and a copy-out stream.  With two device buffer
    # sets, the inputs of step i+1 load while step i computes, and Out of a
    # step leaves while its backward runs: the timed region (its first
    # copy-in to its last copy-out) holds every copy of every step.
    e2e = None
    if e2e_steps > 0:
        host_in = [torch.empty(w.shape, dtype=torch.bfloat16, pin_memory=True) for _ in range(4)]
        for h, t in zip(host_in, (q, k, v, go)):
            h.copy_(t)
        host_out = [torch.empty(w.shape, dtype=torch.bfloat16, pin_memory=True) for _ in range(4)]
        nset = 2 if e2e_steps > 1 else 1
        sets_in = [(q, k, v, go)] + [tuple(torch.empty_like(q) for _ in range(4)) for _ in range(nset - 1)]
        sets_out = [(out, dq, dk, dv)] + [tuple(torch.empty_like(q) for _ in range(4)) for _ in range(nset - 1)]
        s_in, s_out = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)

        def e2e_run(n, start_ev=None):
            loaded = [torch.cuda.Event() for _ in range(nset)]
            inputs_free = [None] * nset   # backward of the set's previous step done
            outputs_out = [None] * nset   # outputs of the set's previous step copied out

            def load(b, after=None):
                if after is not None:
                    s_in.wait_event(after)
                if inputs_free[b] is not None:
                    s_in.wait_event(inputs_free[b])
                with torch.cuda.stream(s_in):
                    for d_, h_ in zip(sets_in[b], host_in):
                        d_.copy_(h_, non_blocking=True)
                loaded[b].record(s_in)

            load(0, start_ev)
            last = None
            for i in range(n):
                b = i % nset
                if nset > 1 and i + 1 < n:
                    load((i + 1) % nset)
                elif nset == 1 and i > 0:
                    load(0)
                stream.wait_event(loaded[b])
                if outputs_out[b] is not None:
                    stream.wait_event(outputs_out[b])
                qq, kk, vv, gg = sets_in[b]
                o, a, bb, c = sets_out[b]
                gattn.check(gattn.gattn_fwd(desc, qq, kk, vv, o, saved, stream=stream), "gattn_fwd")
                ev_f = torch.cuda.Event()
                ev_f.record(stream)
                gattn.check(gattn.gattn_bwd(desc, qq, kk, vv, o, gg, saved, a, bb, c, ws, stream=stream),
                            "gattn_bwd")
                ev_b = torch.cuda.Event()
                ev_b.record(stream)
                inputs_free[b] = ev_b
                s_out.wait_event(ev_f)
                with torch.cuda.stream(s_out):
                    host_out[0].copy_(o, non_blocking=True)
                s_out.wait_event(ev_b)
                with torch.cuda.stream(s_out):
                    for h_, d_ in zip(host_out[1:], (a, bb, c)):
                        h_.copy_(d_, non_blocking=True)
                last = torch.cuda.Event()
                last.record(s_out)
                outputs_out[b] = last
            stream.wait_event(last)

        e2e_run(1)
        torch.cuda.synchronize()
        barrier()
        e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e2.record(stream)
        e2e_run(e2e_steps, e2)
        e3.record(stream)
        torch.cuda.synchronize()
        st = gattn.gattn_stream_status(stream)
        if st != 0:
            raise RuntimeError(f"{w.name}: device status after e2e steps: {gattn.STATUS.get(st, st)}")
        e2e_ms = replicas.max_over_ranks(e2.elapsed_time(e3) / e2e_steps, device=dev)
        bytes_io = 4 * q.numel() * q.element_size()
        e2e = {"value": w.B * w.N * world / (e2e_ms * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": e2e_ms,
               "steps": e2e_steps, "h2d_bytes_per_step": bytes_io, "d2h_bytes_per_step": bytes_io,
               "overlap": "copies on two streams beside the compute stream, two device buffer sets"
                          if nset > 1 else "copies on two streams, one buffer set (one step)"}
        del host_in, host_out, sets_in, sets_out

    # ---- the plain FP32 form on the same values
    fp32 = None
    if fp32_steps > 0:
        q32, k32, v32, g32 = (t.float() for t in (q, k, v, go))
        d32 = gattn.desc_for(q32, tiling, torch.float32)
        o32 = torch.empty_like(q32)
        a32, b32, c32 = (torch.empty_like(q32) for _ in range(3))
        sv32 = torch.empty(gattn.gattn_saved_bytes(d32), dtype=torch.uint8, device=dev)
        ws32 = torch.empty(gattn.gattn_bwd_workspace_bytes(d32), dtype=torch.uint8, device=dev)

        def step32():
            step(qq=q32, kk=k32, vv=v32, gg=g32, d=d32, o=o32, a=a32, b=b32, c=c32, sv=sv32, wsp=ws32)

        step32()
        torch.cuda.synchronize()
        e4, e5 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e4.record(stream)
        for _ in range(fp32_steps):
            step32()
        e5.record(stream)
        torch.cuda.synchronize()
        ms32 = e4.elapsed_time(e5) / fp32_steps
        fp32 = {"value": w.B * w.N * world / (ms32 * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": ms32,
                "steps": fp32_steps, "bf16_speedup": ms32 / ms}
        del q32, k32, v32, g32, o32, a32, b32, c32, sv32, ws32

    # ---- the oracle as it stands on a bounded sample (rank 0, N = 1)
    cpu_res = None
    if cpu and rank == 0 and world == 1:
        sl = (slice(0, 1), slice(0, 1))
        g, cores, desc_s, _ = oracle_sample(w, q[sl].cpu(), k[sl].cpu(), v[sl].cpu(), go[sl].cpu())
        cpu_res = {"value": g, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc_s}

    res = {"workload": w.name, "config": workload_config(w, world), "value": value, "unit": UNIT,
           "ms_per_step": ms, "steps": steps, "warmup": warmup, "roofline": roofline, "attainable": attainable,
           "hbm": hbm, "kernels": kernels, "gpu_launches": sum(n for n, _ in kstats.values()), "e2e": e2e,
           "fp32_form": fp32, "cpu_baseline": cpu_res, "clocks": clk}
    del q, k, v, go, out, dq, dk, dv, saved, ws
    torch.cuda.empty_cache()
    return res


def measured_sm_max_mhz():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["sm_max_mhz"])
    except Exception:
        return 2070.0


def world_size(args):
    """Ranks of this run: WORLD_SIZE under torchrun, else 1."""
    return int(os.environ.get("WORLD_SIZE", "1"))


def self_launch(args):
    """`--gpus N` (N > 1) without torchrun: start N ranks of this script under
    torch.distributed.run (one process per GPU, rendezvous on 127.0.0.1) and
    return their exit status; rank 0 prints the JSON line."""
    import socket

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={args.gpus}",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__), *sys.argv[1:]]
    return subprocess.call(cmd)


def run_reference(args, w):
    """The reference arm: the FP64 oracle as it stands on the host cores, on a
    bounded sample of the same workload, scaled to one step (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if world_size(args) > 1:
        # torchrun pins every rank to one OpenMP thread; rank 0 alone runs the
        # oracle here, on all host cores
        os.environ["OMP_NUM_THREADS"] = str(os.cpu_count() or 1)
    # the oracle sample reads one (batch, head) slice: draw just that slice
    from paper_2604_16590_gb300.inputs import qkv, upstream_grad

    shape1 = (1, 1, w.N, w.d)
    q, k, v = qkv(shape1, w.seed, w.std, w.dtype)
    go = upstream_grad(shape1, w.seed, w.dtype)
    vals, secs = [], []
    for _ in range(args.warmup):
        oracle_sample(w, q, k, v, go, target_s=2.0)
    for _ in range(args.steps):
        g, cores, desc, t = oracle_sample(w, q, k, v, go, target_s=8.0)
        vals.append(g)
        secs.append(t)
    value = statistics.median(vals)
    world = world_size(args)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * w.B * w.N * world / (value * 1e9),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(w, world),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_dry(args):
    """--dry-run: start the ranks (gloo, no GPU work) and have rank 0 print the
    world size it sees; checks the multi-rank launch path on a CPU machine."""
    import torch.distributed as dist

    world, rank = world_size(args), int(os.environ.get("RANK", "0"))
    if world > 1:
        dist.init_process_group("gloo")
        from paper_2604_16590_gb300 import replicas

        ranks = replicas.sum_over_ranks(1.0)
        dist.destroy_process_group()
    else:
        ranks = 1.0
    if rank == 0:
        print(json.dumps({"dry_run": True, "n_gpus": world, "ranks_seen": int(ranks), "gpus_arg": args.gpus}),
              flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gattn", choices=["gattn", "reference"])
    ap.add_argument("--workload", default="c2_262k_p")
    ap.add_argument("--legs", default="c2_262k_s,c4_1m_p,c3_4m_p",
                    help="other GPA workloads timed as extra legs (comma list, '' = none)")
    ap.add_argument("--leg-steps", type=int, default=0,
                    help="timed steps of each extra leg (0 = by size: 10 below 0.1 s per step, else 2, C3 1)")
    ap.add_argument("--fp32-steps", type=int, default=1, help="timed steps of the plain FP32 form (0 = skip)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baselines")
    ap.add_argument("--compress-steps", type=int, default=10,
                    help="timed calls of the temporal compression (0 = skip)")
    ap.add_argument("--compress-workload", default="h3_2k")
    ap.add_argument("--linear-steps", type=int, default=10,
                    help="timed calls of the factorised linear attention (0 = skip)")
    ap.add_argument("--dps-steps", type=int, default=2,
                    help="timed posterior-sampling steps (0 = skip the posterior-sampling leg)")
    ap.add_argument("--gated-steps", type=int, default=2,
                    help="timed calls of the noise-gated self + cross attention (0 = skip)")
    ap.add_argument("--serve-requests", type=int, default=256,
                    help="requests of the serving run (Poisson 40/s, 20 steps; 0 = skip)")
    ap.add_argument("--dry-run", action="store_true", help="launch the ranks and report the world size only")
    args = ap.parse_args()

    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        sys.exit(self_launch(args))
    if args.dry_run:
        run_dry(args)
        return

    from paper_2604_16590_gb300.inputs import WORKLOADS

    w = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, w)
        return

    import torch
    import torch.distributed as dist

    from paper_2604_16590_gb300 import build, gattn, replicas

    world = world_size(args)
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    build.build()
    gattn.load_library()
    peaks = measured_peaks()

    def barrier():
        if world > 1:
            dist.barrier()

    # ---------------------------------------------------------------- serving: continuous batching (rank-local),
    # run first so that its HBM budget does not compete with the step buffers
    serve = None
    if args.serve_requests > 0:
        serve = run_serving(args.serve_requests, rank)
        if world > 1:
            t_srv = replicas.max_over_ranks(serve["wall_s"], device=dev)
            serve["token_steps_per_s_all_ranks"] = replicas.sum_over_ranks(serve["token_steps"], device=dev) / t_srv

    # ---------------------------------------------------------------- other GPA workloads (each its own leg)
    legs = {}
    for name in [x for x in args.legs.split(",") if x]:
        lw = WORKLOADS[name]
        n = args.leg_steps or (1 if lw.name.startswith("c3") else 10 if lw.name.endswith("_s") else 2)
        legs[name] = run_gpa(lw, n, 1, dev, rank, world, peaks, cpu=not args.no_cpu, e2e_steps=1,
                             fp32_steps=0, barrier=barrier)

    # ---------------------------------------------------------------- temporal compression (rank-local)
    compress = None
    if args.compress_steps > 0:
        compress = run_compress(args.compress_steps, 3, dev, rank, cpu=rank == 0 and world == 1 and not args.no_cpu,
                                peaks=peaks, workload=args.compress_workload)
    linear = None
    if args.linear_steps > 0:
        linear = run_linear(args.linear_steps, 3, dev, w, rank, peaks=peaks)
    dps = None
    if args.dps_steps > 0:
        dps = run_dps(args.dps_steps, 1, dev, w, rank)
    gated = None
    if args.gated_steps > 0:
        gated = run_gated(args.gated_steps, 1, dev, w, rank)

    # ---------------------------------------------------------------- the headline workload
    head = run_gpa(w, args.steps, args.warmup, dev, rank, world, peaks, cpu=not args.no_cpu,
                   e2e_steps=max(1, min(args.steps, 5)), fp32_steps=args.fp32_steps, clocks=True, barrier=barrier)

    if rank == 0:
        line = {
            "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": head["config"],
            "clocks": head["clocks"],
            "e2e": head["e2e"],
            "gpu_launches": head["gpu_launches"],
            "roofline": head["roofline"],
            "attainable": head["attainable"],
            "hbm": head["hbm"],
            "kernels": head["kernels"],
            "fp32_form": head["fp32_form"],
            "legs": legs,
            "serve": serve,
            "compress": compress,
            "gated": gated,
            "dps": dps,
            "linear": linear,
            "cpu_baseline": head["cpu_baseline"],
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
