"""Parity at the full sizes of the long-temporal-context and the backward-
throughput workloads, in the library's launch configuration:

* c3_4m_p: 2048 frames x 32 x 64 (N = 4,194,304), 8 heads, d = 128, BF16,
  Tiles = 16 along time (core 128 x 32 x 64, halo 8 frames);
* c4_1m_p: 16 x 256 x 256 (N = 1,048,576), 8 heads, d = 64, BF16,
  Tiles = 16 (core 16 x 64 x 64, halo 0/8/8).

The oracle evaluates sampled rows of Out and dQ one by one (rows on tile
boundaries, which two tiles cover, in cores, and at random); dK and dV are
checked through two identities that hold at every size: per (batch, head) the
dV rows sum to the dOut rows and the dK rows sum to zero."""
import numpy as np
import pytest
import torch

import oracle
from paper_2604_16590_gb300 import build, gattn
from paper_2604_16590_gb300.inputs import WORKLOADS, workload_inputs

pytestmark = pytest.mark.gpu

MAX_REL, RMS_REL = 2e-2, 3e-3


def _slice64(t, b, h):
    return np.ascontiguousarray(t[b, h].double().cpu().numpy())[None, None]


def _errs(got, ref):
    got, ref = np.asarray(got), np.asarray(ref)
    return np.abs(got - ref).max() / np.abs(ref).max(), np.linalg.norm(got - ref) / np.linalg.norm(ref)


def _slot(w, box, bh, tile, p):
    """Slot of token position p in extended tile `tile` (per-dimension indices):
    box j of the tile at offset (p - lo) // box, row rho inside the box, boxes of
    a tile contiguous (128 slots each) and tiles laid out per batch*head."""
    n = [-(-w.grid[a] // w.core[a]) for a in range(3)]
    lo, e, emax = [], [], []
    for a in range(3):
        ext = [min((kk + 1) * w.core[a] + w.halo[a], w.grid[a]) - max(kk * w.core[a] - w.halo[a], 0)
               for kk in range(n[a])]
        lo.append(max(tile[a] * w.core[a] - w.halo[a], 0))
        e.append(ext[tile[a]])
        emax.append(max(ext))
    l = [p[a] - lo[a] for a in range(3)]
    nb = [-(-e[a] // box[a]) for a in range(3)]
    per_tile = 128
    for a in range(3):
        per_tile *= -(-emax[a] // box[a])
    j = ((l[0] // box[0]) * nb[1] + l[1] // box[1]) * nb[2] + l[2] // box[2]
    rho = ((l[0] % box[0]) * box[1] + l[1] % box[1]) * box[2] + l[2] % box[2]
    t = (tile[0] * n[1] + tile[1]) * n[2] + tile[2]
    return ((bh * n[0] * n[1] * n[2] + t) * per_tile + j * 128 + rho)


def _check_row_normalisers(w, q, k, saved, desc):
    """The per-tile row normalisers the forward saves (log2 of the compensated
    FP32 row sum plus the reference max) against the oracle's per-tile
    log-sum-exp at sampled rows of tiles that span 2304 key boxes (144 frames
    of 32 x 64 tokens; Tab. III(a)'s long temporal context): the Kahan-
    compensated sum keeps the normaliser's relative error near FP32 rounding."""
    from oracle import brute

    st, box = gattn.gattn_block_shape(desc)
    assert st == 0
    lse2 = saved[: saved.numel() // 4 * 4].view(torch.float32)
    T, Y, X = w.grid
    b, h = 0, w.nh - 1
    q2 = q[b, h].double().cpu().numpy()
    k2 = k[b, h].double().cpu().numpy()
    rng = np.random.default_rng(11)
    worst = 0.0
    for kt in (0, 7, 15):
        t_lo = max(kt * w.core[0] - w.halo[0], 0)
        t_hi = min((kt + 1) * w.core[0] + w.halo[0], T)
        ts = rng.integers(t_lo, t_hi, 6)
        ps = [(int(t_), int(rng.integers(0, Y)), int(rng.integers(0, X))) for t_ in ts]
        rows = [(t_ * Y + y_) * X + x_ for t_, y_, x_ in ps]
        ref = brute.tile_lse(T, Y, X, w.core, w.halo, q2, k2, 1.0 / np.sqrt(w.d), (kt, 0, 0), rows)
        slots = [_slot(w, box, b * w.nh + h, (kt, 0, 0), p) for p in ps]
        got = lse2[torch.as_tensor(slots, device=lse2.device)].double().cpu().numpy() * np.log(2.0)
        worst = max(worst, float(np.abs(got - ref).max()))
    print(f"c3 row normaliser: max |lse - lse_ref| = {worst:.3e} (nats)")
    assert worst <= 2e-5, worst


@pytest.mark.parametrize("name", ["c4_1m_p", "c3_4m_p"])
def test_full_size_sampled_rows_and_identities(name):
    build.build()
    gattn.load_library()
    w = WORKLOADS[name]
    q, k, v, go = workload_inputs(w, device="cuda")
    tiling = gattn.Tiling(w.grid, w.core, w.halo)
    out, saved = gattn.forward(q, k, v, tiling, out_dtype=torch.bfloat16)
    dq, dk, dv = gattn.backward(q, k, v, out, go, saved, tiling)
    assert gattn.gattn_stream_status() == 0
    if name == "c3_4m_p":
        _check_row_normalisers(w, q, k, saved, gattn.desc_for(q, tiling, torch.bfloat16))
    del saved

    # identities of the operator at every size (dk, dv)
    sdv = dv.sum(dim=2, dtype=torch.float64)
    sgo = go.sum(dim=2, dtype=torch.float64)
    assert float((sdv - sgo).norm() / sgo.norm()) < 1e-3
    sdk = dk.sum(dim=2, dtype=torch.float64)
    assert float((sdk.abs() / dk.abs().sum(dim=2, dtype=torch.float64)).max()) < 1e-3

    # sampled rows of out and dq against the oracle
    T, Y, X = w.grid
    geo1 = oracle.Geometry(1, 1, w.d, T, Y, X, w.core, w.halo)
    rng = np.random.default_rng(7)
    c, hl = w.core, w.halo
    b, h = w.B - 1, w.nh - 1
    # a boundary along the tiled axes: the last position of a core and the first of the next
    ts = sorted({min(T - 1, t_) for t_ in (0, c[0] - 1, c[0], c[0] + hl[0], T - 1)})
    ys = sorted({min(Y - 1, y_) for y_ in (0, c[1] - 1, c[1], c[1] + hl[1])})
    xs = sorted({min(X - 1, x_) for x_ in (0, c[2] - 1, c[2], c[2] + hl[2])})
    rows = sorted({(tt * Y + yy) * X + xx for tt in ts for yy in ys for xx in xs})[:40]
    rows += [int(i) for i in rng.integers(0, w.N, 8)]
    assert all(0 <= i < w.N for i in rows)
    qs, ks, vs, gs = (_slice64(t, b, h) for t in (q, k, v, go))
    o_r, dq_r = oracle.forward_rows(geo1, qs, ks, vs, [(0, 0, i) for i in rows], dout=gs)
    for nm, got, ref in (("out", out[b, h, rows], o_r), ("dq", dq[b, h, rows], dq_r)):
        mx, rms = _errs(got.double().cpu().numpy(), ref)
        assert mx <= MAX_REL and rms <= RMS_REL, (name, nm, mx, rms)
