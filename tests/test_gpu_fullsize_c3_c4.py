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
