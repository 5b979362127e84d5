"""Parity at the benchmark's full size and launch configuration: the 32 x 64 x
128 grid, batch 4, 16 heads, d = 64, Tiles = 16 (core 32x16x32, halo 0/4/8),
BF16 inputs and outputs, the same seeded inputs as bench.py.

The oracle cannot evaluate the whole operator at this size, so the test checks
(a) sampled rows of Out and dQ, which the oracle computes row by row, (b) dK
and dV of sampled keys of one tile and of keys two tiles share, and (c) two exact identities of the
operator at every size: per (batch, head) the dV rows sum to the dOut rows
(each softmax row and each set of merge weights sums to one) and the dK rows
sum to zero (each row of dS sums to zero)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2604_16590_gb300 import build, gattn
from paper_2604_16590_gb300.inputs import WORKLOADS, workload_inputs

pytestmark = pytest.mark.gpu

MAX_REL, RMS_REL = 2e-2, 3e-3


@pytest.fixture(scope="module")
def run():
    build.build()
    gattn.load_library()
    w = WORKLOADS["c2_262k_p"]
    q, k, v, go = workload_inputs(w, device="cuda")
    tiling = gattn.Tiling(w.grid, w.core, w.halo)
    out, saved = gattn.forward(q, k, v, tiling, out_dtype=torch.bfloat16)
    dq, dk, dv = gattn.backward(q, k, v, out, go, saved, tiling)
    assert gattn.gattn_stream_status() == 0
    del saved
    return w, (q, k, v, go), (out, dq, dk, dv)


def _slice64(t, b, h):
    return np.ascontiguousarray(t[b, h].double().cpu().numpy())[None, None]


def _errs(got, ref):
    got, ref = np.asarray(got), np.asarray(ref)
    return np.abs(got - ref).max() / np.abs(ref).max(), np.linalg.norm(got - ref) / np.linalg.norm(ref)


def test_sampled_rows_of_out_and_dq(run):
    w, (q, k, v, go), (out, dq, _, _) = run
    T, Y, X = w.grid
    rng = np.random.default_rng(5)
    geo1 = oracle.Geometry(1, 1, w.d, T, Y, X, w.core, w.halo)
    got_o, ref_o, got_q, ref_q = [], [], [], []
    for b, h in [(0, 0), (1, 7), (3, 15)]:
        # rows on tile boundaries (multiply covered), in cores, and at random
        ys = [0, 14, 16, 19, 20, 31, 47, 63]
        xs = [0, 26, 32, 37, 40, 95, 100, 127]
        rows = [((int(rng.integers(T)) * Y + yy) * X + xx) for yy in ys for xx in xs[:2]]
        rows += [int(i) for i in rng.integers(0, w.N, 8)]
        qs, ks, vs, gs = (_slice64(t, b, h) for t in (q, k, v, go))
        o_r, dq_r = oracle.forward_rows(geo1, qs, ks, vs, [(0, 0, i) for i in rows], dout=gs)
        got_o.append(out[b, h, rows].double().cpu().numpy())
        got_q.append(dq[b, h, rows].double().cpu().numpy())
        ref_o.append(o_r)
        ref_q.append(dq_r)
    for name, g_, r_ in (("out", got_o, ref_o), ("dq", got_q, ref_q)):
        mx, rms = _errs(np.concatenate(g_), np.concatenate(r_))
        assert mx <= MAX_REL and rms <= RMS_REL, (name, mx, rms)


def test_sampled_keys_of_dk_dv(run):
    w, (q, k, v, go), (_, _, dk, dv) = run
    T, Y, X = w.grid
    geo1 = oracle.Geometry(1, 1, w.d, T, Y, X, w.core, w.halo)
    b, h = 2, 5
    # keys inside the core of tile (0, 1, 1) away from its halos (one tile's
    # backward), and keys in the overlap of tiles (0, 1, 1) and (0, 1, 2)
    # (x in [56, 72) is in both extended tiles, y in [20, 28) in one tile row):
    # their dK, dV are the fixed-order sums of two tiles' gradients (merge path)
    rng = np.random.default_rng(6)
    keys = [((int(t) * Y + int(y)) * X + int(x)) for t, y, x in zip(rng.integers(0, T, 12), rng.integers(20, 28, 12),
                                                                   rng.integers(40, 56, 12))]
    keys += [((int(t) * Y + int(y)) * X + int(x)) for t, y, x in zip(rng.integers(0, T, 8), rng.integers(20, 28, 8),
                                                                    rng.integers(56, 72, 8))]
    qs, ks, vs, gs = (_slice64(t, b, h) for t in (q, k, v, go))
    dk_r, dv_r = oracle.key_rows(geo1, qs, ks, vs, gs, [(0, 0, j) for j in keys])
    for name, got, ref in (("dk", dk[b, h, keys], dk_r), ("dv", dv[b, h, keys], dv_r)):
        mx, rms = _errs(got.double().cpu().numpy(), ref)
        assert mx <= MAX_REL and rms <= RMS_REL, (name, mx, rms)


def test_gradient_sum_identities(run):
    w, (_, _, _, go), (_, _, dk, dv) = run
    sdv = dv.double().sum(dim=2)
    sgo = go.double().sum(dim=2)
    rel = (sdv - sgo).norm() / sgo.norm()
    assert rel < 1e-3, float(rel)
    sdk = dk.double().sum(dim=2)
    scale = dk.double().abs().sum(dim=2)
    assert float((sdk.abs() / scale).max()) < 1e-3
