"""Parity of the BF16 tensor-core form (tcgen05 kernels) with the FP64 oracle.

The oracle runs on the same BF16-rounded inputs (as FP64), so input
quantisation is not counted as error.  Tolerance of the BF16 form, per output
and (batch, head): max-rel <= 2e-2 and rms-rel <= 3e-3 (P is rounded to BF16
before the P V product; accumulation is FP32 in tensor memory).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2604_16590_gb300 import build, gattn
from paper_2604_16590_gb300.inputs import qkv, upstream_grad
from tests._parity import assert_close

pytestmark = pytest.mark.gpu

MAX_REL, RMS_REL = 2e-2, 3e-3

FWD_CASES = [
    # name, B, nh, d, grid, core, halo
    ("p_like_small", 1, 2, 64, (4, 16, 32), (4, 8, 16), (0, 2, 4)),
    ("s_spec", 1, 1, 64, (2, 32, 32), (1, 16, 16), (0, 4, 4)),
    ("one_tile_1024", 1, 1, 64, (1, 32, 32), (1, 32, 32), (0, 0, 0)),
    ("ragged_all_dims", 2, 3, 64, (3, 10, 13), (2, 4, 5), (1, 2, 2)),
    ("d128_temporal", 1, 2, 128, (16, 8, 8), (8, 8, 8), (2, 0, 0)),
    ("long_tile_ring_wrap", 1, 1, 64, (8, 32, 32), (8, 16, 16), (0, 4, 4)),
    ("d128_s_spec", 1, 1, 128, (1, 48, 40), (1, 16, 16), (0, 4, 4)),
    # d = 128 with ragged tiles in all three dimensions (masked key boxes, padding rows)
    ("d128_ragged_all_dims", 2, 3, 128, (3, 10, 13), (2, 4, 5), (1, 2, 2)),
    # d = 128, several boxes per tile in every dimension and a long item (two K/V ring wraps)
    ("d128_multi_box", 1, 2, 128, (6, 24, 24), (3, 12, 12), (1, 2, 2)),
    # a halo almost as wide as the core: up to nine covering tiles per token (the merges' general path)
    ("wide_halo", 1, 1, 64, (1, 20, 20), (1, 4, 4), (0, 3, 3)),
    # degenerate: one token (a one-row box; every other key and query of the MMA blocks is padding)
    ("single_token", 1, 2, 64, (1, 1, 1), (1, 1, 1), (0, 0, 0)),
    ("single_token_d128", 1, 1, 128, (1, 1, 1), (1, 1, 1), (0, 0, 0)),
    # one 1x8x48 tile = three 1x8x16 boxes: the second box of the last query pair is empty
    ("odd_box_count", 1, 2, 64, (1, 8, 48), (1, 8, 48), (0, 0, 0)),
    # sum over dimensions of core + 2 halo = 2230, more than the merges' shared-memory
    # window table holds: the merge kernels evaluate the window directly
    ("window_direct", 1, 1, 64, (1, 1, 4200), (1, 1, 2100), (0, 0, 64)),
]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    gattn.load_library()


def _inputs(B, nh, d, grid, seed):
    shape = (B, nh, grid[0] * grid[1] * grid[2], d)
    q, k, v = qkv(shape, seed, 0.5, "bf16")
    go = upstream_grad(shape, seed, "bf16")
    return q, k, v, go


@pytest.mark.parametrize("name,B,nh,d,grid,core,halo", FWD_CASES, ids=[c[0] for c in FWD_CASES])
@pytest.mark.parametrize("out_dtype", [torch.float32, torch.bfloat16], ids=["out_fp32", "out_bf16"])
def test_bf16_forward_matches_oracle(name, B, nh, d, grid, core, halo, out_dtype):
    q, k, v, _ = _inputs(B, nh, d, grid, 300 + len(name))
    dev = torch.device("cuda:0")
    tiling = gattn.Tiling(grid, core, halo)
    out, _ = gattn.forward(q.to(dev), k.to(dev), v.to(dev), tiling, out_dtype=out_dtype)
    st = gattn.gattn_stream_status()
    assert st == 0, gattn.STATUS.get(st, st)
    geo = oracle.Geometry(B, nh, d, *grid, core, halo)
    ref = oracle.forward(geo, q.double().numpy(), k.double().numpy(), v.double().numpy())
    assert_close(f"{name}/out", out.double().cpu().numpy(), ref, MAX_REL, RMS_REL)


def test_bf16_forward_is_deterministic():
    grid, core, halo = (4, 32, 32), (2, 16, 16), (1, 4, 4)
    q, k, v, _ = _inputs(1, 2, 64, grid, 11)
    dev = torch.device("cuda:0")
    tiling = gattn.Tiling(grid, core, halo)
    a, _ = gattn.forward(q.to(dev), k.to(dev), v.to(dev), tiling, out_dtype=torch.float32)
    b, _ = gattn.forward(q.to(dev), k.to(dev), v.to(dev), tiling, out_dtype=torch.float32)
    assert torch.equal(a, b)


BWD_CASES = [c for c in FWD_CASES if c[0] != "long_tile_ring_wrap" and not c[0].startswith("single_token")] + [
    ("bwd_long_tile", 1, 1, 64, (4, 32, 32), (4, 16, 16), (0, 4, 4)),
]


@pytest.mark.parametrize("name,B,nh,d,grid,core,halo", BWD_CASES, ids=[c[0] for c in BWD_CASES])
@pytest.mark.parametrize("out_dtype", [torch.float32, torch.bfloat16], ids=["out_fp32", "out_bf16"])
def test_bf16_backward_matches_oracle(name, B, nh, d, grid, core, halo, out_dtype):
    q, k, v, go = _inputs(B, nh, d, grid, 500 + len(name))
    dev = torch.device("cuda:0")
    tq, tk, tv, tg = (t.to(dev) for t in (q, k, v, go))
    tiling = gattn.Tiling(grid, core, halo)
    out, saved = gattn.forward(tq, tk, tv, tiling, out_dtype=out_dtype)
    dq, dk, dv = gattn.backward(tq, tk, tv, out, tg, saved, tiling)
    st = gattn.gattn_stream_status()
    assert st == 0, gattn.STATUS.get(st, st)
    geo = oracle.Geometry(B, nh, d, *grid, core, halo)
    f64 = [t.double().numpy() for t in (q, k, v, go)]
    rq, rk, rv = oracle.backward(geo, *f64)
    for key, got, ref in (("dq", dq, rq), ("dk", dk, rk), ("dv", dv, rv)):
        assert_close(f"{name}/{key}", got.double().cpu().numpy(), ref, MAX_REL, RMS_REL)


def test_bf16_backward_is_deterministic():
    grid, core, halo = (4, 32, 32), (2, 16, 16), (1, 4, 4)
    q, k, v, go = _inputs(1, 2, 64, grid, 12)
    dev = torch.device("cuda:0")
    tq, tk, tv, tg = (t.to(dev) for t in (q, k, v, go))
    tiling = gattn.Tiling(grid, core, halo)
    out, saved = gattn.forward(tq, tk, tv, tiling, out_dtype=torch.float32)
    a = gattn.backward(tq, tk, tv, out, tg, saved, tiling)
    b = gattn.backward(tq, tk, tv, out, tg, saved, tiling)
    for x, y in zip(a, b):
        assert torch.equal(x, y)


@pytest.mark.parametrize("d", [64, 128])
@pytest.mark.parametrize("out_dtype", [torch.float32, torch.bfloat16], ids=["out_fp32", "out_bf16"])
def test_single_token_backward(d, out_dtype):
    """One token, one tile: the output is V, so dV = dOut exactly and dQ = dK = 0
    (the softmax over one key is the constant 1).  dQ and dK come out as
    P (dP - D) with dP = dOut . V from the tensor core and D = dOut . Out from the
    stored output: small, not exactly zero."""
    q, k, v, go = _inputs(1, 2, d, (1, 1, 1), 77)
    dev = torch.device("cuda:0")
    tq, tk, tv, tg = (t.to(dev) for t in (q, k, v, go))
    tiling = gattn.Tiling((1, 1, 1), (1, 1, 1), (0, 0, 0))
    out, saved = gattn.forward(tq, tk, tv, tiling, out_dtype=out_dtype)
    dq, dk, dv = gattn.backward(tq, tk, tv, out, tg, saved, tiling)
    st = gattn.gattn_stream_status()
    assert st == 0, gattn.STATUS.get(st, st)
    assert_close("single/out", out.double().cpu().numpy(), v.double().numpy(), MAX_REL, RMS_REL)
    assert_close("single/dv", dv.double().cpu().numpy(), go.double().numpy(), MAX_REL, RMS_REL)
    bound = (1e-3 if out_dtype == torch.float32 else 2e-2) * float(go.abs().max()) * float(v.abs().max())
    for name, t in (("dq", dq), ("dk", dk)):
        assert float(t.abs().max()) <= bound, (name, float(t.abs().max()), bound)
