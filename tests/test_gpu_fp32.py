"""Parity of the plain FP32 form (SIMT kernels) with the FP64 oracle.

Every case runs through the C ABI (gattn_fwd / gattn_bwd) on cuda:0 and is
compared element by element with the oracle on the same seeded inputs.
Tolerance of the FP32 form: max-rel and rms-rel <= 1e-5 per output and
(batch, head) for FP32 outputs; 4e-3 max-rel for BF16 outputs (one BF16
rounding, 2^-8 relative, of each output element).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2604_16590_gb300 import build, gattn
from paper_2604_16590_gb300.inputs import qkv, upstream_grad
from tests._parity import assert_close

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5

CASES = [
    # name, B, nh, d, grid, core, halo, window
    ("c1_4k_16tiles", 1, 1, 64, (1, 64, 64), (1, 16, 16), (0, 4, 4), "hann"),
    ("ragged_all_dims", 2, 2, 32, (3, 10, 13), (2, 4, 5), (1, 2, 2), "hann"),
    ("d128_temporal", 1, 2, 128, (12, 8, 8), (4, 8, 8), (2, 0, 0), "hann"),
    ("one_tile_global", 1, 2, 64, (1, 16, 24), (1, 16, 24), (0, 0, 0), "hann"),
    ("halo0_blockdiag", 1, 1, 64, (2, 16, 16), (1, 8, 8), (0, 0, 0), "hann"),
    ("flat_window", 1, 1, 32, (1, 24, 24), (1, 8, 8), (0, 3, 3), "flat"),
    ("wide_halo", 1, 1, 64, (1, 20, 20), (1, 4, 4), (0, 3, 3), "hann"),
    ("single_token", 1, 1, 32, (1, 1, 1), (1, 1, 1), (0, 0, 0), "hann"),
]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    gattn.load_library()


def _run(B, nh, d, grid, core, halo, window, seed, out_dtype=torch.float32, with_bwd=True):
    T, Y, X = grid
    shape = (B, nh, T * Y * X, d)
    q, k, v = qkv(shape, seed, 1.0, "fp32")
    go = upstream_grad(shape, seed, "fp32")
    dev = torch.device("cuda:0")
    tq, tk, tv, tg = (t.to(dev) for t in (q, k, v, go))
    tiling = gattn.Tiling(grid, core, halo, window)
    out, saved = gattn.forward(tq, tk, tv, tiling, out_dtype=out_dtype)
    res = {"out": out}
    if with_bwd:
        res["dq"], res["dk"], res["dv"] = gattn.backward(tq, tk, tv, out, tg, saved, tiling)
    torch.cuda.synchronize()
    assert gattn.gattn_stream_status() == 0
    geo = oracle.Geometry(B, nh, d, T, Y, X, core, halo, window)
    ref = {"out": oracle.forward(geo, q.numpy(), k.numpy(), v.numpy())}
    if with_bwd:
        ref["dq"], ref["dk"], ref["dv"] = oracle.backward(geo, q.numpy(), k.numpy(), v.numpy(), go.numpy())
    return {n: t.float().cpu().numpy() for n, t in res.items()}, ref


@pytest.mark.parametrize("name,B,nh,d,grid,core,halo,window", CASES, ids=[c[0] for c in CASES])
def test_fp32_form_matches_oracle(name, B, nh, d, grid, core, halo, window):
    got, ref = _run(B, nh, d, grid, core, halo, window, seed=1000 + len(name))
    for key in ("out", "dq", "dk", "dv"):
        assert_close(f"{name}/{key}", got[key], ref[key], FP32_TOL, FP32_TOL)


def test_fp32_inputs_bf16_outputs():
    got, ref = _run(1, 2, 64, (2, 16, 16), (1, 8, 8), (1, 2, 2), "hann", seed=77, out_dtype=torch.bfloat16)
    for key in ("out", "dq", "dk", "dv"):
        assert_close(f"bf16out/{key}", got[key], ref[key], 4e-3, 4e-3)


def test_fp32_form_is_deterministic():
    a, _ = _run(1, 2, 64, (2, 24, 24), (1, 8, 8), (1, 4, 4), "hann", seed=5)
    b, _ = _run(1, 2, 64, (2, 24, 24), (1, 8, 8), (1, 4, 4), "hann", seed=5)
    for key in a:
        assert np.array_equal(a[key], b[key]), key


def test_autograd_function_matches_oracle():
    grid, core, halo = (1, 16, 16), (1, 8, 8), (0, 2, 2)
    shape = (1, 2, 256, 32)
    q, k, v = qkv(shape, 9, 1.0, "fp32")
    go = upstream_grad(shape, 9, "fp32")
    dev = torch.device("cuda:0")
    tq, tk, tv = (t.to(dev).requires_grad_(True) for t in (q, k, v))
    out = gattn.global_attention(tq, tk, tv, gattn.Tiling(grid, core, halo))
    out.backward(go.to(dev))
    geo = oracle.Geometry(1, 2, 32, *grid, core, halo)
    dq, dk, dv = oracle.backward(geo, q.numpy(), k.numpy(), v.numpy(), go.numpy())
    assert_close("autograd/out", out.detach().cpu().numpy(), oracle.forward(geo, q.numpy(), k.numpy(), v.numpy()), FP32_TOL, FP32_TOL)
    for name, t, r in (("dq", tq, dq), ("dk", tk, dk), ("dv", tv, dv)):
        assert_close(f"autograd/{name}", t.grad.cpu().numpy(), r, FP32_TOL, FP32_TOL)
