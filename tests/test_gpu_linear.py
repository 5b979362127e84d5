"""Factorised linear attention on the GPU (gattn_linear_fwd) against the FP64
oracle (``oracle/linear.py``): phi = elu + 1 summary and normaliser, BF16
inputs, d = 64.  Tolerances: max-rel <= 2e-2, rms-rel <= 3e-3 per (batch,
head).  Cases: one partial tile, ragged N (not a multiple of 128), several
chunks per (batch, head) with the fixed-order combine, and the full-size
workload (N = 262144, B = 4, 16 heads) on sampled rows.
"""
import numpy as np
import pytest
import torch

from oracle import linear as ol
from paper_2604_16590_gb300 import gattn
from paper_2604_16590_gb300.inputs import qkv
from tests._parity import assert_close

pytestmark = pytest.mark.gpu

CASES = [("one_partial_tile", 1, 1, 100), ("three_tiles_two_heads", 1, 2, 300), ("ragged", 2, 3, 1000),
         ("n4096", 1, 1, 4096), ("many_chunks", 1, 2, 65536 + 77)]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_matches_oracle(case):
    name, B, nh, N = case
    q, k, v = qkv((B, nh, N, 64), 31 + N, 0.5, "bf16", "cuda")
    out = gattn.linear_forward(q, k, v)
    assert gattn.gattn_stream_status() == 0
    ref = ol.forward(*(t.double().cpu().numpy() for t in (q, k, v)))
    assert_close(name, out.double().cpu().numpy(), ref, 2e-2, 3e-3)


def test_deterministic():
    q, k, v = qkv((1, 2, 20000, 64), 5, 0.5, "bf16", "cuda")
    assert torch.equal(gattn.linear_forward(q, k, v), gattn.linear_forward(q, k, v))


def test_full_size_sampled_rows():
    """N = 262144 (32 x 64 x 128 tokens), B = 4, 16 heads: the bench workload."""
    B, nh, N = 4, 16, 32 * 64 * 128
    q, k, v = qkv((B, nh, N, 64), 20262, 0.5, "bf16", "cuda")
    out = gattn.linear_forward(q, k, v)
    rng = np.random.default_rng(1)
    heads = [(0, 0), (3, 15), (2, 7)]
    for b, h in heads:
        S, z = ol.summary(k[b:b + 1, h:h + 1].double().cpu().numpy(), v[b:b + 1, h:h + 1].double().cpu().numpy())
        rows = np.concatenate([[0, N - 1], rng.integers(0, N, 62)])
        qq = q[b:b + 1, h:h + 1].double().cpu().numpy()
        ref = ol.forward_rows(qq, None, None, [(0, 0, int(i)) for i in rows], S, z)
        got = out[b, h, torch.as_tensor(rows, device="cuda")].double().cpu().numpy()
        assert_close(f"full/{b}/{h}", got, ref, 2e-2, 3e-3)


def test_invalid_arguments():
    q, k, v = qkv((1, 1, 256, 64), 9, 0.5, "bf16", "cuda")
    desc = gattn.linear_desc(q)
    ws = torch.empty(gattn.gattn_linear_workspace_bytes(desc), dtype=torch.uint8, device="cuda")
    out = torch.empty_like(q)
    assert gattn.gattn_linear_fwd(desc, q, k, v, out, ws, ws_bytes=ws.numel() - 16) == 3
    desc.d = 128
    assert gattn.gattn_linear_fwd(desc, q, k, v, out, ws) == 1


# ---------------------------------------------------------------- backward
BWD_CASES = [("one_partial_tile", 1, 1, 100), ("three_tiles_two_heads", 1, 2, 300), ("ragged", 2, 3, 1000),
             ("n4096", 1, 1, 4096), ("many_chunks", 1, 2, 65536 + 77)]


def _bwd_inputs(B, nh, N, seed):
    q, k, v = qkv((B, nh, N, 64), seed, 0.5, "bf16", "cuda")
    (g,) = qkv((B, nh, N, 64), seed + 7919, 1.0, "bf16", "cuda", n=1)
    return q, k, v, g


@pytest.mark.parametrize("case", BWD_CASES, ids=[c[0] for c in BWD_CASES])
def test_backward_matches_oracle(case):
    """dq, dk, dv of sum(out * g) against the oracle's analytic gradient (itself
    pinned by torch autograd of the O(N^2) form and by finite differences)."""
    name, B, nh, N = case
    q, k, v, g = _bwd_inputs(B, nh, N, 77 + N)
    out, saved = gattn.linear_forward(q, k, v, keep_summary=True)
    dq, dk, dv = gattn.linear_backward(q, k, v, g, saved)
    assert gattn.gattn_stream_status() == 0
    ref = ol.backward(*(t.double().cpu().numpy() for t in (q, k, v, g)))
    for nm, got, r in zip(("dq", "dk", "dv"), (dq, dk, dv), ref):
        assert_close(f"{name}/{nm}", got.double().cpu().numpy(), r, 2e-2, 3e-3)


def test_backward_deterministic_and_autograd():
    """The autograd op gives the same gradients as the direct calls, bitwise,
    and two runs agree bitwise (fixed-order partial sums, no atomics)."""
    q, k, v, g = _bwd_inputs(1, 2, 3000, 12)
    out, saved = gattn.linear_forward(q, k, v, keep_summary=True)
    ref = gattn.linear_backward(q, k, v, g, saved)
    again = gattn.linear_backward(q, k, v, g, saved)
    qa, ka, va = (t.clone().requires_grad_(True) for t in (q, k, v))
    o = gattn.linear_attention(qa, ka, va)
    assert torch.equal(o, out)
    got = torch.autograd.grad(o, (qa, ka, va), g)
    for a_, b_, c_ in zip(ref, again, got):
        assert torch.equal(a_, b_) and torch.equal(a_, c_)


def test_backward_directional_finite_difference():
    """<grad, direction> of L = sum(out * g) from the GPU against a central
    finite difference of the FP64 operator (step 1e-6) along a random
    direction in q, k and v together."""
    B, nh, N = 1, 1, 700
    q, k, v, g = _bwd_inputs(B, nh, N, 5)
    out, saved = gattn.linear_forward(q, k, v, keep_summary=True)
    grads = gattn.linear_backward(q, k, v, g, saved)
    x = [t.double().cpu().numpy() for t in (q, k, v)]
    gg = g.double().cpu().numpy()
    rng = np.random.default_rng(3)
    dirs = [rng.standard_normal(t.shape) for t in x]
    eps = 1e-6
    plus = ol.forward(*(a + eps * d for a, d in zip(x, dirs)))
    minus = ol.forward(*(a - eps * d for a, d in zip(x, dirs)))
    fd = ((plus - minus) * gg).sum() / (2 * eps)
    an = sum((gr.double().cpu().numpy() * d).sum() for gr, d in zip(grads, dirs))
    scale = sum(np.abs(gr.double().cpu().numpy() * d).sum() for gr, d in zip(grads, dirs))
    assert abs(an - fd) <= 3e-3 * scale, (an, fd, scale)


def test_backward_full_size_sampled_rows():
    """N = 262144 (the bench shape), two (batch, head) slices: dq, dk, dv at
    sampled rows against the oracle (whole-slice gradients in FP64)."""
    B, nh, N = 2, 2, 32 * 64 * 128
    q, k, v, g = _bwd_inputs(B, nh, N, 20262)
    out, saved = gattn.linear_forward(q, k, v, keep_summary=True)
    dq, dk, dv = gattn.linear_backward(q, k, v, g, saved)
    rng = np.random.default_rng(2)
    rows = torch.as_tensor(np.concatenate([[0, N - 1], rng.integers(0, N, 126)]), device="cuda")
    for b, h in ((0, 0), (1, 1)):
        sl = [t[b:b + 1, h:h + 1].double().cpu().numpy() for t in (q, k, v, g)]
        ref = ol.backward(*sl)
        for nm, got, r in zip(("dq", "dk", "dv"), (dq, dk, dv), ref):
            assert_close(f"full/{b}/{h}/{nm}", got[b, h, rows].double().cpu().numpy(),
                         r[0, 0][rows.cpu().numpy()], 2e-2, 3e-3)


def test_backward_invalid_arguments():
    q, k, v, g = _bwd_inputs(1, 1, 256, 9)
    out, saved = gattn.linear_forward(q, k, v, keep_summary=True)
    desc = gattn.linear_desc(q)
    ws = torch.empty(gattn.gattn_linear_bwd_workspace_bytes(desc), dtype=torch.uint8, device="cuda")
    dq, dk, dv = (torch.empty_like(q) for _ in range(3))
    assert gattn.gattn_linear_bwd(desc, q, k, v, g, saved, dq, dk, dv, ws, ws_bytes=ws.numel() - 16) == 3
    assert gattn.gattn_linear_bwd(desc, q, k, v, g, saved, dq, dk, dv, ws, saved_bytes=saved.numel() - 16) == 3
    assert gattn.gattn_linear_bwd(desc, q, k, v, None, saved, dq, dk, dv, ws) == 1
