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
