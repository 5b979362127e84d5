"""Temporal compression on the GPU (gattn_compress_fwd) against the FP64
oracle (``oracle/compress.py``), on the same seeded inputs.

Learned query per head over the S history frames of every location
(arXiv 2604.16590, Sec. III-B).  Tolerances: BF16 inputs max-rel <= 2e-2 and
rms-rel <= 3e-3 per (batch, head) slice; FP32 inputs 1e-5 relative.  The
cases cover one frame and one location, ragged frame tails (S not a multiple
of the four-frame step), the 256-frame inner-block boundary, ragged location
blocks (M not a multiple of 32), split frame ranges with their merge, d = 32,
64, 128, long histories (S = 65536 and 131072, the compensated sums), and the
full-size workload on sampled locations.
"""
import numpy as np
import pytest
import torch

from oracle import compress as oc
from paper_2604_16590_gb300 import gattn, inputs
from tests._parity import assert_close, rel_errors

pytestmark = pytest.mark.gpu

BF16_MAX, BF16_RMS = 2e-2, 3e-3
FP32_REL = 1e-5

# (name, B, nh, S, M, d)
CASES = [
    ("one_frame_one_location", 1, 1, 1, 1, 64),
    ("ragged_tail_ragged_m", 2, 3, 7, 33, 64),
    ("inner_block_boundary", 1, 2, 257, 70, 128),
    ("exact_inner_blocks", 1, 1, 512, 32, 64),
    ("split_few_locations", 1, 8, 1000, 5, 64),
    ("split_d128", 2, 2, 1543, 3, 128),
    ("many_locations", 2, 2, 64, 1000, 128),
]


def _inputs(B, nh, S, M, d, dtype, seed):
    k, v = inputs.qkv((B, nh, S, M, d), seed, 0.5, dtype, "cuda", n=2)
    g = torch.Generator(device="cuda")
    g.manual_seed(seed + 1)
    q = torch.randn((nh, d), generator=g, device="cuda", dtype=torch.float32)
    return q, k, v


def _oracle(q, k, v):
    return oc.forward(q.double().cpu().numpy(), k.double().cpu().numpy(), v.double().cpu().numpy())


@pytest.mark.parametrize("out_dtype", [torch.bfloat16, torch.float32], ids=["out_bf16", "out_fp32"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_bf16_matches_oracle(case, out_dtype):
    name, B, nh, S, M, d = case
    q, k, v = _inputs(B, nh, S, M, d, "bf16", seed=sum(map(ord, name)))
    out, lse = gattn.compress_forward(q, k, v, out_dtype=out_dtype)
    assert gattn.gattn_stream_status() == 0
    ref, ref_lse = _oracle(q, k, v)
    assert_close(f"{name}/out", out.double().cpu().numpy(), ref, BF16_MAX, BF16_RMS)
    np.testing.assert_allclose(lse.double().cpu().numpy(), ref_lse, rtol=1e-5, atol=1e-5)


@pytest.mark.parametrize("d", [32, 64, 128])
@pytest.mark.parametrize("S,M", [(1, 3), (37, 45), (700, 4)])
def test_fp32_matches_oracle(d, S, M):
    q, k, v = _inputs(1, 2, S, M, d, "fp32", seed=d * 1000 + S + M)
    out, lse = gattn.compress_forward(q, k, v)
    ref, ref_lse = _oracle(q, k, v)
    mx, rms = rel_errors(out.double().cpu().numpy(), ref)
    assert mx <= FP32_REL and rms <= FP32_REL, (mx, rms)
    np.testing.assert_allclose(lse.double().cpu().numpy(), ref_lse, rtol=1e-6, atol=1e-6)


def test_constant_values_come_back_exactly_in_fp32():
    """Normalised: a location whose value is the same in every frame returns it."""
    q, k, v = _inputs(1, 2, 300, 40, 64, "fp32", seed=5)
    v[:] = v[:, :, :1].clone()
    out, _ = gattn.compress_forward(q, k, v)
    ref = v[:, :, 0]
    assert torch.allclose(out, ref, rtol=1e-5, atol=1e-5)


def test_long_history_fp32_compensated_sums():
    """S = 65536 frames: the blocked sums keep FP32 within 1e-5 of FP64."""
    q, k, v = _inputs(1, 2, 65536, 8, 64, "fp32", seed=6)
    desc = gattn.compress_desc(k)
    assert gattn.gattn_compress_workspace_bytes(desc) > 0  # split path
    out, lse = gattn.compress_forward(q, k, v)
    ref, ref_lse = _oracle(q, k, v)
    mx, rms = rel_errors(out.double().cpu().numpy(), ref)
    assert mx <= FP32_REL and rms <= FP32_REL, (mx, rms)
    np.testing.assert_allclose(lse.double().cpu().numpy(), ref_lse, rtol=1e-6, atol=1e-6)


def test_long_history_bf16_workload():
    """The 131072-frame history workload; 8 of its 64 locations checked."""
    w = inputs.HISTORY_WORKLOADS["h_128k"]
    q, k, v = inputs.history_inputs(w, "cuda")
    out, lse = gattn.compress_forward(q, k, v)
    sel = torch.tensor([0, 7, 9, 20, 33, 47, 58, 63], device="cuda")
    ref, ref_lse = _oracle(q, k[:, :, :, sel], v[:, :, :, sel])
    assert_close("h_128k/out", out[:, :, sel].double().cpu().numpy(), ref, BF16_MAX, BF16_RMS)
    np.testing.assert_allclose(lse[:, :, sel].double().cpu().numpy(), ref_lse, rtol=1e-5, atol=1e-5)


def test_split_path_is_deterministic():
    q, k, v = _inputs(1, 4, 3000, 6, 128, "bf16", seed=7)
    a, la = gattn.compress_forward(q, k, v)
    b, lb = gattn.compress_forward(q, k, v)
    assert torch.equal(a, b) and torch.equal(la, lb)


def test_full_size_workload_sampled_locations():
    """The bench workload (2048 frames x 32 x 64, 8 heads, d = 128, BF16) in
    the bench's launch configuration; 48 sampled locations against the oracle."""
    w = inputs.HISTORY_WORKLOADS["h3_2k"]
    q, k, v = inputs.history_inputs(w, "cuda")
    out, lse = gattn.compress_forward(q, k, v)
    rng = np.random.default_rng(8)
    locs = [(0, 0, 0), (0, w.nh - 1, w.M - 1), (0, 3, 31), (0, 5, 32)]
    locs += [(0, int(h), int(m)) for h, m in zip(rng.integers(0, w.nh, 44), rng.integers(0, w.M, 44))]
    got, ref = [], []
    for b, h, m in locs:
        kl = k[b, h, :, m].double().cpu().numpy()[None, None, :, None, :]  # [1, 1, S, 1, d]
        vl = v[b, h, :, m].double().cpu().numpy()[None, None, :, None, :]
        ro, rl = oc.forward(q[h:h + 1].double().cpu().numpy(), kl, vl)
        g = out[b, h, m].double().cpu().numpy()
        assert np.abs(g - ro[0, 0, 0]).max() / np.abs(ro[0, 0, 0]).max() <= BF16_MAX
        assert abs(float(lse[b, h, m]) - rl[0, 0, 0]) <= 1e-5 * max(1.0, abs(rl[0, 0, 0]))
        got.append(g)
        ref.append(ro[0, 0, 0])
    got, ref = np.array(got), np.array(ref)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= BF16_RMS


def test_invalid_arguments_are_rejected_before_launch():
    q, k, v = _inputs(1, 1, 4, 4, 64, "bf16", seed=9)
    desc = gattn.compress_desc(k)
    out = torch.empty((1, 1, 4, 64), dtype=torch.bfloat16, device="cuda")
    desc.S = 0
    assert gattn.gattn_compress_fwd(desc, q, k, v, out, None, None) == 1
    desc = gattn.compress_desc(k)
    desc.d = 32  # BF16 needs d in {64, 128}
    assert gattn.gattn_compress_fwd(desc, q, k, v, out, None, None) == 1
    q2, k2, v2 = _inputs(1, 8, 1000, 5, 64, "bf16", seed=10)
    desc = gattn.compress_desc(k2)
    out2 = torch.empty((1, 8, 5, 64), dtype=torch.bfloat16, device="cuda")
    assert gattn.gattn_compress_workspace_bytes(desc) > 0
    assert gattn.gattn_compress_fwd(desc, q2, k2, v2, out2, None, None) == 3  # workspace missing
