"""Noise-gated self + cross attention on the GPU (gattn_gated_fwd) against the
FP64 oracle (``oracle/gated.py``), arXiv 2604.16590, Sec. III-B.

Queries from the current state attend tile-locally to their own keys/values
(self) and to the compressed temporal representation (cross); the per-head
gate blends the two.  Tolerances as for GPA: BF16 max-rel <= 2e-2, rms-rel
<= 3e-3; FP32 1e-5.  Cases: halos with multiply-covered rows, ragged tiles,
gates 0 and 1 and in between, d = 64 and 128.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import gated as og
from paper_2604_16590_gb300 import gattn
from paper_2604_16590_gb300.inputs import qkv
from tests._parity import assert_close

pytestmark = pytest.mark.gpu

# name, B, nh, d, grid, core, halo
CASES = [
    ("halo_2d", 1, 3, 64, (1, 32, 48), (1, 16, 16), (0, 4, 4)),
    ("ragged_3d", 2, 2, 64, (3, 20, 28), (2, 8, 12), (1, 2, 3)),
    ("d128", 1, 2, 128, (1, 24, 40), (1, 12, 16), (0, 3, 4)),
]


def _gate(nh):
    return torch.tensor([0.0, 1.0, 0.3, 0.75][:nh] if nh <= 4 else np.linspace(0, 1, nh), dtype=torch.float32)


@pytest.mark.parametrize("dtype", ["bf16", "fp32"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_gated_matches_oracle(case, dtype):
    name, B, nh, d, grid, core, halo = case
    N = grid[0] * grid[1] * grid[2]
    std = 0.5 if dtype == "bf16" else 1.0
    q, k, v, kc, vc = qkv((B, nh, N, d), 4242 + N, std, dtype, "cuda", n=5)
    gate = _gate(nh)
    tiling = gattn.Tiling(grid, core, halo)
    out = gattn.gated_forward(q, k, v, kc, vc, gate.cuda(), tiling, out_dtype=torch.float32)
    assert gattn.gattn_stream_status() == 0
    geo = oracle.Geometry(B, nh, d, *grid, core, halo)
    ref = og.forward(geo, *(t.double().cpu().numpy() for t in (q, k, v, kc, vc)), gate.numpy())
    tol = (2e-2, 3e-3) if dtype == "bf16" else (1e-5, 1e-5)
    assert_close(f"{name}/{dtype}", out.double().cpu().numpy(), ref, *tol)


def test_short_workspace_is_rejected():
    q, k, v = qkv((1, 2, 16 * 16, 64), 7, 0.5, "bf16", "cuda")
    tiling = gattn.Tiling((1, 16, 16), (1, 8, 8), (0, 2, 2))
    desc = gattn.desc_for(q, tiling)
    need = gattn.gattn_gated_workspace_bytes(desc)
    ws = torch.empty(need - 256, dtype=torch.uint8, device="cuda")
    out = torch.empty_like(q)
    gate = torch.zeros(2, device="cuda")
    assert gattn.gattn_gated_fwd(desc, q, k, v, k, v, gate, out, ws) == 3
