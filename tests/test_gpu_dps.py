"""Posterior-sampling steps on the GPU (gattn_dps_step) against the FP64
oracle (``oracle/dps.py``), arXiv 2604.16590, Sec. III-A and III-C.

One step = GPA forward (the synthetic denoiser), residual of the masked
observations, GPA backward with that residual as dOut, and the reverse-SDE
update.  Compared: the increment z_next - z, per (batch, head) slice, for one
step and for a five-step trajectory on shared noise.  Tolerances: BF16 the GPA
ones (max-rel <= 2e-2, rms-rel <= 3e-3 of the increment); FP32 4e-5: the
increment is a weighted sum of four GPA outputs (D and the three gradients
that form J^T r), each within 1e-5 of its own scale, with weights delta /
sigma^2 and lam * delta of order one.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import dps as od
from paper_2604_16590_gb300 import gattn
from tests._parity import assert_close

pytestmark = pytest.mark.gpu

CASES = [
    ("halo_2d", 1, 2, 64, (1, 32, 48), (1, 16, 16), (0, 4, 4)),
    ("ragged_3d", 2, 1, 64, (2, 20, 28), (2, 8, 12), (0, 2, 3)),
]


def _state(B, nh, N, d, seed):
    g = torch.Generator().manual_seed(seed)
    z = torch.randn((B, nh, N, d), generator=g) * 0.7
    y = torch.randn((B, nh, N, d), generator=g) * 0.5
    mask = (torch.rand((B, N), generator=g) < 0.25).to(torch.uint8)
    return z, y, mask


@pytest.mark.parametrize("attn", ["bf16", "fp32"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_steps_match_oracle(case, attn):
    name, B, nh, d, grid, core, halo = case
    N = grid[0] * grid[1] * grid[2]
    z, y, mask = _state(B, nh, N, d, 1000 + N)
    geo = oracle.Geometry(B, nh, d, *grid, core, halo)
    sampler = gattn.PosteriorSampler(z.cuda(), gattn.Tiling(grid, core, halo), attn)
    sig = od.sigma_schedule(5, 1.5, 0.1)
    zr = z.double().numpy()
    tol = (2e-2, 3e-3) if attn == "bf16" else (4e-5, 4e-5)
    g = torch.Generator().manual_seed(7)
    worst = (0.0, 0.0)
    for i in range(5):
        eps = torch.randn(z.shape, generator=g)
        before = sampler.z.double().cpu().numpy()
        sampler.step(y.cuda(), mask.cuda(), eps.cuda(), sig[i], sig[i + 1], 0.8)
        assert gattn.gattn_stream_status() == 0
        got = sampler.z.double().cpu().numpy()
        # one step from the GPU's own state (no drift between the trajectories)
        ref, _ = od.step(geo, before, y.double().numpy(), mask.double().numpy(), eps.double().numpy(),
                         sig[i], sig[i + 1], 0.8, attn_dtype="bf16" if attn == "bf16" else "fp64")
        mx, rms = assert_close(f"{name}/{attn}/step{i}", got - before, ref - before, *tol)
        worst = (max(worst[0], mx), max(worst[1], rms))
        zr, _ = od.step(geo, zr, y.double().numpy(), mask.double().numpy(), eps.double().numpy(),
                        sig[i], sig[i + 1], 0.8, attn_dtype="bf16" if attn == "bf16" else "fp64")
    # the five-step trajectory stays close to the oracle's own trajectory
    traj = np.linalg.norm(sampler.z.double().cpu().numpy() - zr) / np.linalg.norm(zr - z.double().numpy())
    # the measured margins (shown with pytest -s)
    print(f"{name}/{attn}: worst step max-rel {worst[0]:.2e} rms-rel {worst[1]:.2e}, trajectory {traj:.2e}")
    assert traj <= (2e-2 if attn == "bf16" else 4e-5), traj


def test_bf16_copy_tracks_the_state():
    z, y, mask = _state(1, 1, 16 * 16, 64, 3)
    sampler = gattn.PosteriorSampler(z.cuda(), gattn.Tiling((1, 16, 16), (1, 8, 8), (0, 2, 2)), "bf16")
    sampler.step(y.cuda(), mask.cuda(), torch.randn(z.shape).cuda(), 1.0, 0.5, 0.3)
    assert torch.equal(sampler.zb, sampler.z.to(torch.bfloat16))


def test_invalid_parameters_are_rejected():
    z, y, mask = _state(1, 1, 16 * 16, 64, 4)
    s = gattn.PosteriorSampler(z.cuda(), gattn.Tiling((1, 16, 16), (1, 8, 8), (0, 2, 2)), "bf16")
    p = gattn.gattn_dps_params()
    p.sigma, p.sigma_next, p.lam = 0.5, 0.9, 1.0  # sigma must not grow
    eps = torch.zeros_like(s.z)
    assert gattn.gattn_dps_step(s.desc, p, s.z, s.zb, y.cuda(), mask.cuda(), eps, s.ws) == 1
    p.sigma_next = 0.2
    assert gattn.gattn_dps_step(s.desc, p, s.z, s.zb, y.cuda(), mask.cuda(), eps, s.ws,
                                ws_bytes=s.ws.numel() - 256) == 3
