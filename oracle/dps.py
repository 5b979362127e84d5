"""FP64 CPU oracle of one diffusion-posterior-sampling step with the GPA
denoiser (arXiv 2604.16590, Sec. III-A "Diffusion-based posterior sampling",
Eqs. reverse:SDE, score_decomp, dps_final and Eq. denoise; Sec. III-C, the
propagation of context across tiles over denoising steps).

TEST INFRASTRUCTURE ONLY (same rule as the rest of ``oracle/``).

The step, in the paper's terms:
  * denoised estimate  D = D(z)  -- here a synthetic one-layer denoiser, the
    GPA operator on the state: D(z) = GPA(z, z, z) (heads as channels);
  * prior score        S_prior = (D - z) / sigma^2                  (Eq. denoise)
  * likelihood score   S_lik = -lam * J_D(z)^T H^T (H D - y)         (Eq. dps_final,
    H a mask that observes whole tokens, Gaussian errors; lam folds zeta_t, the
    factor 2 and the error variance into one guidance weight)
  * posterior score    S = S_prior + S_lik                           (Eq. score_decomp)
  * reverse SDE step from sigma to sigma_next < sigma (Euler-Maruyama of the
    variance-exploding reverse SDE, Eq. reverse:SDE, whose drift and diffusion
    integrate to delta = sigma^2 - sigma_next^2 over the step):
        z_next = z + delta * S + sqrt(delta) * eps

The attention can read a BF16 rounding of the state (``attn_dtype="bf16"``,
the GPU's tensor-core form; the upstream gradient H^T (H D - y) is then rounded
to BF16 as well); everything else is FP64.
"""
from __future__ import annotations

import numpy as np
import torch

from . import backward as gpa_backward
from . import forward as gpa_forward


def bf16_round(a) -> np.ndarray:
    """Round-to-nearest-even to bfloat16, returned as float64."""
    t = torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float32)))
    return t.to(torch.bfloat16).to(torch.float64).numpy()


def step(geo, z, y, mask, eps, sigma: float, sigma_next: float, lam: float, attn_dtype: str = "fp64"):
    """One posterior-sampling step; z, y, eps [B, nh, N, d]; mask [B, N] (1 = observed).
    Returns (z_next, D)."""
    z = np.asarray(z, dtype=np.float64)
    m = np.asarray(mask, dtype=np.float64)[:, None, :, None]
    za = bf16_round(z) if attn_dtype == "bf16" else z
    D = gpa_forward(geo, za, za, za)
    r = m * (D - np.asarray(y, dtype=np.float64))
    if attn_dtype == "bf16":
        r = bf16_round(r)
    dq, dk, dv = gpa_backward(geo, za, za, za, r)
    score = (D - z) / sigma**2 - lam * (dq + dk + dv)
    delta = sigma**2 - sigma_next**2
    return z + delta * score + np.sqrt(delta) * np.asarray(eps, dtype=np.float64), D


def sigma_schedule(n: int, sigma_max: float = 2.0, sigma_min: float = 0.02, rho: float = 7.0) -> np.ndarray:
    """n + 1 noise levels from sigma_max down to sigma_min (Karras et al. 2022,
    the diffusion model the paper builds on), ending with 0."""
    i = np.arange(n)
    s = (sigma_max ** (1 / rho) + i / max(n - 1, 1) * (sigma_min ** (1 / rho) - sigma_max ** (1 / rho))) ** rho
    return np.concatenate([s, [0.0]])
