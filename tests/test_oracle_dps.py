"""Pins of the posterior-sampling step oracle (``oracle/dps.py``), arXiv
2604.16590, Sec. III-A (reverse SDE, score decomposition, DPS likelihood score,
Eq. denoise) and Sec. III-C (context propagation across tiles per step).

Pinned against torch (SDPA and autograd for the untiled step), central finite
differences of the observation misfit, and the tile-locality the paper's
propagation argument rests on.
"""
import numpy as np
import torch

import oracle
from oracle import dps
from paper_2604_16590_gb300 import gattn


def _setup(geo, seed, frac=0.3):
    rng = np.random.default_rng(seed)
    z = rng.standard_normal(geo.shape)
    y = rng.standard_normal(geo.shape)
    eps = rng.standard_normal(geo.shape)
    mask = (rng.random((geo.B, geo.N)) < frac).astype(np.float64)
    return z, y, eps, mask


def test_untiled_step_matches_torch_autograd():
    """Tiles = 1: D = SDPA(z, z, z); the likelihood term is autograd of
    0.5 * ||mask * (D(z) - y)||^2."""
    geo = oracle.Geometry(1, 2, 8, 1, 6, 8, core=(1, 6, 8), halo=(0, 0, 0))
    z, y, eps, mask = _setup(geo, 1)
    sigma, sigma_next, lam = 1.3, 0.9, 0.7
    got, D = dps.step(geo, z, y, mask, eps, sigma, sigma_next, lam)
    tz = torch.from_numpy(z).requires_grad_()
    tD = torch.nn.functional.scaled_dot_product_attention(tz, tz, tz)
    m = torch.from_numpy(mask)[:, None, :, None]
    (0.5 * (m * (tD - torch.from_numpy(y))) ** 2).sum().backward()
    delta = sigma**2 - sigma_next**2
    ref = z + delta * ((tD.detach().numpy() - z) / sigma**2 - lam * tz.grad.numpy()) + np.sqrt(delta) * eps
    np.testing.assert_allclose(D, tD.detach().numpy(), rtol=0, atol=1e-13)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12)


def test_likelihood_term_matches_finite_differences():
    geo = oracle.Geometry(1, 1, 4, 1, 4, 6, core=(1, 2, 3), halo=(0, 1, 1))
    z, y, eps, mask = _setup(geo, 2, frac=0.5)
    sigma, sigma_next = 1.0, 0.5
    base, _ = dps.step(geo, z, y, mask, eps, sigma, sigma_next, 0.0)
    with_lik, _ = dps.step(geo, z, y, mask, eps, sigma, sigma_next, 1.0)
    delta = sigma**2 - sigma_next**2
    grad = (base - with_lik) / delta  # = J^T mask (D - y)

    def misfit(zz):
        D = oracle.forward(geo, zz, zz, zz)
        return 0.5 * float(((mask[:, None, :, None] * (D - y)) ** 2).sum())

    h = 1e-6
    flat, gflat = z.reshape(-1), grad.reshape(-1)
    for i in range(0, flat.size, 7):
        old = flat[i]
        flat[i] = old + h
        fp = misfit(z)
        flat[i] = old - h
        fm = misfit(z)
        flat[i] = old
        assert abs((fp - fm) / (2 * h) - gflat[i]) < 1e-6, (i, (fp - fm) / (2 * h), gflat[i])


def test_no_step_when_sigma_does_not_move():
    geo = oracle.Geometry(1, 1, 4, 1, 4, 4, core=(1, 2, 2), halo=(0, 1, 1))
    z, y, eps, mask = _setup(geo, 3)
    got, _ = dps.step(geo, z, y, mask, eps, 0.8, 0.8, 2.0)
    np.testing.assert_array_equal(got, z)


def test_observations_reach_only_neighbouring_tiles_in_one_step():
    """Sec. III-C: per step, context moves from a tile to its neighbours only.
    Observations inside the first tile's core change the step's result only
    within one tile distance (halo 2, core 4 along x)."""
    geo = oracle.Geometry(1, 1, 4, 1, 1, 32, core=(1, 1, 4), halo=(0, 0, 2))
    rng = np.random.default_rng(4)
    z = rng.standard_normal(geo.shape)
    eps = rng.standard_normal(geo.shape)
    y = rng.standard_normal(geo.shape)
    mask = np.zeros((1, 32))
    mask[0, :4] = 1.0
    with_obs, _ = dps.step(geo, z, y, mask, eps, 1.0, 0.7, 1.0)
    without, _ = dps.step(geo, z, y, np.zeros_like(mask), eps, 1.0, 0.7, 1.0)
    diff = np.abs(with_obs - without).max(axis=(0, 1, 3))
    # tile 0 core [0, 4) + halo reaches token 5; tokens feeding those rows are in tiles 0 and 1
    assert diff[:4].max() > 1e-3
    assert diff[12:].max() == 0.0


def test_sigma_schedule_is_decreasing_and_ends_at_zero():
    s = dps.sigma_schedule(20)
    assert s.shape == (21,) and s[-1] == 0.0
    assert np.all(np.diff(s) < 0)
    np.testing.assert_allclose([s[0], s[-2]], [2.0, 0.02], rtol=1e-12)


def test_bf16_attention_reading_rounds_the_state():
    geo = oracle.Geometry(1, 1, 8, 1, 4, 4, core=(1, 4, 4), halo=(0, 0, 0))
    z, y, eps, mask = _setup(geo, 5)
    a, _ = dps.step(geo, z, y, mask, eps, 1.0, 0.6, 0.5, attn_dtype="bf16")
    zb = dps.bf16_round(z)
    b, _ = dps.step(geo, zb, y, mask, eps, 1.0, 0.6, 0.5)
    # same attention input; the prior score subtracts the FP64 state
    delta = 1.0 - 0.36
    assert np.abs(a - b - (z - zb) * (1 - delta)).max() < 5e-3


def test_sigma_schedule_roots_are_equally_spaced():
    """The schedule of Karras et al. (2022) interpolates sigma^(1/rho) linearly
    between the end points: the rho-th roots of the levels are an arithmetic
    sequence (a wrong exponent or spacing breaks it), for the oracle and for
    the library's host-side schedule alike."""
    for n, smax, smin, rho in ((20, 2.0, 0.05, 7.0), (7, 80.0, 0.002, 7.0), (12, 1.0, 0.1, 3.0)):
        for s in (dps.sigma_schedule(n, smax, smin, rho), np.array(gattn.sigma_schedule(n, smax, smin, rho))):
            r = s[:-1] ** (1.0 / rho)
            np.testing.assert_allclose(np.diff(r), (smin ** (1 / rho) - smax ** (1 / rho)) / (n - 1), rtol=1e-9)
            np.testing.assert_allclose([s[0], s[-2], s[-1]], [smax, smin, 0.0], rtol=1e-12)


def test_step_to_zero_noise_lands_on_the_denoiser_output():
    """Without noise and guidance, the Euler step from sigma to 0 moves the
    state by sigma^2 times the prior score (D(z) - z) / sigma^2: it lands on
    the denoiser's output D(z) itself (Tweedie's estimate), whatever sigma."""
    geo = oracle.Geometry(1, 2, 8, 1, 6, 8, core=(1, 3, 4), halo=(0, 1, 1))
    z, y, eps, mask = _setup(geo, 8)
    for sigma in (0.3, 1.0, 2.5):
        got, D = dps.step(geo, z, y, mask, np.zeros_like(eps), sigma, 0.0, 0.0)
        np.testing.assert_allclose(got, D, rtol=0, atol=1e-12)


def test_noise_of_a_step_has_the_variance_sigma_drop():
    """A state whose tokens are all equal is a fixed point of the denoiser
    (constant values are returned), so the prior score vanishes and, without
    guidance, the step adds exactly sqrt(sigma^2 - sigma_next^2) eps: the
    variance the noise level drops by (a noise term scaled by delta instead of
    its square root fails)."""
    geo = oracle.Geometry(1, 1, 4, 1, 4, 6, core=(1, 2, 3), halo=(0, 1, 1))
    _, y, eps, mask = _setup(geo, 9)
    z = np.broadcast_to(np.array([0.3, -1.2, 0.7, 2.0]), (1, 1, 24, 4)).copy()
    sigma, sigma_next = 1.5, 0.4
    got, D = dps.step(geo, z, y, mask, eps, sigma, sigma_next, 0.0)
    np.testing.assert_allclose(D, z, rtol=0, atol=1e-13)
    np.testing.assert_allclose(got - z, np.sqrt(sigma**2 - sigma_next**2) * eps, rtol=0, atol=1e-12)
