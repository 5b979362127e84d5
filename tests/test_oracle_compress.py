"""Pins of the FP64 temporal-compression oracle (``oracle/compress.py``)
against things other than itself (CPU only).

Temporal compression: a learned query per head attends over the S history
frames of each spatial location and returns one token (arXiv 2604.16590,
Sec. III-B, STORM-DiT architecture).  Each test ties the oracle to a library
routine (torch SDPA and autograd), a closed form, an invariant or finite
differences, so that a dropped term, a wrong sign, a wrong reduction axis or a
transposed operand fails at least one of them.
"""
import numpy as np
import pytest
import torch
from scipy.special import expit, logsumexp

from oracle import compress as oc


def _inputs(B, nh, S, M, d, seed, std=1.0):
    rng = np.random.default_rng(seed)
    q = rng.standard_normal((nh, d)) * std
    k = rng.standard_normal((B, nh, S, M, d)) * std
    v = rng.standard_normal((B, nh, S, M, d))
    return q, k, v


def _sdpa_pool(q, k, v, scale):
    """torch fp64 SDPA with one query per (b, h, m) over that location's S keys."""
    B, nh, S, M, d = k.shape
    tq = torch.from_numpy(q)[None, :, None, None, :].expand(B, nh, M, 1, d)
    tk = torch.from_numpy(k).permute(0, 1, 3, 2, 4)  # [B, nh, M, S, d]
    tv = torch.from_numpy(v).permute(0, 1, 3, 2, 4)
    o = torch.nn.functional.scaled_dot_product_attention(tq, tk, tv, scale=scale)
    return o[:, :, :, 0, :].numpy()


@pytest.mark.parametrize("shape", [(1, 1, 5, 3, 8), (2, 3, 17, 4, 16), (1, 2, 64, 7, 32)])
def test_matches_torch_sdpa_with_one_query_per_location(shape):
    B, nh, S, M, d = shape
    q, k, v = _inputs(B, nh, S, M, d, seed=sum(shape))
    scale = 1.0 / np.sqrt(d)
    out, lse = oc.forward(q, k, v)
    np.testing.assert_allclose(out, _sdpa_pool(q, k, v, scale), rtol=0, atol=1e-13)
    s = scale * np.einsum("hd,bhtmd->bhmt", q, k)
    np.testing.assert_allclose(lse, logsumexp(s, axis=-1), rtol=1e-14, atol=1e-13)


def test_single_frame_returns_its_value():
    q, k, v = _inputs(2, 2, 1, 5, 8, seed=3)
    out, lse = oc.forward(q, k, v, scale=0.7)
    np.testing.assert_allclose(out, v[:, :, 0], rtol=0, atol=1e-15)
    np.testing.assert_allclose(lse, 0.7 * np.einsum("hd,bhmd->bhm", q, k[:, :, 0]), rtol=1e-14, atol=1e-14)


def test_constant_values_are_returned():
    q, k, v = _inputs(1, 3, 33, 4, 16, seed=4)
    v[:] = v[:, :, :1]  # the same value in every frame of a location
    out, _ = oc.forward(q, k, v)
    np.testing.assert_allclose(out, v[:, :, 0], rtol=0, atol=1e-13)


def test_zero_query_is_the_frame_mean():
    _, k, v = _inputs(2, 2, 40, 3, 8, seed=5)
    q = np.zeros((2, 8))
    out, lse = oc.forward(q, k, v)
    np.testing.assert_allclose(out, v.mean(axis=2), rtol=0, atol=1e-14)
    np.testing.assert_allclose(lse, np.full(lse.shape, np.log(40.0)), rtol=1e-15, atol=0)


def test_two_frames_closed_form():
    q, k, v = _inputs(1, 2, 2, 6, 8, seed=6)
    scale = 0.3
    out, _ = oc.forward(q, k, v, scale)
    s = scale * np.einsum("hd,bhtmd->bhtm", q, k)
    w0 = expit(s[:, :, 0] - s[:, :, 1])[..., None]
    np.testing.assert_allclose(out, w0 * v[:, :, 0] + (1 - w0) * v[:, :, 1], rtol=0, atol=1e-14)


def test_frame_permutation_invariance():
    q, k, v = _inputs(1, 2, 25, 3, 8, seed=7)
    perm = np.random.default_rng(8).permutation(25)
    a, la = oc.forward(q, k, v)
    b, lb = oc.forward(q, k[:, :, perm], v[:, :, perm])
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-14)
    np.testing.assert_allclose(la, lb, rtol=1e-15, atol=1e-14)


def test_score_shift_invariance():
    """Adding c * q / |q|^2 to every key of a location shifts all its scores by
    scale * c: out is unchanged, lse moves by scale * c."""
    q, k, v = _inputs(1, 1, 9, 4, 8, seed=9)
    c = np.array([0.5, -2.0, 3.0, 10.0])
    k2 = k + (c[None, None, None, :, None] * q[0] / (q[0] @ q[0]))
    a, la = oc.forward(q, k, v, 0.25)
    b, lb = oc.forward(q, k2, v, 0.25)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-13)
    np.testing.assert_allclose(lb - la, np.broadcast_to(0.25 * c, la.shape), rtol=0, atol=1e-13)


def test_distinct_locations_are_independent():
    """Changing the history of one location leaves every other output alone."""
    q, k, v = _inputs(1, 2, 8, 5, 8, seed=10)
    a, _ = oc.forward(q, k, v)
    k2, v2 = k.copy(), v.copy()
    k2[:, :, :, 2] += 1.0
    v2[:, :, :, 2] -= 3.0
    b, _ = oc.forward(q, k2, v2)
    keep = [0, 1, 3, 4]
    np.testing.assert_array_equal(a[:, :, keep], b[:, :, keep])
    assert np.abs(a[:, :, 2] - b[:, :, 2]).max() > 1e-3


def test_forward_locations_matches_forward():
    q, k, v = _inputs(2, 3, 11, 6, 8, seed=11)
    out, lse = oc.forward(q, k, v)
    locs = [(0, 0, 0), (1, 2, 5), (0, 1, 3), (1, 0, 2)]
    o2, l2 = oc.forward_locations(q, k, v, locs)
    for i, (b, h, m) in enumerate(locs):
        np.testing.assert_allclose(o2[i], out[b, h, m], rtol=0, atol=1e-14)
        np.testing.assert_allclose(l2[i], lse[b, h, m], rtol=1e-15, atol=1e-14)


def test_backward_matches_torch_autograd():
    B, nh, S, M, d = 2, 2, 7, 3, 8
    q, k, v = _inputs(B, nh, S, M, d, seed=12)
    g = np.random.default_rng(13).standard_normal((B, nh, M, d))
    scale = 0.4
    dq, dk, dv = oc.backward(q, k, v, g, scale)
    tq = torch.from_numpy(q).requires_grad_()
    tk = torch.from_numpy(k).requires_grad_()
    tv = torch.from_numpy(v).requires_grad_()
    o = torch.nn.functional.scaled_dot_product_attention(
        tq[None, :, None, None, :].expand(B, nh, M, 1, d), tk.permute(0, 1, 3, 2, 4), tv.permute(0, 1, 3, 2, 4),
        scale=scale)[:, :, :, 0, :]
    (o * torch.from_numpy(g)).sum().backward()
    np.testing.assert_allclose(dq, tq.grad.numpy(), rtol=0, atol=1e-12)
    np.testing.assert_allclose(dk, tk.grad.numpy(), rtol=0, atol=1e-12)
    np.testing.assert_allclose(dv, tv.grad.numpy(), rtol=0, atol=1e-12)


def test_backward_matches_finite_differences():
    B, nh, S, M, d = 1, 1, 4, 2, 4
    q, k, v = _inputs(B, nh, S, M, d, seed=14)
    g = np.random.default_rng(15).standard_normal((B, nh, M, d))
    dq, dk, dv = oc.backward(q, k, v, g)

    def loss(q_, k_, v_):
        return float((oc.forward(q_, k_, v_)[0] * g).sum())

    h = 1e-6
    for arr, grad in ((q, dq), (k, dk), (v, dv)):
        flat = arr.reshape(-1)
        gflat = grad.reshape(-1)
        for i in range(0, flat.size, max(1, flat.size // 12)):
            old = flat[i]
            flat[i] = old + h
            lp = loss(q, k, v)
            flat[i] = old - h
            lm = loss(q, k, v)
            flat[i] = old
            assert abs((lp - lm) / (2 * h) - gflat[i]) < 1e-7, (i, (lp - lm) / (2 * h), gflat[i])
