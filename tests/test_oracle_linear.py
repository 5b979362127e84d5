"""Pins of the factorised linear attention oracle (``oracle/linear.py``):
O(N^2) brute force with explicit weights, the feature map against torch's elu,
the normalised closed forms and the permutation symmetries of the operator."""
import numpy as np
import pytest
import torch

from oracle import linear as ol


def _qkv(shape, seed):
    rng = np.random.default_rng(seed)
    return [rng.standard_normal(shape) for _ in range(3)]


def test_feature_map_is_elu_plus_one():
    x = np.linspace(-30, 30, 1001)
    ref = torch.nn.functional.elu(torch.from_numpy(x)).numpy() + 1.0
    # elu(x) + 1 = expm1(x) + 1 loses the relative precision of tiny values: absolute check
    np.testing.assert_allclose(ol.phi(x), ref, rtol=1e-14, atol=1e-15)
    assert (ol.phi(x) > 0).all()


@pytest.mark.parametrize("shape", [(1, 1, 64, 8), (2, 3, 100, 16), (1, 2, 257, 64)])
def test_factorised_equals_quadratic_brute_force(shape):
    q, k, v = _qkv(shape, sum(shape))
    np.testing.assert_allclose(ol.forward(q, k, v), ol.brute(q, k, v), rtol=1e-12, atol=1e-12)


def test_effective_weights_sum_to_one_and_are_positive():
    q, k, _ = _qkv((1, 2, 50, 8), 1)
    d = 50
    v = np.broadcast_to(np.eye(d)[None, None], (1, 2, d, d))  # out = the weight matrix when d = N
    k = np.ascontiguousarray(k[..., :8])
    w = ol.forward(q[..., :8], k, np.ascontiguousarray(v))
    np.testing.assert_allclose(w.sum(axis=-1), 1.0, rtol=0, atol=1e-13)
    assert (w > 0).all()


def test_constant_values_are_returned():
    q, k, v = _qkv((1, 2, 80, 16), 2)
    v[:] = v[:, :, :1]
    np.testing.assert_allclose(ol.forward(q, k, v), v, rtol=0, atol=1e-13)


def test_token_permutation_equivariance():
    q, k, v = _qkv((1, 1, 40, 8), 3)
    p = np.random.default_rng(4).permutation(40)
    a = ol.forward(q, k, v)
    b = ol.forward(q[:, :, p], k, v)  # permuting queries permutes outputs
    np.testing.assert_allclose(b, a[:, :, p], rtol=0, atol=1e-13)
    c = ol.forward(q, k[:, :, p], v[:, :, p])  # permuting key/value pairs changes nothing
    np.testing.assert_allclose(c, a, rtol=0, atol=1e-13)


def test_summary_is_additive_over_token_splits():
    """The split-N reduction the GPU performs: partial summaries add up."""
    _, k, v = _qkv((1, 2, 90, 8), 5)
    S, z = ol.summary(k, v)
    S1, z1 = ol.summary(k[:, :, :37], v[:, :, :37])
    S2, z2 = ol.summary(k[:, :, 37:], v[:, :, 37:])
    np.testing.assert_allclose(S, S1 + S2, rtol=1e-13, atol=1e-12)
    np.testing.assert_allclose(z, z1 + z2, rtol=1e-13, atol=1e-12)


def test_forward_rows_matches_forward():
    q, k, v = _qkv((2, 2, 30, 8), 6)
    out = ol.forward(q, k, v)
    rows = [(0, 0, 0), (1, 1, 29), (0, 1, 7)]
    got = ol.forward_rows(q, k, v, rows)
    for i, (b, h, n) in enumerate(rows):
        np.testing.assert_allclose(got[i], out[b, h, n], rtol=0, atol=1e-14)


def test_backward_matches_torch_autograd_of_the_quadratic_form():
    """Autograd through the O(N^2) form with torch's elu: an independent route."""
    q, k, v = _qkv((2, 2, 40, 8), 7)
    g = np.random.default_rng(8).standard_normal(q.shape)
    dq, dk, dv = ol.backward(q, k, v, g)
    tq, tk, tv = (torch.from_numpy(a).requires_grad_() for a in (q, k, v))
    fq = torch.nn.functional.elu(tq) + 1
    fk = torch.nn.functional.elu(tk) + 1
    w = torch.einsum("bhid,bhjd->bhij", fq, fk)
    out = torch.einsum("bhij,bhjd->bhid", w, tv) / w.sum(-1, keepdim=True)
    (out * torch.from_numpy(g)).sum().backward()
    np.testing.assert_allclose(dq, tq.grad.numpy(), rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(dk, tk.grad.numpy(), rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(dv, tv.grad.numpy(), rtol=1e-10, atol=1e-12)


def test_backward_matches_finite_differences():
    q, k, v = _qkv((1, 1, 12, 4), 9)
    g = np.random.default_rng(10).standard_normal(q.shape)
    grads = ol.backward(q, k, v, g)
    h = 1e-6
    for arr, grad in zip((q, k, v), grads):
        flat, gf = arr.reshape(-1), grad.reshape(-1)
        for i in range(0, flat.size, 5):
            old = flat[i]
            flat[i] = old + h
            lp = float((ol.forward(q, k, v) * g).sum())
            flat[i] = old - h
            lm = float((ol.forward(q, k, v) * g).sum())
            flat[i] = old
            assert abs((lp - lm) / (2 * h) - gf[i]) < 1e-7
