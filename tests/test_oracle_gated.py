"""Pins of the noise-gated self + cross attention oracle (``oracle/gated.py``),
arXiv 2604.16590, Sec. III-B: a library routine for the untiled case, and the
invariants of the blend."""
import numpy as np
import torch

import oracle
from oracle import gated


def _rand(shape, seed, n=5):
    rng = np.random.default_rng(seed)
    return [rng.standard_normal(shape) for _ in range(n)]


def test_untiled_is_a_blend_of_two_sdpa_calls():
    """Tiles = 1: self = SDPA(q, k, v), cross = SDPA(q, kc, vc) (torch FP64)."""
    geo = oracle.Geometry(1, 3, 8, 1, 6, 8, core=(1, 6, 8), halo=(0, 0, 0))
    q, k, v, kc, vc = _rand(geo.shape, 1)
    gate = np.array([0.0, 0.35, 1.0])
    t = [torch.from_numpy(a) for a in (q, k, v, kc, vc)]
    sdpa = torch.nn.functional.scaled_dot_product_attention
    ref_s, ref_c = sdpa(t[0], t[1], t[2]).numpy(), sdpa(t[0], t[3], t[4]).numpy()
    g = gate.reshape(1, -1, 1, 1)
    np.testing.assert_allclose(gated.forward(geo, q, k, v, kc, vc, gate), g * ref_s + (1 - g) * ref_c,
                               rtol=0, atol=1e-13)


def test_same_kv_source_is_plain_gpa_for_any_gate():
    geo = oracle.Geometry(1, 2, 8, 2, 8, 12, core=(1, 4, 5), halo=(1, 2, 2))
    q, k, v, _, _ = _rand(geo.shape, 2)
    ref = oracle.forward(geo, q, k, v)
    for g in ([0.0, 1.0], [0.2, 0.9]):
        np.testing.assert_allclose(gated.forward(geo, q, k, v, k, v, g), ref, rtol=0, atol=1e-13)


def test_gate_one_ignores_the_temporal_branch_and_zero_the_spatial_one():
    geo = oracle.Geometry(1, 2, 8, 1, 8, 12, core=(1, 4, 4), halo=(0, 2, 2))
    q, k, v, kc, vc = _rand(geo.shape, 3)
    a = gated.forward(geo, q, k, v, kc, vc, [1.0, 0.0])
    b = gated.forward(geo, q, k, v, kc + 1.0, vc * 2.0, [1.0, 0.0])
    np.testing.assert_array_equal(a[:, 0], b[:, 0])
    c = gated.forward(geo, q, k - 0.5, v * 3.0, kc, vc, [1.0, 0.0])
    np.testing.assert_array_equal(a[:, 1], c[:, 1])


def test_blend_is_affine_in_the_gate():
    geo = oracle.Geometry(1, 1, 8, 1, 8, 8, core=(1, 4, 4), halo=(0, 2, 2))
    q, k, v, kc, vc = _rand(geo.shape, 4)
    o0 = gated.forward(geo, q, k, v, kc, vc, [0.0])
    o1 = gated.forward(geo, q, k, v, kc, vc, [1.0])
    o3 = gated.forward(geo, q, k, v, kc, vc, [0.3])
    np.testing.assert_allclose(o3, o0 + 0.3 * (o1 - o0), rtol=0, atol=1e-13)
