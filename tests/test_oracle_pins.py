"""Pins of the FP64 oracle against things other than itself (CPU only).

Each test ties the oracle to a library routine, a closed form, an invariant
or an independent brute force, so that a dropped term, a wrong sign or index,
a transposed operand or a shifted window in ``oracle/gpa_oracle.c`` fails at
least one of them.  STORM-GPA: arXiv 2604.16590, Sec. III-C and Fig. 3(a).
"""
import numpy as np
import pytest
import torch
from scipy.signal import windows as sw

import oracle
from oracle import brute


def _rand(shape, seed, std=1.0):
    rng = np.random.default_rng(seed)
    return [rng.standard_normal(shape) * std for _ in range(4)]


def _sdpa(q, k, v, mask=None, scale=None):
    """torch's fp64 scaled-dot-product attention (library routine)."""
    tq, tk, tv = (torch.from_numpy(np.ascontiguousarray(a)) for a in (q, k, v))
    m = None if mask is None else torch.from_numpy(mask)
    o = torch.nn.functional.scaled_dot_product_attention(tq, tk, tv, attn_mask=m, scale=scale)
    return o.numpy()


# ---------------------------------------------------------------- special cases
@pytest.mark.parametrize("grid,d", [((1, 8, 16), 16), ((2, 4, 8), 8), ((3, 5, 7), 12)])
def test_one_tile_is_exact_global_attention(grid, d):
    """Tiles = 1 is STORM-DiT without GPA (Sec. IV-B): plain global SDPA."""
    T, Y, X = grid
    geo = oracle.Geometry(2, 3, d, T, Y, X, core=grid, halo=(0, 0, 0))
    q, k, v, _ = _rand(geo.shape, 1)
    out = oracle.forward(geo, q, k, v)
    ref = _sdpa(q, k, v)
    np.testing.assert_allclose(out, ref, rtol=0, atol=1e-13)


def test_one_tile_with_halo_clipped_to_grid_is_global_attention():
    """A halo that reaches past the grid is clipped away: still global SDPA."""
    geo = oracle.Geometry(1, 2, 8, 2, 6, 6, core=(2, 6, 6), halo=(1, 3, 2))
    q, k, v, _ = _rand(geo.shape, 2)
    np.testing.assert_allclose(oracle.forward(geo, q, k, v), _sdpa(q, k, v), rtol=0, atol=1e-13)


def test_zero_halo_is_block_diagonal_attention():
    """halo = 0: tiles are processed independently (Sec. III-C, first tiling)."""
    T, Y, X = 2, 8, 12
    core = (1, 4, 5)  # 2 x 2 x 3 tiles, the last x tile short (12 = 5 + 5 + 2)
    geo = oracle.Geometry(1, 2, 8, T, Y, X, core=core, halo=(0, 0, 0))
    q, k, v, _ = _rand(geo.shape, 3)
    t, y, x = np.meshgrid(np.arange(T), np.arange(Y), np.arange(X), indexing="ij")
    tid = ((t // core[0]) * 100 + (y // core[1]) * 10 + (x // core[2])).reshape(-1)
    mask = tid[:, None] == tid[None, :]
    np.testing.assert_allclose(oracle.forward(geo, q, k, v), _sdpa(q, k, v, mask=mask), rtol=0, atol=1e-13)


# ---------------------------------------------------------------- window
@pytest.mark.parametrize("M", [2, 5, 8, 24, 48, 144])
def test_window_is_half_sample_hann(M):
    """The per-dimension window equals the odd samples of a periodic Hann of
    length 2M (scipy), i.e. a Hann sampled at half-integer offsets."""
    ref = sw.hann(2 * M, sym=False)[1::2]
    got = np.array([oracle.window_1d(n, M) for n in range(M)])
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-15)
    assert (got > 0).all()
    np.testing.assert_allclose(got, got[::-1], atol=1e-15)  # symmetric: centre trusted most


def test_two_cover_token_1d_by_hand():
    """1-D, two tiles with a halo: a token in the overlap is the Hann-weighted
    mean of the two tiles' SDPA outputs; single-cover tokens are untouched."""
    X, c, h, d = 16, 8, 2, 6
    geo = oracle.Geometry(1, 1, d, 1, 1, X, core=(1, 1, c), halo=(0, 0, h))
    q, k, v, _ = _rand(geo.shape, 4)
    out = oracle.forward(geo, q, k, v)[0, 0]
    # tile 0 covers [0, 10) (nominal [-2, 10)); tile 1 covers [6, 16) (nominal [6, 18))
    o0 = _sdpa(q[:, :, 0:10], k[:, :, 0:10], v[:, :, 0:10])[0, 0]
    o1 = _sdpa(q[:, :, 6:16], k[:, :, 6:16], v[:, :, 6:16])[0, 0]
    win = sw.hann(2 * (c + 2 * h), sym=False)[1::2]
    for x in range(X):
        if x < 6:
            ref = o0[x]
        elif x >= 10:
            ref = o1[x - 6]
        else:
            w0, w1 = win[x + 2], win[x - 6]
            ref = (w0 * o0[x] + w1 * o1[x - 6]) / (w0 + w1)
        np.testing.assert_allclose(out[x], ref, rtol=0, atol=1e-13, err_msg=f"x={x}")


def test_flat_window_is_plain_mean():
    X, c, h, d = 12, 4, 1, 5
    geo = oracle.Geometry(1, 1, d, 1, 1, X, core=(1, 1, c), halo=(0, 0, h), window="flat")
    q, k, v, _ = _rand(geo.shape, 5)
    out = oracle.forward(geo, q, k, v)[0, 0]
    parts = [(0, 5), (3, 9), (7, 12)]
    outs = [_sdpa(q[:, :, a:b], k[:, :, a:b], v[:, :, a:b])[0, 0] for a, b in parts]
    for x in range(X):
        contrib = [o[x - a] for o, (a, b) in zip(outs, parts) if a <= x < b]
        np.testing.assert_allclose(out[x], np.mean(contrib, axis=0), atol=1e-13)


# ---------------------------------------------------------------- brute force
@pytest.mark.parametrize(
    "grid,core,halo,d,window",
    [
        ((1, 64, 64), (1, 16, 16), (0, 4, 4), 64, "hann"),  # the 4096-token forward workload
        ((5, 6, 7), (2, 3, 3), (1, 1, 2), 8, "hann"),  # every dimension tiled, short last tiles
        ((4, 9, 10), (4, 4, 4), (0, 2, 3), 8, "flat"),
        ((3, 8, 8), (1, 8, 3), (1, 0, 1), 4, "hann"),  # halo wider than half the core in t
    ],
)
def test_oracle_matches_dense_brute_force(grid, core, halo, d, window):
    T, Y, X = grid
    geo = oracle.Geometry(1, 2, d, T, Y, X, core=core, halo=halo, window=window)
    q, k, v, _ = _rand(geo.shape, 6)
    out = oracle.forward(geo, q, k, v)
    ref = brute.forward(T, Y, X, core, halo, q, k, v, window=window)
    err = np.abs(out - ref).max() / np.abs(ref).max()
    assert err < 1e-12, err


# ---------------------------------------------------------------- invariants / closed forms
GEOS = [
    ((2, 12, 16), (1, 4, 8), (1, 2, 3)),
    ((1, 20, 24), (1, 8, 8), (0, 3, 2)),
]


@pytest.mark.parametrize("grid,core,halo", GEOS)
def test_constant_values_return_the_constant(grid, core, halo):
    """Every row of the effective matrix sums to one: V = c gives Out = c."""
    geo = oracle.Geometry(1, 2, 6, *grid, core=core, halo=halo)
    q, k, _, _ = _rand(geo.shape, 7, std=2.0)
    c = np.linspace(-3, 5, geo.d)
    v = np.broadcast_to(c, geo.shape).copy()
    np.testing.assert_allclose(oracle.forward(geo, q, k, v), v, rtol=0, atol=1e-13)


def test_effective_weights_unit_sum_nonnegative_and_local():
    """With d = N and V = identity the output is the effective matrix itself:
    rows sum to 1, entries are >= 0, and A_eff[i, j] is nonzero exactly when
    some extended tile contains both i and j."""
    T, Y, X, core, halo = 1, 4, 8, (1, 2, 4), (0, 1, 1)
    N = T * Y * X
    geo = oracle.Geometry(1, 1, N, T, Y, X, core=core, halo=halo)
    rng = np.random.default_rng(8)
    q = rng.standard_normal(geo.shape)
    k = rng.standard_normal(geo.shape)
    v = np.eye(N)[None, None]
    A = oracle.forward(geo, q, k, v)[0, 0]
    np.testing.assert_allclose(A.sum(axis=1), 1.0, atol=1e-14)
    assert (A >= 0).all()
    # support pattern from the tile definition, enumerated by brute force
    share = np.zeros((N, N), bool)
    ys = [(max(a * core[1] - halo[1], 0), min((a + 1) * core[1] + halo[1], Y)) for a in range(Y // core[1])]
    xs = [(max(a * core[2] - halo[2], 0), min((a + 1) * core[2] + halo[2], X)) for a in range(X // core[2])]
    for y0, y1 in ys:
        for x0, x1 in xs:
            idx = np.array([y * X + x for y in range(y0, y1) for x in range(x0, x1)])
            share[np.ix_(idx, idx)] = True
    assert ((A > 0) == share).all()


@pytest.mark.parametrize("grid,core,halo", GEOS)
def test_linear_in_values_and_key_shift_invariant(grid, core, halo):
    geo = oracle.Geometry(1, 2, 5, *grid, core=core, halo=halo)
    q, k, v1, v2 = _rand(geo.shape, 9)
    f = lambda kk, vv: oracle.forward(geo, q, kk, vv)  # noqa: E731
    np.testing.assert_allclose(f(k, 2.0 * v1 - 3.0 * v2), 2.0 * f(k, v1) - 3.0 * f(k, v2), atol=1e-12)
    # adding one vector to every key shifts each score row by a constant
    shift = np.random.default_rng(10).standard_normal((1, 2, 1, geo.d))
    np.testing.assert_allclose(f(k + shift, v1), f(k, v1), atol=1e-12)


def test_token_permutation_equivariance_for_one_tile():
    grid = (2, 4, 6)
    geo = oracle.Geometry(1, 1, 6, *grid, core=grid, halo=(0, 0, 0))
    q, k, v, _ = _rand(geo.shape, 11)
    perm = np.random.default_rng(12).permutation(geo.N)
    out = oracle.forward(geo, q, k, v)
    outp = oracle.forward(geo, q[:, :, perm], k[:, :, perm], v[:, :, perm])
    np.testing.assert_allclose(outp, out[:, :, perm], atol=1e-13)


def test_swap_inside_single_cover_region_is_equivariant():
    """Swapping two tokens that are covered only by the same tile swaps their
    outputs (the window cancels for single-cover tokens)."""
    geo = oracle.Geometry(1, 1, 4, 1, 16, 16, core=(1, 8, 8), halo=(0, 2, 2))
    q, k, v, _ = _rand(geo.shape, 13)
    a, b = 1 * 16 + 1, 4 * 16 + 3  # both within y,x < 6: tile (0,0) only
    perm = np.arange(geo.N)
    perm[[a, b]] = perm[[b, a]]
    out = oracle.forward(geo, q, k, v)
    outp = oracle.forward(geo, q[:, :, perm], k[:, :, perm], v[:, :, perm])
    np.testing.assert_allclose(outp, out[:, :, perm], atol=1e-13)


def test_locality_one_step_of_propagation():
    """Out(i) depends on exactly the tokens of the tiles that cover i: moving a
    token outside them changes nothing (bitwise); moving one inside does."""
    geo = oracle.Geometry(1, 1, 4, 1, 24, 24, core=(1, 8, 8), halo=(0, 2, 2))
    q, k, v, _ = _rand(geo.shape, 14)
    out = oracle.forward(geo, q, k, v)
    i = 2 * 24 + 2  # tile (0,0) only: its extended box is y,x in [0,10)
    far = 20 * 24 + 20
    near = 9 * 24 + 9
    for j, should_change in ((far, False), (near, True)):
        v2 = v.copy()
        v2[0, 0, j] += 1.0
        o2 = oracle.forward(geo, q, k, v2)
        assert (not np.array_equal(o2[0, 0, i], out[0, 0, i])) == should_change


def test_heads_and_batches_are_independent():
    geo = oracle.Geometry(2, 3, 4, 1, 8, 8, core=(1, 4, 4), halo=(0, 1, 1))
    q, k, v, _ = _rand(geo.shape, 15)
    out = oracle.forward(geo, q, k, v)
    one = oracle.Geometry(1, 1, 4, 1, 8, 8, core=(1, 4, 4), halo=(0, 1, 1))
    for b in range(2):
        for h in range(3):
            sl = (slice(b, b + 1), slice(h, h + 1))
            np.testing.assert_array_equal(oracle.forward(one, q[sl], k[sl], v[sl]), out[sl])


# ---------------------------------------------------------------- backward
def _loss(geo, q, k, v, g):
    return float((oracle.forward(geo, q, k, v) * g).sum())


@pytest.mark.parametrize(
    "grid,core,halo,window",
    [((1, 8, 8), (1, 4, 4), (0, 2, 2), "hann"), ((3, 4, 6), (2, 2, 4), (1, 1, 1), "hann"), ((1, 6, 9), (1, 3, 4), (0, 1, 2), "flat")],
)
def test_backward_matches_central_finite_differences(grid, core, halo, window):
    geo = oracle.Geometry(1, 2, 4, *grid, core=core, halo=halo, window=window)
    q, k, v, g = _rand(geo.shape, 16)
    dq, dk, dv = oracle.backward(geo, q, k, v, g)
    rng = np.random.default_rng(17)
    eps = 1e-6
    for which, grad in ((0, dq), (1, dk), (2, dv)):
        # random directional derivatives
        for _ in range(4):
            dirn = rng.standard_normal(geo.shape)
            args_p = [q, k, v]
            args_m = [q, k, v]
            args_p = [a + eps * dirn if n == which else a for n, a in enumerate(args_p)]
            args_m = [a - eps * dirn if n == which else a for n, a in enumerate(args_m)]
            fd = (_loss(geo, *args_p, g) - _loss(geo, *args_m, g)) / (2 * eps)
            an = float((grad * dirn).sum())
            assert abs(fd - an) <= 1e-7 * max(1.0, abs(an)), (which, fd, an)
        # random single elements
        for _ in range(6):
            idx = tuple(rng.integers(0, s) for s in geo.shape)
            e = np.zeros(geo.shape)
            e[idx] = eps
            args_p = [a + e if n == which else a for n, a in enumerate((q, k, v))]
            args_m = [a - e if n == which else a for n, a in enumerate((q, k, v))]
            fd = (_loss(geo, *args_p, g) - _loss(geo, *args_m, g)) / (2 * eps)
            assert abs(fd - grad[idx]) <= 1e-7 * max(1.0, abs(grad[idx])), (which, idx, fd, grad[idx])


def test_backward_one_tile_matches_torch_autograd():
    grid = (2, 4, 5)
    geo = oracle.Geometry(2, 2, 6, *grid, core=grid, halo=(0, 0, 0))
    q, k, v, g = _rand(geo.shape, 18)
    dq, dk, dv = oracle.backward(geo, q, k, v, g)
    tq, tk, tv = (torch.tensor(a, requires_grad=True) for a in (q, k, v))
    o = torch.nn.functional.scaled_dot_product_attention(tq, tk, tv)
    (o * torch.from_numpy(g)).sum().backward()
    for a, b in ((dq, tq.grad), (dk, tk.grad), (dv, tv.grad)):
        np.testing.assert_allclose(a, b.numpy(), rtol=0, atol=1e-12)


# ---------------------------------------------------------------- sampled-row entry points
def test_sampled_rows_agree_with_full_oracle():
    geo = oracle.Geometry(2, 2, 8, 2, 10, 12, core=(1, 4, 6), halo=(1, 2, 2))
    q, k, v, g = _rand(geo.shape, 19)
    out = oracle.forward(geo, q, k, v)
    dq, dk, dv = oracle.backward(geo, q, k, v, g)
    rng = np.random.default_rng(20)
    rows = np.stack([rng.integers(0, 2, 12), rng.integers(0, 2, 12), rng.integers(0, geo.N, 12)], 1)
    o_r, dq_r = oracle.forward_rows(geo, q, k, v, rows, dout=g)
    dk_r, dv_r = oracle.key_rows(geo, q, k, v, g, rows)
    for n, (b, h, i) in enumerate(rows):
        np.testing.assert_allclose(o_r[n], out[b, h, i], atol=1e-13)
        np.testing.assert_allclose(dq_r[n], dq[b, h, i], atol=1e-13)
        np.testing.assert_allclose(dk_r[n], dk[b, h, i], atol=1e-13)
        np.testing.assert_allclose(dv_r[n], dv[b, h, i], atol=1e-13)


def test_tile_lse_is_the_tile_softmax_normaliser():
    """brute.tile_lse against torch's logsumexp (library): over the whole grid
    when one tile covers it, and over a tile's token set built by hand when the
    grid is cut into 2 x 2 cores without halo."""
    import torch

    from oracle import brute

    rng = np.random.default_rng(5)
    T, Y, X, d = 2, 8, 12, 16
    q2 = rng.standard_normal((T * Y * X, d))
    k2 = rng.standard_normal((T * Y * X, d))
    s = 0.3
    rows = [0, 17, 100, T * Y * X - 1]
    got = brute.tile_lse(T, Y, X, (T, Y, X), (0, 0, 0), q2, k2, s, (0, 0, 0), rows)
    ref = torch.logsumexp(s * torch.from_numpy(q2[rows]) @ torch.from_numpy(k2).T, dim=1).numpy()
    assert np.allclose(got, ref, rtol=0, atol=1e-12)
    # tile (1, 0, 1) of cores (1, 4, 6): frame 1, rows 0..3, columns 6..11
    idx = np.array([(1 * Y + y) * X + x for y in range(4) for x in range(6, 12)])
    rows = [int(idx[0]), int(idx[7]), int(idx[-1])]
    got = brute.tile_lse(T, Y, X, (1, 4, 6), (0, 0, 0), q2, k2, s, (1, 0, 1), rows)
    ref = torch.logsumexp(s * torch.from_numpy(q2[rows]) @ torch.from_numpy(k2[idx]).T, dim=1).numpy()
    assert np.allclose(got, ref, rtol=0, atol=1e-12)
