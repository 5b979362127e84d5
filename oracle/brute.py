"""Dense brute force of STORM-GPA (arXiv 2604.16590, Sec. III-C), FP64 numpy.

TEST INFRASTRUCTURE ONLY (same rule as the rest of ``oracle/``).

Independent of ``gpa_oracle.c``: it builds the N x N effective attention
matrix

    A_eff[i, j] = sum_t w_t(i) P^t[i, j] [i, j in E_t] / sum_t w_t(i)

explicitly (vectorised numpy, its own tile enumeration, and the Hann window
taken from ``scipy.signal.windows.hann`` rather than a hand-typed formula),
then Out = A_eff @ V.  Only for small N (the matrix is N^2 doubles).
"""
from __future__ import annotations

import itertools

import numpy as np
from scipy.signal import windows as _win


def _dim_tiles(G: int, c: int, h: int):
    """Per dimension: list of (nominal_start, clipped_lo, clipped_hi)."""
    n = -(-G // c)
    out = []
    for k in range(n):
        a, b = k * c - h, (k + 1) * c + h
        out.append((a, max(a, 0), min(b, G)))
    return out


def _dim_window(G: int, c: int, h: int, window: str) -> np.ndarray | None:
    """Window samples over the nominal extent, or None for weight 1."""
    n = -(-G // c)
    if window == "flat" or (n == 1 and h == 0):
        return None
    M = c + 2 * h
    # half-sample-offset Hann of length M = odd samples of a periodic Hann of length 2M
    return _win.hann(2 * M, sym=False)[1::2]


def effective_matrix(T, Y, X, core, halo, q2, k2, scale, window="hann") -> np.ndarray:
    """A_eff for one (batch, head): q2, k2 are [N, d]."""
    N = T * Y * X
    grid = np.arange(N).reshape(T, Y, X)
    dims = [(T, core[0], halo[0]), (Y, core[1], halo[1]), (X, core[2], halo[2])]
    per_dim = [_dim_tiles(*dm) for dm in dims]
    wins = [_dim_window(*dm, window) for dm in dims]
    num = np.zeros((N, N))
    den = np.zeros(N)
    for combo in itertools.product(*per_dim):
        sl = tuple(slice(lo, hi) for (_, lo, hi) in combo)
        idx = grid[sl].reshape(-1)
        # separable weight of this tile at each of its tokens
        w = np.ones(grid[sl].shape)
        for a, (nom, lo, hi) in enumerate(combo):
            if wins[a] is None:
                continue
            wa = wins[a][lo - nom : hi - nom]
            shape = [1, 1, 1]
            shape[a] = -1
            w = w * wa.reshape(shape)
        w = w.reshape(-1)
        s = scale * (q2[idx] @ k2[idx].T)
        s -= s.max(axis=1, keepdims=True)
        p = np.exp(s)
        p /= p.sum(axis=1, keepdims=True)
        num[np.ix_(idx, idx)] += w[:, None] * p
        den[idx] += w
    return num / den[:, None]


def forward(T, Y, X, core, halo, q, k, v, scale=None, window="hann") -> np.ndarray:
    """Out for [B, nh, N, d] inputs via the dense effective matrix."""
    q = np.asarray(q, dtype=np.float64)
    k = np.asarray(k, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    d = q.shape[-1]
    scale = 1.0 / np.sqrt(d) if scale is None else scale
    out = np.empty_like(v)
    for b in range(q.shape[0]):
        for h in range(q.shape[1]):
            A = effective_matrix(T, Y, X, core, halo, q[b, h], k[b, h], scale, window)
            out[b, h] = A @ v[b, h]
    return out


def tile_lse(T, Y, X, core, halo, q2, k2, scale, tile, rows) -> np.ndarray:
    """log sum_{j in E_t} exp(scale q_i . k_j) for query rows i of one extended
    tile (the softmax normaliser of Sec. III-C's per-tile attention), FP64.
    tile: per-dimension tile indices (k_t, k_y, k_x); rows: global token
    indices inside that extended tile; q2, k2: [N, d] of one (batch, head)."""
    grid = np.arange(T * Y * X).reshape(T, Y, X)
    dims = [(T, core[0], halo[0]), (Y, core[1], halo[1]), (X, core[2], halo[2])]
    sl = []
    for a, (G, c, h) in enumerate(dims):
        _, lo, hi = _dim_tiles(G, c, h)[tile[a]]
        sl.append(slice(lo, hi))
    idx = grid[tuple(sl)].reshape(-1)
    assert set(int(i) for i in rows) <= set(int(i) for i in idx)
    kk = np.asarray(k2, dtype=np.float64)[idx]
    out = np.empty(len(rows))
    for r, i in enumerate(rows):
        s = scale * (kk @ np.asarray(q2[i], dtype=np.float64))
        m = s.max()
        out[r] = m + np.log(np.exp(s - m).sum())
    return out
