"""FP64 CPU oracle of STORM-DiT's temporal compression (arXiv 2604.16590,
Sec. III-B, the STORM-DiT architecture paragraph and Fig. 2(b)).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this module.  The CUDA library
never imports or calls it, and it imports nothing of the library.

The operation.  History states are folded into one global temporal
representation by cross-attention across the temporal dimension: at every
spatial location m, a learned query per head attends over the S history
frames of that location and returns one token (the same primitive serves the
aggregation across the variable dimension, with S = the number of variables).
With a learned query q_h in R^d per head and history keys/values
k, v of shape [B, nh, S, M, d]:

    s[b,h,t,m]  = scale * q_h . k[b,h,t,m]
    out[b,h,m]  = sum_t softmax_t(s[b,h,:,m]) v[b,h,t,m]
    lse[b,h,m]  = log sum_t exp(s[b,h,t,m])

and, for a loss L with upstream gradient g = dL/dout,

    P[t]        = exp(s[t] - lse)
    dv[t]       = P[t] g
    ds[t]       = P[t] (g . v[t] - g . out)
    dk[t]       = scale * ds[t] q_h
    dq_h        = scale * sum_{b, m, t} ds[b,h,t,m] k[b,h,t,m]

The cost is linear in S: each history token is read once per pass.
Plain numpy in float64, the steps in the order above (no blocking or
reordering): a reader can check it against the definition by eye.
"""
from __future__ import annotations

import numpy as np


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def scores(q, k, scale: float) -> np.ndarray:
    """s[b,h,t,m] = scale * q_h . k[b,h,t,m]; q [nh, d], k [B, nh, S, M, d]."""
    q, k = _f64(q), _f64(k)
    assert q.ndim == 2 and k.ndim == 5 and q.shape == (k.shape[1], k.shape[4]), (q.shape, k.shape)
    return scale * np.einsum("hd,bhtmd->bhtm", q, k)


def forward(q, k, v, scale: float | None = None):
    """(out [B, nh, M, d], lse [B, nh, M]) in float64."""
    k, v = _f64(k), _f64(v)
    assert k.shape == v.shape, (k.shape, v.shape)
    if scale is None:
        scale = 1.0 / np.sqrt(k.shape[4])
    s = scores(q, k, scale)
    smax = s.max(axis=2, keepdims=True)
    e = np.exp(s - smax)
    den = e.sum(axis=2)
    out = np.einsum("bhtm,bhtmd->bhmd", e, v) / den[..., None]
    lse = np.log(den) + smax[:, :, 0, :]
    return out, lse


def backward(q, k, v, g, scale: float | None = None):
    """(dq [nh, d], dk, dv [B, nh, S, M, d]) of the loss sum(out * g), float64."""
    q, k, v, g = _f64(q), _f64(k), _f64(v), _f64(g)
    if scale is None:
        scale = 1.0 / np.sqrt(k.shape[4])
    out, lse = forward(q, k, v, scale)
    s = scores(q, k, scale)
    P = np.exp(s - lse[:, :, None, :])
    dv = P[..., None] * g[:, :, None, :, :]
    gv = np.einsum("bhmd,bhtmd->bhtm", g, v)
    go = np.einsum("bhmd,bhmd->bhm", g, out)
    ds = P * (gv - go[:, :, None, :])
    dk = scale * ds[..., None] * q[None, :, None, None, :]
    dq = scale * np.einsum("bhtm,bhtmd->hd", ds, k)
    return dq, dk, dv


def forward_locations(q, k, v, locs, scale: float | None = None):
    """out and lse at sampled (b, h, m) locations only: [n, d], [n].

    Reads only the S history tokens of each sampled location, so that full-size
    inputs can be checked on a sample."""
    locs = np.asarray(locs, dtype=np.int64).reshape(-1, 3)
    d = k.shape[4]
    if scale is None:
        scale = 1.0 / np.sqrt(d)
    out = np.empty((locs.shape[0], d))
    lse = np.empty(locs.shape[0])
    for i, (b, h, m) in enumerate(locs):
        kk = _f64(k[b, h, :, m, :])  # [S, d]
        vv = _f64(v[b, h, :, m, :])
        s = scale * (kk @ _f64(q[h]))
        smax = s.max()
        e = np.exp(s - smax)
        den = e.sum()
        out[i] = (e @ vv) / den
        lse[i] = np.log(den) + smax
    return out, lse
