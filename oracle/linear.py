"""FP64 CPU oracle of factorised (kernelised) linear attention.

TEST INFRASTRUCTURE ONLY (same rule as the rest of ``oracle/``).

This operator is not in the paper (whose global attention is the tiled GPA
operator): it is the textbook linear-complexity global attention in which keys
and values over all N tokens are reduced into a fixed-size per-head summary
and normaliser that every query then reads.  The feature map is taken as
phi(x) = elu(x) + 1 (Katharopoulos et al., 2020, "Transformers are RNNs"),
which is positive, so the normaliser never vanishes.  Per (b, h):

    S      = sum_n phi(k_n) v_n^T          (d x d summary)
    z      = sum_n phi(k_n)                (d normaliser)
    out_i  = phi(q_i)^T S / (phi(q_i)^T z)

and, for a loss with upstream gradient g_i = dL/dout_i (den_i = phi(q_i) . z):

    dphi(q_i) = (S g_i - z (g_i . out_i)) / den_i,      dq_i = dphi(q_i) * phi'(q_i)
    dS        = sum_i phi(q_i) (g_i / den_i)^T           (query-side gradient summary)
    dz        = -sum_i phi(q_i) (g_i . out_i) / den_i
    dphi(k_n) = dS v_n + dz,                             dk_n = dphi(k_n) * phi'(k_n)
    dv_n      = dS^T phi(k_n)

with phi'(x) = 1 for x > 0 and exp(x) otherwise.  The definition written out
in that order (numpy float64); ``brute`` is the O(N^2) form with explicit
weights w_ij = phi(q_i) . phi(k_j).
"""
from __future__ import annotations

import numpy as np


def phi(x) -> np.ndarray:
    x = np.asarray(x, dtype=np.float64)
    return np.where(x > 0, x + 1.0, np.exp(np.minimum(x, 0.0)))


def summary(k, v):
    """(S [B, nh, d, d], z [B, nh, d]) from k, v [B, nh, N, d]."""
    fk = phi(k)
    S = np.einsum("bhnk,bhnv->bhkv", fk, np.asarray(v, dtype=np.float64))
    z = fk.sum(axis=2)
    return S, z


def forward(q, k, v) -> np.ndarray:
    """out [B, nh, N, d], float64."""
    S, z = summary(k, v)
    fq = phi(q)
    num = np.einsum("bhnk,bhkv->bhnv", fq, S)
    den = np.einsum("bhnk,bhk->bhn", fq, z)
    return num / den[..., None]


def dphi(x) -> np.ndarray:
    x = np.asarray(x, dtype=np.float64)
    return np.where(x > 0, 1.0, np.exp(np.minimum(x, 0.0)))


def backward(q, k, v, g):
    """(dq, dk, dv) of the loss sum(out * g), float64."""
    q, k, v, g = (np.asarray(t, dtype=np.float64) for t in (q, k, v, g))
    S, z = summary(k, v)
    fq, fk = phi(q), phi(k)
    den = np.einsum("bhnk,bhk->bhn", fq, z)
    out = np.einsum("bhnk,bhkv->bhnv", fq, S) / den[..., None]
    go = np.einsum("bhnv,bhnv->bhn", g, out)
    dfq = (np.einsum("bhkv,bhnv->bhnk", S, g) - z[:, :, None, :] * go[..., None]) / den[..., None]
    dS = np.einsum("bhnk,bhnv->bhkv", fq, g / den[..., None])
    dz = -np.einsum("bhnk,bhn->bhk", fq, go / den)
    dfk = np.einsum("bhkv,bhnv->bhnk", dS, v) + dz[:, :, None, :]
    dv = np.einsum("bhkv,bhnk->bhnv", dS, fk)
    return dfq * dphi(q), dfk * dphi(k), dv


def forward_rows(q, k, v, rows, S=None, z=None):
    """out at sampled (b, h, i) rows, [n, d]; S, z may be passed (from summary)."""
    if S is None or z is None:
        S, z = summary(k, v)
    rows = np.asarray(rows, dtype=np.int64).reshape(-1, 3)
    out = np.empty((rows.shape[0], S.shape[-1]))
    for r, (b, h, i) in enumerate(rows):
        fq = phi(q[b, h, i])
        out[r] = (fq @ S[b, h]) / (fq @ z[b, h])
    return out


def brute(q, k, v) -> np.ndarray:
    """O(N^2) evaluation: w_ij = phi(q_i) . phi(k_j); out_i = sum_j w_ij v_j / sum_j w_ij."""
    w = np.einsum("bhid,bhjd->bhij", phi(q), phi(k))
    return np.einsum("bhij,bhjd->bhid", w, np.asarray(v, dtype=np.float64)) / w.sum(axis=-1)[..., None]
