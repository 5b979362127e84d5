"""Error metrics for GPU-vs-oracle parity (per output tensor, per (batch, head)).

max-rel = max|got - ref| / max|ref| and rms-rel = ||got - ref||_2 / ||ref||_2,
both over the (N, d) slice of one (batch, head); the worst slice is reported.
Elementwise relative error is not used: GPA outputs are near-averages of the
values and cross zero everywhere.
"""
import numpy as np


def rel_errors(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert got.shape == ref.shape, (got.shape, ref.shape)
    if got.ndim == 2:
        got, ref = got[None, None], ref[None, None]
    diff = got - ref
    B, H = ref.shape[:2]
    mx = rms = 0.0
    for b in range(B):
        for h in range(H):
            r, dlt = ref[b, h], diff[b, h]
            den = np.abs(r).max()
            mx = max(mx, np.abs(dlt).max() / den if den > 0 else np.abs(dlt).max())
            n2 = np.linalg.norm(r)
            rms = max(rms, np.linalg.norm(dlt) / n2 if n2 > 0 else np.linalg.norm(dlt))
    return mx, rms


def assert_close(name, got, ref, max_rel, rms_rel):
    mx, rms = rel_errors(got, ref)
    assert np.isfinite(got).all(), f"{name}: non-finite output"
    assert mx <= max_rel and rms <= rms_rel, f"{name}: max-rel {mx:.3e} (<= {max_rel}), rms-rel {rms:.3e} (<= {rms_rel})"
    return mx, rms
