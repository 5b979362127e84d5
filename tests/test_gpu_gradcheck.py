"""Hand-written backward vs FP64 finite differences (gradient-check workload:
32 x 32 grid, N = 1,024, 2 heads, d = 32, 4 tiles with halos; step 1e-6).
The GPU gradient (plain FP32 form, d = 32) is compared with central
differences of the FP64 oracle forward along random directions and single
elements: FP32 accuracy, relative error <= 1e-5."""
import numpy as np
import pytest
import torch

import oracle
from paper_2604_16590_gb300 import build, gattn
from paper_2604_16590_gb300.inputs import WORKLOADS, workload_inputs

pytestmark = pytest.mark.gpu


def test_backward_against_fp64_finite_differences():
    build.build()
    gattn.load_library()
    w = WORKLOADS["c4_grad"]
    q, k, v, go = workload_inputs(w)
    tiling = gattn.Tiling(w.grid, w.core, w.halo)
    tq, tk, tv, tg = (t.cuda() for t in (q, k, v, go))
    out, saved = gattn.forward(tq, tk, tv, tiling, out_dtype=torch.float32)
    grads = [t.double().cpu().numpy() for t in gattn.backward(tq, tk, tv, out, tg, saved, tiling)]
    assert gattn.gattn_stream_status() == 0
    geo = oracle.Geometry(w.B, w.nh, w.d, *w.grid, w.core, w.halo)
    x = [t.double().numpy() for t in (q, k, v)]
    g = go.double().numpy()
    loss = lambda a: float((oracle.forward(geo, *a) * g).sum())  # noqa: E731
    rng = np.random.default_rng(7)
    eps = 1e-6
    for which in range(3):
        for _ in range(12):
            u = rng.standard_normal(x[which].shape)
            xp = [a + eps * u if n == which else a for n, a in enumerate(x)]
            xm = [a - eps * u if n == which else a for n, a in enumerate(x)]
            fd = (loss(xp) - loss(xm)) / (2 * eps)
            an = float((grads[which] * u).sum())
            assert abs(fd - an) <= 1e-5 * max(1.0, abs(fd)), (which, fd, an)
        for _ in range(24):
            idx = tuple(int(rng.integers(0, s)) for s in x[which].shape)
            e = np.zeros(x[which].shape)
            e[idx] = eps
            xp = [a + e if n == which else a for n, a in enumerate(x)]
            xm = [a - e if n == which else a for n, a in enumerate(x)]
            fd = (loss(xp) - loss(xm)) / (2 * eps)
            assert abs(fd - grads[which][idx]) <= 1e-5 * max(1.0, abs(fd)), (which, idx, fd, grads[which][idx])
