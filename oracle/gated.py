"""FP64 CPU oracle of STORM-DiT's noise-gated self + cross attention
(arXiv 2604.16590, Sec. III-B, the STORM-DiT layer and the noise-gated
attention paragraph).

TEST INFRASTRUCTURE ONLY (same rule as the rest of ``oracle/``).

Each layer runs spatial self-attention on the current state and
cross-attention from the current state (queries) to the compressed temporal
representation (keys and values), both tile-local GPA operators on the same
grid and tiling, and blends them with a per-head gate g set by the noise level:

    out = g_h * GPA(q, k, v) + (1 - g_h) * GPA(q, kc, vc)

The two branches are the pinned GPA oracle; the blend is the definition.
"""
from __future__ import annotations

import numpy as np

from . import forward as gpa_forward


def forward(geo, q, k, v, kc, vc, gate) -> np.ndarray:
    """[B, nh, N, d] float64; gate: [nh]."""
    g = np.asarray(gate, dtype=np.float64).reshape(1, -1, 1, 1)
    assert g.shape[1] == geo.nh
    return g * gpa_forward(geo, q, k, v) + (1.0 - g) * gpa_forward(geo, q, kc, vc)
