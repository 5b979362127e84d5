"""Writes tests/golden/gpa_small.json: a regression fixture of the FP64 oracle.

The paper prints no worked numerical example of STORM-GPA, so no fixture here
holds a value from the paper.  This one is written by the oracle itself
(oracle.forward / oracle.backward, Sec. III-C: tiles with halos, softmax
attention per extended tile, Hann-weighted average of the overlaps, and its
analytic gradient) on a small seeded case, and tests/test_oracle_golden.py
checks that the oracle still reproduces it.  It is not an independent pin
(those are in tests/test_oracle_pins.py); it makes any change to the
oracle's arithmetic visible as a change of this file, which then needs this
script and a commit that names the passage justifying the change.

Run from the repository root:  python tests/golden/make_gpa_small.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402

# two frames of a 5 x 6 grid, 2 x 2 x 3 cores, a one-token halo in every
# dimension: tokens covered by up to eight tiles; B = 1, two heads, d = 4
CASE = {"B": 1, "nh": 2, "d": 4, "grid": [2, 5, 6], "core": [1, 2, 3], "halo": [1, 1, 1], "seed": 20260417}


def inputs(case):
    rng = np.random.default_rng(case["seed"])
    N = int(np.prod(case["grid"]))
    shape = (case["B"], case["nh"], N, case["d"])
    return [rng.standard_normal(shape) for _ in range(4)]  # q, k, v, dOut


def compute(case):
    q, k, v, go = inputs(case)
    geo = oracle.Geometry(case["B"], case["nh"], case["d"], *case["grid"], tuple(case["core"]), tuple(case["halo"]))
    out = oracle.forward(geo, q, k, v)
    dq, dk, dv = oracle.backward(geo, q, k, v, go)
    return {"out": out, "dq": dq, "dk": dk, "dv": dv}


def main():
    res = compute(CASE)
    doc = {"case": CASE, "source": "oracle.forward / oracle.backward (FP64), inputs from numpy default_rng(seed)",
           **{k: [float(f"{x:.17g}") for x in v.ravel()] for k, v in res.items()}}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "gpa_small.json")
    with open(path, "w") as f:
        json.dump(doc, f, indent=None, separators=(",", ":"))
        f.write("\n")
    print("wrote", path, {k: len(v) for k, v in doc.items() if isinstance(v, list)})


if __name__ == "__main__":
    main()
