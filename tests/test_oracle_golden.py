"""The FP64 oracle against its stored regression fixture (tests/golden).

The fixture was written by tests/golden/make_gpa_small.py from the oracle
itself (the paper prints no worked numerical example): a change of the
oracle's arithmetic shows up here first, and regenerating the fixture is a
deliberate step with its own commit.  Independent pins of the oracle are in
tests/test_oracle_pins.py."""
import importlib.util
import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def _maker():
    spec = importlib.util.spec_from_file_location("make_gpa_small", os.path.join(HERE, "golden", "make_gpa_small.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_oracle_reproduces_the_stored_fixture():
    with open(os.path.join(HERE, "golden", "gpa_small.json")) as f:
        doc = json.load(f)
    mk = _maker()
    assert doc["case"] == mk.CASE
    got = mk.compute(doc["case"])
    for key in ("out", "dq", "dk", "dv"):
        ref = np.asarray(doc[key])
        # FP64, the same operation order; the C compiler may contract a*b+c
        # differently on another instruction set, hence not bitwise
        np.testing.assert_allclose(got[key].ravel(), ref, rtol=1e-12, atol=1e-14, err_msg=key)
