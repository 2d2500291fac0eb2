"""The oracle reproduces its stored results on the two plain image workloads.

The fixtures are written by tests/golden/make_golden.py, which calls only
the oracle; this guards the oracle against unintended drift.
"""
import json
import os

import numpy as np
import pytest

from tests.golden.make_golden import run

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.mark.parametrize("which,name", [(1, "image64_f64.json"), (2, "image512_f32.json")])
def test_oracle_matches_golden(which, name):
    ref = json.load(open(os.path.join(HERE, name)))
    got = run(which)
    assert got["iters"] == ref["iters"]
    assert np.allclose(got["rho"], ref["rho"], rtol=1e-9, atol=0)
    assert got["mu"] == ref["mu"]
    assert np.allclose(got["sample_X"], ref["sample_X"], rtol=1e-8, atol=1e-12)
