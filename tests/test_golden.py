"""The oracle against its stored regression records (tests/golden/, written
by tests/golden/make_golden.py from the oracle itself): same step sequence,
iteration counts and status; costs, controls and final states to 1e-12."""
import json
import os

import numpy as np
import pytest

from golden.make_golden import CASES, compute

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.mark.parametrize("name", sorted(CASES))
def test_oracle_matches_golden(name):
    ref = json.load(open(os.path.join(HERE, name + ".json")))
    cur = compute(name)
    assert cur["alpha_hist"] == ref["alpha_hist"]
    assert cur["iters"] == ref["iters"] and cur["status"] == ref["status"]
    for k in ("J", "U", "X_T"):
        np.testing.assert_allclose(np.array(cur[k]), np.array(ref[k]), rtol=1e-12, atol=1e-14)
