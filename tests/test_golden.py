"""Stored expected values (tests/golden/) are what the oracle computes now:
a change of the oracle's arithmetic that moves them fails here and has to be
justified when the fixtures are regenerated (tests/golden/make_golden.py).
Fixtures whose regeneration is slow are checked instead through the
equations that define them, evaluated by the oracle at the stored solution."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import make_golden as mg  # noqa: E402


def _flat(d):
    out = {}
    for k, x in d.items():
        out[k] = np.atleast_1d(np.asarray(x, dtype=np.float64))
    return out


@pytest.mark.parametrize("name", sorted(mg.FIXTURES))
def test_fixture_matches_oracle(name):
    stored = mg.load(name)
    if name in mg.VERIFY:
        for what, (value, bound) in mg.VERIFY[name](stored).items():
            assert value < bound, (what, value)
        return
    fresh, tol = mg.FIXTURES[name](), 1e-10
    assert stored["inputs"] == fresh["inputs"]
    assert stored["citation"] == fresh["citation"]
    a, b = _flat(stored["values"]), _flat(fresh["values"])
    assert a.keys() == b.keys()
    for k in a:
        assert a[k].shape == b[k].shape, k
        assert np.abs(a[k] - b[k]).max() < tol, k
