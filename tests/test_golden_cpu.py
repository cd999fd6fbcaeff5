"""The stored oracle values under tests/golden/ still match the oracle (a
regression guard on the oracle; the fixtures are written by
tests/golden/make_golden.py from the oracle alone)."""
import importlib.util
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def _make_golden():
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "golden", "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_c1_gamma_fixture_matches_oracle():
    mg = _make_golden()
    stored = np.loadtxt(os.path.join(HERE, "golden", "c1_gamma.txt"))
    assert stored.shape == (216, 2)
    assert np.all(stored >= 0) and stored.max() > 0
    got = mg.c1_gamma()
    # summation order may differ between NumPy builds and CPUs by a few ulps
    assert np.abs(got - stored).max() <= 1e-12 * stored.max()
