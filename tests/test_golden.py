"""The oracle still reproduces the stored fixtures written by
tests/golden/make_golden.py (bit for bit on the per-face and per-cell
assembly, to rounding on the dense solve)."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import make_golden  # noqa: E402

import oracle  # noqa: E402


@pytest.mark.parametrize("name", sorted(make_golden.FIXTURES))
def test_oracle_reproduces_golden(name):
    c, gold = make_golden.case(name)
    p, fc, sy, _ = oracle.solve(c, direct=True)
    assert np.array_equal(fc.lam, gold["lam"])
    assert np.array_equal(fc.gamma, gold["gamma"])
    assert np.array_equal(fc.jump, gold["jump"])
    assert np.array_equal(sy.diag, gold["diag"])
    assert np.array_equal(sy.b, gold["b"])
    assert np.linalg.norm(p - gold["p"]) <= 1e-13 * np.linalg.norm(gold["p"])
