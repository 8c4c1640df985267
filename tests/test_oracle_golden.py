"""Regression guard: the oracle still reproduces its stored tiny-scene output
(tests/golden/oracle_tiny.json, written by tests/golden/make_golden.py from the
oracle alone)."""
import json
import os

import pytest

from tests.golden.make_golden import make


def test_oracle_reproduces_golden():
    with open(os.path.join(os.path.dirname(__file__), "golden", "oracle_tiny.json")) as f:
        want = json.load(f)
    got = make()
    assert got["keys_tile8_first16"] == want["keys_tile8_first16"]
    assert got["vals_tile8_first16"] == want["vals_tile8_first16"]
    assert got["M_tile8"] == want["M_tile8"]
    for a, b in zip(got["pixels"], want["pixels"]):
        assert a["nb"] == b["nb"]
        assert a["T"] == pytest.approx(b["T"], rel=1e-12)
        assert a["rgb"] == pytest.approx(b["rgb"], rel=1e-12, abs=1e-15)
    assert got["sum_d_means"] == pytest.approx(want["sum_d_means"], rel=1e-9, abs=1e-15)
    assert got["sum_d_color"] == pytest.approx(want["sum_d_color"], rel=1e-9)
