"""The oracle reproduces its stored single-halo summary (regression record
written by tests/golden/make_golden.py, which calls only the oracle)."""
import json
import os

import pytest

from tests.golden.make_golden import summary

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_single_halo_summary_unchanged():
    with open(os.path.join(HERE, "single_halo.json")) as f:
        ref = json.load(f)
    now = summary()
    for k, v in ref.items():
        if isinstance(v, float):
            assert now[k] == pytest.approx(v, rel=1e-12), k
        elif isinstance(v, list) and v and isinstance(v[0], float):
            assert now[k] == pytest.approx(v, rel=1e-12), k
        else:
            assert now[k] == v, k
