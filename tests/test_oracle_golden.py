"""The oracle reproduces its committed regression fixtures bit for bit
(fixtures written by tests/golden/make_golden.py, which calls only the
oracle and the input generator)."""
import os
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_golden  # noqa: E402


@pytest.mark.parametrize("name", sorted(make_golden.CASES))
def test_oracle_matches_golden(name):
    with open(os.path.join(HERE, "golden", name + ".txt")) as f:
        stored = f.read().splitlines()
    assert make_golden.case_lines(name) == stored
