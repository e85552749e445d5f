"""The oracle against its own stored fingerprints (tests/golden/
oracle_regression.json, written by tests/golden/make_oracle_regression.py):
a guard against unnoticed changes of the oracle's results, beside the pins
that tie it to the paper and to exact results.  A deliberate change of the
oracle's arithmetic regenerates the file in the same commit."""
import json
import os

import pytest

from tests.golden import make_oracle_regression as mk

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_regression.json")

with open(GOLDEN) as f:
    STORED = json.load(f)


@pytest.mark.parametrize("name", sorted(mk.cases()))
def test_oracle_matches_its_fingerprint(name):
    assert name in STORED
    assert mk.fingerprint(mk.cases()[name]) == STORED[name]
