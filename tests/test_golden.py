"""The oracle reproduces its recorded results on fixed synthetic inputs
(tests/golden/oracle_digests.json, written by tests/golden/make_golden.py)."""
import json
import os

import pytest

from tests.golden import make_golden

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_digests.json")


def recorded():
    with open(GOLDEN) as f:
        return json.load(f)


def test_recorded_configuration_is_the_one_the_script_uses():
    assert recorded()["config"] == make_golden.CFG
    assert [c["name"] for c in recorded()["cases"]] == [c[0] for c in make_golden.CASES]


@pytest.mark.parametrize("case", make_golden.CASES, ids=[c[0] for c in make_golden.CASES])
def test_oracle_reproduces_recorded_results(case):
    want = next(c for c in recorded()["cases"] if c["name"] == case[0])
    got = make_golden.run(case)
    assert got == want
