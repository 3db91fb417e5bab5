"""The oracle against its own recorded values (tests/golden/oracle_small_steps.json,
written by tests/golden/make_golden.py, which calls only the oracle and the
seeded input generators).  A regression guard, not a pin against the paper
(the pins are in test_oracle_*.py): a change to the oracle's arithmetic shows
here and must come with the passage or reading that justifies it and a
rewritten record.  Tolerance 1e-12 relative, not bits, so that a different
host compiler or thread count does not trip it."""
import json
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def record():
    with open(os.path.join(HERE, "golden", "oracle_small_steps.json")) as fh:
        return json.load(fh)


def test_oracle_reproduces_its_record(record):
    import sys
    sys.path.insert(0, os.path.join(HERE, "golden"))
    import make_golden
    now = make_golden.compute()
    for k in ("theta_l2", "state_after_5_steps_l2"):
        assert abs(now[k] - record[k]) <= 1e-12 * abs(record[k]), k
    for group, scale in (("theta_at", record["theta_l2"]), ("state_after_5_steps_at", record["state_after_5_steps_l2"])):
        for s, v in record[group].items():
            assert abs(now[group][s] - v) <= 1e-12 * scale, (group, s)
    for k, v in record["observables_after_5_steps"].items():
        assert abs(now["observables_after_5_steps"][k] - v) <= 1e-12 * max(1.0, abs(v)), k
