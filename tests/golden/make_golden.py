"""Write oracle_small_steps.json: what the FP64 oracle gives on the 8^2 x 16^2
small workload (seeded input), for tests/test_oracle_golden.py.  It calls
only the oracle and the seeded input generators; no value comes from the
CUDA path.  A regression record of the oracle, not a pin against the paper:
a change to the oracle's arithmetic that moves these values must be made on
purpose, with the passage or reading that justifies it, and the file rewritten
with this script.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2511_11354_gb300 import inputs  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_small_steps.json")
SAMPLES = [(0, 0, 0, 0), (1, 6, 3, 12), (3, 2, 8, 8), (5, 5, 15, 1), (7, 0, 10, 5), (6, 7, 4, 14)]


def compute():
    prob, f0 = inputs.workload_small(nx=8, nk=16)
    o = oracle.Oracle(prob)
    th = o.theta(f0)
    f5 = o.step(f0, 5)
    ob = o.observables(f5)
    return {
        "workload": "workload_small(nx=8, nk=16): L = 20, dt = 0.01, cosine V_ext, soft-Coulomb pair, packets at -+3",
        "theta_at": {"%d,%d,%d,%d" % s: float(th[s]) for s in SAMPLES},
        "theta_l2": float(np.linalg.norm(th)),
        "state_after_5_steps_at": {"%d,%d,%d,%d" % s: float(f5[s]) for s in SAMPLES},
        "state_after_5_steps_l2": float(np.linalg.norm(f5)),
        "observables_after_5_steps": {k: float(ob[k]) for k in ("mass", "energy", "purity", "l2norm")},
    }


if __name__ == "__main__":
    with open(OUT, "w") as fh:
        json.dump(compute(), fh, indent=1, sort_keys=True)
    print(OUT)
