"""The stored oracle counts of Problem I (tests/golden/problem_one_oracle.json,
used by the GPU test at 1 km) are reproduced by the oracle at 4 km."""
import json
import os

import workloads as W
from oracle.newton import newton

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "problem_one_oracle.json")


def test_golden_problem_one_count_at_4km():
    ref = json.load(open(GOLDEN))["runs"]["128"]
    r = newton(W.problem_one(128), tol=1e-4)
    assert r.converged and r.newton_iters == ref["newton_iters"], (r.newton_iters, ref["newton_iters"])
