"""Writes problem_one_oracle.json: the oracle's svN Newton counts for the
paper's Problem I (Section 5.2: 10^4 residual reduction, direct solves) at
128^2, 256^2 and 512^2 cells (4, 2 and 1 km).  Calls only oracle/ and
workloads/; run from the repository root:  python tests/golden/make_problem_one.py
(about 10 minutes on one core)."""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as W  # noqa: E402
from oracle.newton import newton  # noqa: E402


def main():
    out = {"source": "oracle.newton on workloads.problem_one, tol 1e-4 (10^4 reduction), direct solves",
           "paper_section": "Section 5.2, Problem I; the paper prints 30 / 37 / 45 at 1 / 0.5 / 0.25 km",
           "runs": {}}
    for N in (128, 256, 512):
        p = W.problem_one(N)
        r = newton(p, tol=1e-4)
        out["runs"][str(N)] = {"km": 512.0 / N, "newton_iters": r.newton_iters, "converged": r.converged,
                               "rel_res": [h / r.res_hist[0] for h in r.res_hist]}
        print(N, r.newton_iters, flush=True)
    with open(os.path.join(HERE, "problem_one_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
