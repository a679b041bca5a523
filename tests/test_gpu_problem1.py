"""Problem I (Section 5.2): the paper's svN needs 30 Newton iterations at 1 km
(N = 512) for a 10^4 residual reduction with direct solves (37 and 45 at 0.5
and 0.25 km).  The oracle, with direct solves on the same discretisation,
needs 20 at 1 km (tests/golden/problem_one_oracle.json, written by
tests/golden/make_problem_one.py); readings of the paper's setup that could
move the count -- the residual norm (l2 vector, M and M^-1 weighted), the
quadrature order (2x2, 3x3, 4x4 Gauss), the line search (energy or residual
norm), P* taken literally as 27.5 N/m^2, Delta_min -- change it by -2 to +5
at 4 and 2 km, none towards the paper's growth with refinement.  The GPU
path (near-exact FGMRES solves) must reproduce the oracle's count within +-1;
the paper's number is printed beside it as context."""
import json
import os

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "problem_one_oracle.json")


def test_problem_one_newton_count_matches_oracle():
    import torch
    from paper_2204_10822_gb300 import Solver
    ref = json.load(open(GOLDEN))["runs"]["512"]["newton_iters"]
    p = W.problem_one(512)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    s = Solver(512, p.L, f_c=0.0, krylov_rtol=1e-8, max_krylov=2000, cheb_degree=6, cheb_lo=0.02)
    s.set_forcing(t(p.h), t(p.A), t(p.wind), t(p.ocean), t(p.v_old))
    _, st = s.step(p.dt, 1e-4)
    print("Problem I, 1 km: GPU %d Newton iterations, oracle %d, paper 30" % (st["newton_iters"], ref))
    assert abs(st["newton_iters"] - ref) <= 1, (st["newton_iters"], ref)
