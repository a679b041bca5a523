"""Soft pin against the paper's printed numbers (Problem I, Section 5.2):
svN needs 30 Newton iterations at 1 km (N = 512) for a 10^4 reduction with
direct solves.  Discretisation details differ (2x2 Gauss for every term, the
line-search floor), so the count is expected in the same range, not equal;
measured here: 20 (and 22, 24 at 0.5, 0.25 km, against the paper's 37, 45)."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def test_problem_one_newton_count_same_range_as_paper():
    import torch
    from paper_2204_10822_gb300 import Solver
    p = W.problem_one(512)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    s = Solver(512, p.L, f_c=0.0, krylov_rtol=1e-8, max_krylov=2000, cheb_degree=6, cheb_lo=0.02)
    s.set_forcing(t(p.h), t(p.A), t(p.wind), t(p.ocean), t(p.v_old))
    _, st = s.step(p.dt, 1e-4)
    assert 15 <= st["newton_iters"] <= 45, st["newton_iters"]
