"""Forcing terms of the inexact Newton iteration (the Krylov tolerance of each
Newton step; the paper solves each linearisation directly, Section 5.1).

With Eisenstat-Walker forcing, `ew_tail` raises the tolerance of a step whose
residual is already near the stopping threshold to
min(ew_eta_max, ew_tail * tol * ||R_0|| / ||R_k||) (Kelley 1995, Sect. 6.3).
Until the first Newton iteration where that floor is above the Eisenstat-Walker
value the two runs are the same computation; at that iteration FGMRES solves
the same system to a looser tolerance and so stops no later.  Both runs must
reach the requested residual, and their solutions agree to within what that
residual allows."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

SETTINGS = dict(precision="mixed", vcycle_fp32=1, eisenstat_walker=1, krylov_rtol=1e-3, ew_eta_max=0.03,
                max_krylov=600, cheb_degree=6, cheb_lo=0.02)


def test_tail_floor_relaxes_only_the_last_steps():
    import torch
    from paper_2204_10822_gb300 import Solver
    N, tol = 512, 1e-8
    p = W.config(2, N=N)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    dev_in = [t(p.h), t(p.A), t(p.wind), t(p.ocean), t(p.v_old)]
    runs = {}
    for tail in (0.0, 0.5):
        s = Solver(N, p.L, **dict(SETTINGS, ew_tail=tail))
        s.set_forcing(*dev_in)
        v, st = s.step(p.dt, tol)
        runs[tail] = (v.clone(), st)
        s.close()
    (va, a), (vb, b) = runs[0.0], runs[0.5]
    ka, kb = a["krylov_per_newton"], b["krylov_per_newton"]
    print("ew_tail 0: %d Newton, %d FGMRES, rel-res %.2e; ew_tail 0.5: %d Newton, %d FGMRES, rel-res %.2e" % (
        a["newton_iters"], a["krylov_iters_total"], a["rel_res_final"], b["newton_iters"],
        b["krylov_iters_total"], b["rel_res_final"]))
    assert a["rel_res_final"] <= tol and b["rel_res_final"] <= tol
    # the floor takes effect at some Newton iteration
    assert ka != kb
    k = next(i for i in range(min(len(ka), len(kb))) if ka[i] != kb[i])
    # identical before it, and no later to stop at it (unless the looser
    # direction was recomputed by the retry safeguard)
    assert ka[:k] == kb[:k]
    if b["direction_retries"] == 0:
        assert kb[k] <= ka[k], (k, ka, kb)
    d = float(torch.linalg.vector_norm(vb - va) / torch.linalg.vector_norm(va))
    assert d <= 1e-6, d
