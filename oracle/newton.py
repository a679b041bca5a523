"""Damped Newton for the implicit step: svN and standard Newton (FP64, CPU).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Algorithm (Sections 4.1, 4.2 and 5.1):
  v_0 = v_old (boundary forced to zero), pi_0 = tau(v_0) / Delta(v_0);
  for l = 0, 1, ...:
      stop when ||R(v_l)|| <= tol ||R(v_old)||                     (Section 5.1)
      solve K dv = -R(v_l) with a sparse direct factorisation
      svN: dpi from Eq. "tautilde" (+ Eq. "modification")
      backtracking: alpha = 1, 1/2, ... while Phi does not decrease (Section 5.1)
      v <- v + alpha dv, pi <- pi + alpha dpi                        (same alpha)

Line-search reading (the paper gives no halving limit and no rounding rule):
at most ``max_halvings`` halvings; a step is accepted when Phi strictly
decreases, or when |Phi_new - Phi_old| is at the rounding level of the sum
(1e-13 times the sum of |contributions|) and the residual norm decreases --
the residual-norm backtracking that the paper reports to behave the same.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.sparse.linalg as spla

from .direct import nd_solve
from .fem import Step


@dataclasses.dataclass
class NewtonResult:
    v: np.ndarray
    pi: np.ndarray | None
    newton_iters: int
    res_hist: list
    alphas: list
    halvings_total: int
    converged: bool
    status: str
    phi_hist: list = dataclasses.field(default_factory=list)


# above this many dofs the nested-dissection multifrontal Cholesky of
# ``direct.py`` replaces SuperLU (it is faster from about 128^2 cells on)
ND_MIN_DOFS = 30000


def superlu_solve(K, b):
    """Sparse direct solve (SuperLU with a symmetric fill-reducing ordering)."""
    lu = spla.splu(K.tocsc(), permc_spec="MMD_AT_PLUS_A",
                   options={"SymmetricMode": True})
    return lu.solve(b)


def direct_solve(K, b):
    """Sparse direct solve of a free-dof system: SuperLU on small grids, the
    nested-dissection multifrontal Cholesky on large ones (both exact up to
    rounding; pinned against each other)."""
    if K.shape[0] >= ND_MIN_DOFS:
        return nd_solve(K, b)
    return superlu_solve(K, b)


def line_search(st: Step, v, dv, res_norm, max_halvings=30, floor=1e-13):
    """Backtracking on Phi_h (Section 5.1); returns (alpha, halvings) or (None, n)."""
    phi0 = st.energy(v)
    scale = st.energy_scale(v)
    alpha = 1.0
    for k in range(max_halvings + 1):
        vt = v + alpha * dv
        phi1 = st.energy(vt)
        if phi1 < phi0:
            return alpha, k, phi1
        if abs(phi1 - phi0) <= floor * scale and st.residual_norm(vt) < res_norm:
            return alpha, k, phi1
        alpha *= 0.5
    return None, max_halvings, phi0


def newton(prob, tol=1e-10, method="svn", max_newton=200, max_halvings=30,
           solve=direct_solve, v0=None, pi0=None, linear_solver_hook=None, step=None):
    """Solve one implicit step; ``method`` is "svn" or "stdn".

    ``step`` may pass a prepared ``Step`` (e.g. with a manufactured source in
    the atmospheric-stress slot)."""
    st = Step(prob) if step is None else step
    if solve is direct_solve:
        solve = getattr(st, "direct_solver", direct_solve)
    m = st.mesh
    v = m.zero_boundary(prob.v_old if v0 is None else v0)
    pi = None
    if method == "svn":
        pi = st.pi_of(v) if pi0 is None else np.array(pi0, dtype=np.float64)
    r_ref = st.residual_norm(m.zero_boundary(prob.v_old))
    hist, alphas, halv = [], [], 0
    phis = [st.energy(v)]
    for it in range(max_newton + 1):
        R = st.residual(v)
        r = math.sqrt(math.fsum((R * R).ravel()))
        hist.append(r)
        if r <= tol * r_ref or r == 0.0:
            return NewtonResult(v, pi, it, hist, alphas, halv, True, "ok", phis)
        if it == max_newton:
            break
        K = st.svn_matrix(v, pi) if method == "svn" else st.stdn_matrix(v)
        rhs = -st.to_free(R)
        x = solve(K, rhs) if linear_solver_hook is None else linear_solver_hook(K, rhs)
        dv = st.from_free(x)
        alpha, k, phi1 = line_search(st, v, dv, r, max_halvings)
        halv += k
        if alpha is None:
            return NewtonResult(v, pi, it, hist, alphas, halv, False, "linesearch", phis)
        if method == "svn":
            pi = pi + alpha * st.dual_step(v, dv, pi)
        v = v + alpha * dv
        alphas.append(alpha)
        phis.append(phi1)
    return NewtonResult(v, pi, max_newton, hist, alphas, halv, False, "no_convergence", phis)
