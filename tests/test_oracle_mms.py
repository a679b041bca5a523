"""Manufactured-solution pin of the oracle's discretisation.

The strong form of the implicit step (Eq. "momen" discretised by implicit
Euler, Section 3) is written with SymPy from the paper's ORIGINAL rheology
  sigma = 2 eta eps'(v) + zeta tr(eps(v)) I - P/2 I,
  eta = zeta / e^2, zeta = P / (2 Delta),
  Delta = sqrt(2 e^-2 eps':eps' + tr(eps)^2 + Delta_min^2)      (Eq. "Delta")
-- not from the tau-form the oracle uses -- so a wrong factor in tau(v), in
Delta or in the viscous-plastic term of the residual shows up as a missing
second-order convergence.  The source enters through the atmospheric-stress
slot at the quadrature points.  Expected: L2 error O(dx^2).
"""
import dataclasses

import numpy as np
import pytest

import workloads as W
from oracle.fem import Step
from oracle.newton import newton

sympy = pytest.importorskip("sympy")


def manufactured(c, L, U, dt, rhoH, P):
    x, y = sympy.symbols("x y", real=True)
    pi = sympy.pi
    vx = U * sympy.sin(pi * x / L) * sympy.sin(2 * pi * y / L)
    vy = -U * sympy.sin(2 * pi * x / L) * sympy.sin(pi * y / L)
    ox = -0.1 * sympy.sin(pi * x / L) * sympy.cos(pi * y / L)
    oy = 0.1 * sympy.cos(pi * x / L) * sympy.sin(pi * y / L)
    g = sympy.Matrix([[sympy.diff(vx, x), sympy.diff(vx, y)],
                      [sympy.diff(vy, x), sympy.diff(vy, y)]])
    eps = (g + g.T) / 2
    tr = eps.trace()
    epsd = eps - tr / 2 * sympy.eye(2)
    dd = sum(epsd[i, j] ** 2 for i in range(2) for j in range(2))
    Delta = sympy.sqrt(2 / c.e ** 2 * dd + tr ** 2 + c.delta_min ** 2)
    zeta = P / (2 * Delta)
    eta = zeta / c.e ** 2
    sigma = 2 * eta * epsd + zeta * tr * sympy.eye(2) - P / 2 * sympy.eye(2)
    div = [sympy.diff(sigma[k, 0], x) + sympy.diff(sigma[k, 1], y) for k in range(2)]
    wx, wy = ox - vx, oy - vy
    nw = sympy.sqrt(wx ** 2 + wy ** 2)
    drag = [c.Co * c.rho_o * nw * wx, c.Co * c.rho_o * nw * wy]
    # v^n = 0:  rho H v - dt div sigma - dt tau_ocean + dt rho H f e_r x (0 - v_o) = dt g
    cor = [rhoH * c.f_c * oy, -rhoH * c.f_c * ox]      # e_r x (-v_o) = (o_y, -o_x)
    src = [(rhoH * v - dt * dv - dt * dr + dt * cr) / dt
           for v, dv, dr, cr in zip((vx, vy), div, drag, cor)]
    f_src = sympy.lambdify((x, y), src, "numpy")
    f_v = sympy.lambdify((x, y), [vx, vy], "numpy")
    return f_src, f_v


def qp_coords(st):
    from oracle.fem import QPTS
    N, dx = st.mesh.N, st.mesh.dx
    jj, ii = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    X = np.stack([(ii + xi) * dx for xi, _ in QPTS], axis=-1)
    Y = np.stack([(jj + eta) * dx for _, eta in QPTS], axis=-1)
    return X, Y


def test_manufactured_solution_second_order():
    L, U, dt = 512e3, 0.1, 1800.0
    c = dataclasses.replace(W.Constants(), delta_min=1e-7)
    P = c.Pstar          # h = 1, A = 1
    rhoH = c.rho_ice
    f_src, f_v = manufactured(c, L, U, dt, rhoH, P)
    errs = []
    Ns = (8, 16, 32)
    for N in Ns:
        ocean = W.ocean_gyre(N, L)
        p = W.Problem(N=N, L=L, const=c, h=np.ones((N, N)), A=np.ones((N, N)),
                      wind=np.zeros((N + 1, N + 1, 2)), ocean=ocean,
                      v_old=np.zeros((N + 1, N + 1, 2)), dt=dt)
        st = Step(p)
        X, Y = qp_coords(st)
        sx, sy = f_src(X, Y)
        st.tau_atm = np.stack([np.broadcast_to(sx, X.shape), np.broadcast_to(sy, X.shape)], -1)
        res = newton(p, tol=1e-11, step=st)
        assert res.converged
        vq = st.mesh.node_to_qp(res.v)
        ex, ey = f_v(X, Y)
        e2 = np.sum(st.mesh.w * ((vq[..., 0] - ex) ** 2 + (vq[..., 1] - ey) ** 2))
        errs.append(np.sqrt(e2))
    orders = [np.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert orders[-1] > 1.8, (errs, orders)
