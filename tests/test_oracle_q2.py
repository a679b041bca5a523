"""Pins of the oracle's Q2 (biquadratic) velocity discretisation.

  * the 9-node basis reproduces biquadratic fields and their gradients exactly
    at the 3 x 3 Gauss points;
  * with P* = 0 and Co = 0 the step is a mass-matrix solve whose Q2 mass matrix
    on the uniform grid is the Kronecker product of the 1-D quadratic element
    matrices (dx/30) [[4, 2, -1], [2, 16, 2], [-1, 2, 4]] (written here, not
    taken from the oracle);
  * R = grad Phi_h and K_stdN = grad R (finite differences), K_svN at
    pi = tau/Delta equals K_stdN, and the modified operator is SPD;
  * the linear limit (Delta_min huge, Co = 0) is solved by one Newton step;
  * a manufactured solution (the same strong form as the Q1 pin, from the
    original VP rheology) converges at third order in L2, one order more than
    Q1; a planted factor in tau drops it to zero.
"""
import dataclasses
import math

import numpy as np
import pytest

import workloads as W
from oracle.fem_q2 import QPTS2, Q2Mesh, Step2
from oracle.newton import newton


def problem(N=4, seed=3, **kw):
    c = dataclasses.replace(W.Constants(), **kw)
    return W.make_problem_q2(N, seed=seed, const=c)


def random_velocity(N, seed, scale=0.1):
    rng = np.random.default_rng(seed)
    v = scale * rng.standard_normal((2 * N + 1, 2 * N + 1, 2))
    v[0], v[-1], v[:, 0], v[:, -1] = 0, 0, 0, 0
    return v


def qp_coords(N, L):
    dx = L / N
    jj, ii = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    X = np.stack([(ii + xi) * dx for xi, _ in QPTS2], axis=-1)
    Y = np.stack([(jj + eta) * dx for _, eta in QPTS2], axis=-1)
    return X, Y


def test_basis_reproduces_biquadratic_fields():
    N, L = 3, 6.0
    m = Q2Mesh(N, L, 2.0)
    x = np.linspace(0, L, 2 * N + 1)
    Xn, Yn = np.meshgrid(x, x, indexing="xy")
    f = lambda X, Y: 1 + 2 * X - Y + 0.5 * X * Y + X * X - 0.3 * Y * Y + 0.2 * X * X * Y * Y
    fx = lambda X, Y: 2 + 0.5 * Y + 2 * X + 0.4 * X * Y * Y
    fy = lambda X, Y: -1 + 0.5 * X - 0.6 * Y + 0.4 * X * X * Y
    u = np.stack([f(Xn, Yn), -f(Yn, Xn)], axis=-1)
    X, Y = qp_coords(N, L)
    uq = m.node_to_qp(u)
    assert np.abs(uq[..., 0] - f(X, Y)).max() < 1e-12
    g = np.einsum("qkdl,nml->nmqkd", m.Gq, m.gather(u))
    assert np.abs(g[..., 0, 0] - fx(X, Y)).max() < 1e-11
    assert np.abs(g[..., 0, 1] - fy(X, Y)).max() < 1e-11


def test_mass_matrix_is_the_kronecker_product_of_1d_quadratic_elements():
    N, L = 4, 512e3
    dx = L / N
    c = dataclasses.replace(W.Constants(), Pstar=0.0, Co=0.0)
    p = W.make_problem_q2(N, seed=1, const=c)
    p.h[:] = 1.0
    st = Step2(p)
    K = st.stdn_matrix(np.zeros_like(p.v_old)).toarray()
    n1 = 2 * N + 1
    M1 = np.zeros((n1, n1))
    Me = dx / 30.0 * np.array([[4.0, 2.0, -1.0], [2.0, 16.0, 2.0], [-1.0, 2.0, 4.0]])
    for e in range(N):
        M1[2 * e:2 * e + 3, 2 * e:2 * e + 3] += Me
    M1 = M1[1:-1, 1:-1]
    M2 = c.rho_ice * np.kron(M1, M1)
    # free dofs interleave the two components: node-major, component-minor
    Kx = K[0::2, 0::2]
    assert np.abs(Kx - M2).max() <= 1e-12 * np.abs(M2).max()
    assert np.abs(K[0::2, 1::2]).max() <= 1e-12 * np.abs(M2).max()


def test_residual_is_energy_gradient():
    p = problem(N=4)
    st = Step2(p)
    v = random_velocity(4, 1)
    R = st.residual(v)
    rng = np.random.default_rng(7)
    for _ in range(3):
        d = random_velocity(4, rng.integers(1 << 30), scale=1.0)
        eps = 1e-5
        fd = (st.energy(v + eps * d) - st.energy(v - eps * d)) / (2 * eps)
        an = float(np.sum(R * d))
        assert abs(fd - an) <= 1e-6 * abs(an), (fd, an)


def test_stdn_jacobian_is_residual_derivative_and_svn_matches_at_consistent_pi():
    p = problem(N=3)
    st = Step2(p)
    v = random_velocity(3, 2)
    K = st.stdn_matrix(v)
    d = random_velocity(3, 5, scale=1.0)
    eps = 1e-6
    fd = (st.residual(v + eps * d) - st.residual(v - eps * d)) / (2 * eps)
    an = st.from_free(K @ st.to_free(d))
    assert np.linalg.norm(fd - an) <= 1e-6 * np.linalg.norm(an)
    Ks = st.svn_matrix(v, st.pi_of(v))
    assert abs(Ks - K).max() <= 1e-13 * abs(K).max()


@pytest.mark.parametrize("big", [False, True])
def test_svn_operator_symmetric_positive_definite(big):
    p = problem(N=3)
    st = Step2(p)
    v = random_velocity(3, 5)
    rng = np.random.default_rng(13)
    pi = rng.standard_normal((3, 3, 9, 3)) * (3.0 if big else 0.2)
    K = st.svn_matrix(v, pi).toarray()
    assert np.abs(K - K.T).max() <= 1e-14 * np.abs(K).max()
    assert np.linalg.eigvalsh(K).min() > 0


def test_linear_limit_one_newton_step():
    p = problem(N=6, delta_min=1.0, Co=0.0)
    res = newton(p, tol=1e-10, step=Step2(p))
    assert res.converged and res.newton_iters == 1, res.res_hist


def test_newton_converges_and_pi_consistent():
    p = problem(N=8, seed=0)
    st = Step2(p)
    res = newton(p, tol=1e-10, step=st)
    assert res.converged
    pc = st.pi_of(res.v)
    assert np.abs(res.pi - pc).max() <= 1e-6 * np.abs(pc).max()


sympy = pytest.importorskip("sympy")


def mms_errors(Ns, tau_factor=1.0):
    from test_oracle_mms import manufactured
    L, U, dt = 512e3, 0.1, 1800.0
    c = dataclasses.replace(W.Constants(), delta_min=1e-7)
    f_src, f_v = manufactured(c, L, U, dt, c.rho_ice, c.Pstar)
    errs = []
    for N in Ns:
        p = W.Problem(N=N, L=L, const=c, h=np.ones((N, N)), A=np.ones((N, N)),
                      wind=np.zeros((2 * N + 1, 2 * N + 1, 2)), ocean=W.ocean_gyre(2 * N, L),
                      v_old=np.zeros((2 * N + 1, 2 * N + 1, 2)), dt=dt)
        st = Step2(p)
        if tau_factor != 1.0:          # planted mistake: tau scaled in the operator tables
            st.mesh.Bq = st.mesh.Bq * tau_factor
        X, Y = qp_coords(N, L)
        sx, sy = f_src(X, Y)
        st.tau_atm = np.stack([np.broadcast_to(sx, X.shape), np.broadcast_to(sy, X.shape)], -1)
        res = newton(p, tol=1e-11, step=st)
        assert res.converged
        vq = st.mesh.node_to_qp(res.v)
        ex, ey = f_v(X, Y)
        errs.append(math.sqrt(np.sum(st.mesh.w * ((vq[..., 0] - ex) ** 2 + (vq[..., 1] - ey) ** 2))))
    return errs


def test_manufactured_solution_third_order():
    errs = mms_errors((4, 8, 16))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert orders[-1] > 2.7, (errs, orders)


def test_manufactured_solution_planted_tau_factor_loses_convergence():
    errs = mms_errors((8, 16), tau_factor=1.1)
    assert math.log2(errs[0] / errs[1]) < 0.5, errs
