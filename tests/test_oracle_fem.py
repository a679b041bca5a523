"""Pins of the CPU oracle's discretisation against facts the paper and the
mathematics fix, independent of the oracle's own formulas.

  * R = grad Phi_h (Theorem of Section 3; a finite difference of the energy)
  * K_stdN = Jacobian of R (finite difference of the residual)
  * K_svN(v, pi = tau/Delta) == K_stdN(v) (Section 4.2: svN replaces
    tau/Delta by pi, and the modification is inactive when sqrt(2 pi:pi) < 1)
  * the dual step of Eq. "tautilde" is the linearisation of pi(v) = tau/Delta
  * symmetry and positive definiteness of the modified svN operator
    (Eq. "modification"), with pointwise eigenvalue floor
  * convexity of Phi_h along lines
  * closed forms: P* = 0, Co = 0 reduces the step to a mass-matrix solve
    whose Q1 / 2x2-Gauss mass matrix is the Kronecker product of the 1-D
    matrices dx/6 tridiag(1, 4, 1); the explicit Coriolis term rotates v^n
  * linear limit: Delta_min huge and Co = 0 make one Newton step exact.
"""
import dataclasses
import math

import numpy as np
import pytest

import workloads as W
from oracle.fem import Step, comp_to_voigt
from oracle.newton import newton


def small_problem(N=8, seed=3, **const_kw):
    c = dataclasses.replace(W.Constants(), **const_kw)
    p = W.make_problem(N, seed=seed, const=c)
    return p


def random_velocity(N, seed, scale=0.1):
    rng = np.random.default_rng(seed)
    v = scale * rng.standard_normal((N + 1, N + 1, 2))
    v[0], v[-1], v[:, 0], v[:, -1] = 0, 0, 0, 0
    return v


def test_residual_is_energy_gradient():
    p = small_problem(N=8)
    st = Step(p)
    v = random_velocity(8, 1)
    R = st.residual(v)
    rng = np.random.default_rng(7)
    for _ in range(3):
        d = random_velocity(8, rng.integers(1 << 30), scale=1.0)
        eps = 1e-5
        fd = (st.energy(v + eps * d) - st.energy(v - eps * d)) / (2 * eps)
        an = float(np.sum(R * d))
        assert abs(fd - an) <= 1e-6 * (abs(an) + 1e-30) + 1e-9 * st.energy_scale(v) / eps * 1e-6, (fd, an)


def test_stdn_jacobian_is_residual_derivative():
    p = small_problem(N=6)
    st = Step(p)
    v = random_velocity(6, 2)
    K = st.stdn_matrix(v)
    rng = np.random.default_rng(11)
    d = random_velocity(6, 5, scale=1.0)
    eps = 1e-6
    fd = (st.residual(v + eps * d) - st.residual(v - eps * d)) / (2 * eps)
    an = st.from_free(K @ st.to_free(d))
    err = np.linalg.norm(fd - an) / np.linalg.norm(an)
    assert err < 1e-6, err


def test_svn_operator_equals_stdn_at_consistent_pi():
    p = small_problem(N=6)
    st = Step(p)
    v = random_velocity(6, 3)
    Ks = st.svn_matrix(v, st.pi_of(v))
    Kn = st.stdn_matrix(v)
    diff = abs(Ks - Kn).max()
    assert diff <= 1e-13 * abs(Kn).max(), diff


def test_dual_step_linearises_pi():
    p = small_problem(N=6)
    st = Step(p)
    v = random_velocity(6, 4)
    d = random_velocity(6, 9, scale=1.0)
    pi = st.pi_of(v)
    eps = 1e-7
    fd = (st.pi_of(v + eps * d) - st.pi_of(v - eps * d)) / (2 * eps)
    # Eq. "tautilde" is linear in dv except the constant -pi + tau/Delta (zero here)
    an = st.dual_step(v, d, pi)
    err = np.abs(fd - an).max() / np.abs(an).max()
    assert err < 1e-6, err
    # the constant part vanishes exactly when pi = tau/Delta
    zero = st.dual_step(v, np.zeros_like(v), pi)
    assert np.abs(zero).max() <= 1e-15 * np.abs(pi).max() + 1e-300


@pytest.mark.parametrize("big", [False, True])
def test_svn_operator_symmetric_positive_definite(big):
    p = small_problem(N=6)
    st = Step(p)
    v = random_velocity(6, 5)
    rng = np.random.default_rng(13)
    pi = rng.standard_normal((6, 6, 4, 3)) * (3.0 if big else 0.2)
    K = st.svn_matrix(v, pi).toarray()
    assert np.abs(K - K.T).max() <= 1e-14 * np.abs(K).max()
    lam = np.linalg.eigvalsh(K)
    assert lam.min() > 0
    np.linalg.cholesky(K)
    # pointwise: t p^T + p t^T has top eigenvalue t.p + |t||p| <= 2 |t||p|, so
    # lambda_min(C) >= dt (P/Delta) (1 - 2 |t_tau| |t_pi| / (Delta m)) > 0 because
    # |t_tau| < Delta / sqrt2 and |t_pi| / m <= 1 / sqrt2.
    C = st.svn_coefficients(v, pi)
    t = st.mesh.tau_at_qp(st.mesh.gather(v))
    Dl = st.delta(t)
    pv = comp_to_voigt(pi)
    m = np.maximum(1.0, np.sqrt(2 * np.sum(pv * pv, -1)))
    npi = np.linalg.norm(pv, axis=-1) / m          # <= 1/sqrt2
    floor = st.dt * st.P[..., None] / Dl * (1 - 2 * npi * np.linalg.norm(t, axis=-1) / Dl)
    eig = np.linalg.eigvalsh(C)[..., 0]
    assert np.all(floor > 0)
    assert np.all(eig >= floor * (1 - 1e-9))


def test_energy_convex_along_lines():
    p = small_problem(N=8)
    st = Step(p)
    v = random_velocity(8, 6)
    d = random_velocity(8, 8)
    s = np.linspace(-2, 2, 21)
    phi = np.array([st.energy(v + a * d) for a in s])
    second = phi[:-2] - 2 * phi[1:-1] + phi[2:]
    assert np.all(second >= -1e-12 * np.abs(phi).max())


def kron_mass_solve(N, L, rhs_per_node):
    """Solve (M1 (x) M1) x = b on interior nodes, M1 = dx/6 tridiag(1, 4, 1)."""
    dx = L / N
    n = N - 1
    M1 = (dx / 6.0) * (4 * np.eye(n) + np.eye(n, k=1) + np.eye(n, k=-1))
    M = np.kron(M1, M1)
    return np.linalg.solve(M, rhs_per_node.reshape(-1)).reshape(n, n)


def test_mass_and_coriolis_closed_form():
    N, L = 8, 512e3
    c = dataclasses.replace(W.Constants(), Pstar=0.0, Co=0.0, f_c=1.46e-4)
    rng = np.random.default_rng(21)
    vn = np.zeros((N + 1, N + 1, 2))
    vn[1:-1, 1:-1] = 0.1 * rng.standard_normal((N - 1, N - 1, 2))
    wind = np.zeros((N + 1, N + 1, 2))
    wind[..., 0], wind[..., 1] = 7.0, -4.0
    p = W.Problem(N=N, L=L, const=c, h=np.full((N, N), 1.5), A=np.ones((N, N)),
                  wind=wind, ocean=np.zeros_like(wind), v_old=vn, dt=1800.0)
    res = newton(p, tol=1e-13, max_newton=3)
    v = res.v
    rhoH = c.rho_ice * 1.5
    ta = c.Ca * c.rho_a * math.hypot(7.0, -4.0) * np.array([7.0, -4.0])
    dx = L / N
    # interior Q1 basis functions integrate to dx^2
    exp = np.empty((N - 1, N - 1, 2))
    for k in range(2):
        exp[..., k] = (p.dt / rhoH) * kron_mass_solve(N, L, np.full((N - 1, N - 1), dx * dx * ta[k]))
    vi = vn[1:-1, 1:-1]
    exp[..., 0] += vi[..., 0] + p.dt * c.f_c * vi[..., 1]      # v - dt f e_r x v^n
    exp[..., 1] += vi[..., 1] - p.dt * c.f_c * vi[..., 0]
    err = np.abs(v[1:-1, 1:-1] - exp).max() / np.abs(exp).max()
    assert err < 1e-12, err
    assert res.newton_iters == 1


def test_linear_limit_one_newton_step():
    p = small_problem(N=16, delta_min=1.0, Co=0.0)
    res = newton(p, tol=1e-10)
    assert res.converged and res.newton_iters == 1, res.res_hist


def test_newton_converges_and_pi_consistent():
    p = W.config(0, N=16)
    res = newton(p, tol=1e-10)
    assert res.converged
    st = Step(p)
    # Eq. "pi": at the solution pi = tau(v)/Delta(v); the modification is inactive
    pc = st.pi_of(res.v)
    assert np.abs(res.pi - pc).max() <= 1e-6 * np.abs(pc).max()
    pv = comp_to_voigt(res.pi)
    assert np.sqrt(2 * np.sum(pv * pv, -1)).max() < 1.0
    # energy decreases monotonically along the Newton path (re-run, recording Phi)
    assert all(a > 0 for a in res.alphas)


def test_energy_decreases_each_accepted_step():
    p = W.config(0, N=16)
    res = newton(p, tol=1e-10)
    st = Step(p)
    phis = res.phi_hist
    assert len(phis) == res.newton_iters + 1
    scale = st.energy_scale(res.v)
    for a, b in zip(phis[:-1], phis[1:]):
        assert b < a or abs(b - a) <= 1e-13 * scale
    assert phis[-1] < phis[0]


def test_svn_and_stdn_reach_the_same_minimiser():
    # Phi is strictly convex (rho H > 0), so both Newton variants must stop at
    # the same velocity; svN needs fewer iterations (Section 5.2)
    p = W.config(0, N=24)
    a = newton(p, tol=1e-10, method="svn")
    b = newton(p, tol=1e-10, method="stdn", max_newton=200)
    assert a.converged and b.converged
    assert np.linalg.norm(a.v - b.v) <= 1e-7 * np.linalg.norm(a.v)
    assert a.newton_iters < b.newton_iters


def test_mass_floor_bounds_the_hessian():
    # Phi_h's Hessian is at least the rho H-weighted Q1 mass matrix, whose
    # smallest eigenvalue on the free dofs is >= rho H_min (dx/3)^2 (1-D mass
    # matrix dx/6 tridiag(1, 4, 1) with eigenvalues > dx/3; Kronecker product
    # in 2-D); the full-size GPU certificate rests on this bound
    p = W.config(0, N=12)
    st = Step(p)
    rng = np.random.default_rng(3)
    v = np.zeros((13, 13, 2))
    v[1:-1, 1:-1] = 0.05 * rng.standard_normal((11, 11, 2))
    for K in (st.stdn_matrix(v), st.svn_matrix(v, st.pi_of(v))):
        lam = np.linalg.eigvalsh(K.toarray()).min()
        floor = p.const.rho_ice * p.h.min() * (p.L / p.N) ** 2 / 9.0
        assert lam >= floor > 0, (lam, floor)
    # and it is attained up to the weights: with Pstar = Co = 0 the Hessian is
    # the mass matrix, whose smallest eigenvalue is within 1.5x of the bound
    c = dataclasses.replace(W.Constants(), Pstar=0.0, Co=0.0)
    q = W.make_problem(12, seed=1, const=c)
    q.h[:] = 1.0
    lam = np.linalg.eigvalsh(Step(q).stdn_matrix(v).toarray()).min()
    floor = c.rho_ice * (q.L / q.N) ** 2 / 9.0
    assert floor <= lam <= 1.5 * floor, (lam, floor)


@pytest.mark.parametrize("N", [4, 10, 24, 41 + 1, 66])
def test_nested_dissection_cholesky_matches_superlu(N):
    # the multifrontal Cholesky used for large grids solves the same systems as
    # SuperLU to rounding, on grids whose interior width is odd, even, and
    # below, at and above the leaf size
    from oracle.direct import NestedDissection
    from oracle.newton import superlu_solve
    p = small_problem(N=N, seed=N)
    st = Step(p)
    v = random_velocity(N, 7)
    rng = np.random.default_rng(N)
    pi = rng.standard_normal((N, N, 4, 3))            # scaled branch at most points
    K = st.svn_matrix(v, pi)
    nd = NestedDissection(N - 1, leaf=4).factor(K)
    for _ in range(2):
        b = rng.standard_normal(K.shape[0])
        x_nd, x_lu = nd.solve(b), superlu_solve(K, b)
        assert np.linalg.norm(x_nd - x_lu) <= 1e-12 * np.linalg.norm(x_lu)
        assert np.linalg.norm(K @ x_nd - b) <= 1e-13 * np.linalg.norm(b) * 1e2
    # every dof is eliminated exactly once
    own = np.concatenate([f.own for f in nd.fronts])
    assert np.array_equal(np.sort(own), np.arange(K.shape[0]))


def test_newton_count_does_not_depend_on_the_direct_solver():
    from oracle.direct import nd_solve
    from oracle.newton import superlu_solve
    p = W.config(0, N=32)
    a = newton(p, tol=1e-10, solve=superlu_solve)
    b = newton(p, tol=1e-10, solve=nd_solve)
    assert a.newton_iters == b.newton_iters
    assert np.linalg.norm(a.v - b.v) <= 1e-10 * np.linalg.norm(a.v)
