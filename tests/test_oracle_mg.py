"""Pins of the oracle's multigrid / Krylov pieces against closed forms,
library routines and invariants (no GPU).

  * P is bilinear interpolation: equals scipy's RegularGridInterpolator
  * Galerkin: for constant coefficients, P^T K_fine P equals the operator
    assembled directly on the coarse mesh (nested Q1 spaces, exact 2x2 Gauss)
  * Chebyshev on a diagonal matrix damps eigenvalue lambda by the closed form
    T_k((theta - lambda)/delta) / T_k(theta/delta)
  * the Gershgorin number bounds the spectrum of D^-1 A
  * the V-cycle with equal pre/post Chebyshev polynomials is symmetric
  * FGMRES: exact preconditioner -> 1 iteration; k distinct eigenvalues ->
    at most k iterations; solution agrees with a sparse direct solve.
"""
import dataclasses

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from scipy.interpolate import RegularGridInterpolator

import workloads as W
from oracle import mg
from oracle.fem import Step


def test_prolongation_is_bilinear_interpolation():
    Nc, L = 6, 1.0
    rng = np.random.default_rng(0)
    uc = np.zeros((Nc + 1, Nc + 1, 2))
    uc[1:-1, 1:-1] = rng.standard_normal((Nc - 1, Nc - 1, 2))
    P = mg.prolongation(Nc)
    xc = np.linspace(0, L, Nc + 1)
    xf = np.linspace(0, L, 2 * Nc + 1)
    Yf, Xf = np.meshgrid(xf, xf, indexing="ij")
    pts = np.stack([Yf.ravel(), Xf.ravel()], -1)
    uf = np.empty((2 * Nc + 1, 2 * Nc + 1, 2))
    for k in range(2):
        f = RegularGridInterpolator((xc, xc), uc[..., k], method="linear")
        uf[..., k] = f(pts).reshape(2 * Nc + 1, 2 * Nc + 1)
    got = P @ uc[1:-1, 1:-1].reshape(-1)
    exp = uf[1:-1, 1:-1].reshape(-1)
    assert np.abs(got - exp).max() < 1e-14


def constant_problem(N):
    c = dataclasses.replace(W.Constants(), f_c=0.0)
    z = np.zeros((N + 1, N + 1, 2))
    return W.Problem(N=N, L=512e3, const=c, h=np.full((N, N), 1.3), A=np.full((N, N), 0.97),
                     wind=z, ocean=z.copy(), v_old=z.copy(), dt=1800.0)


def test_galerkin_equals_coarse_assembly_constant_coefficients():
    Nc = 4
    sf, sc = Step(constant_problem(2 * Nc)), Step(constant_problem(Nc))
    vf = np.zeros((2 * Nc + 1, 2 * Nc + 1, 2))
    vc = np.zeros((Nc + 1, Nc + 1, 2))
    Kf = sf.svn_matrix(vf, np.zeros((2 * Nc, 2 * Nc, 4, 3)))
    Kc = sc.svn_matrix(vc, np.zeros((Nc, Nc, 4, 3)))
    G = mg.galerkin(Kf, mg.prolongation(Nc))
    assert abs(G - Kc).max() <= 1e-12 * abs(Kc).max()


def test_chebyshev_closed_form():
    lam = np.linspace(0.05, 1.0, 40)
    A = sp.diags(lam).tocsr()
    Dinv = sp.identity(40, format="csr")
    e0 = np.ones(40)
    lmax, lo, k = 1.0, 0.1, 4
    # solving A x = 0 from x0 = e0: the error is x itself
    x = mg.chebyshev(A, Dinv, np.zeros(40), e0.copy(), k, lmax, lo)
    a, b = lo * lmax, lmax
    th, de = (a + b) / 2, (b - a) / 2

    def T(n, s):
        s = np.asarray(s, dtype=float)
        return np.where(np.abs(s) <= 1, np.cos(n * np.arccos(np.clip(s, -1, 1))),
                        np.cosh(n * np.arccosh(np.maximum(np.abs(s), 1))) * np.sign(s) ** n)

    exp = T(k, (th - lam) / de) / T(k, th / de)
    assert np.abs(x - exp).max() < 1e-13


def svn_operator(N=16, seed=4):
    p = W.config(0, N=N)
    st = Step(p)
    rng = np.random.default_rng(seed)
    v = np.zeros((N + 1, N + 1, 2))
    v[1:-1, 1:-1] = 0.05 * rng.standard_normal((N - 1, N - 1, 2))
    return st, st.svn_matrix(v, st.pi_of(v))


def test_gershgorin_bounds_spectrum():
    _, K = svn_operator()
    Dinv = mg.block_diag_inverse(K)
    n = K.shape[0] // 2
    mask = sp.bsr_matrix((np.ones((n, 2, 2)), np.arange(n), np.arange(n + 1)), shape=K.shape)
    assert abs(Dinv @ K - sp.identity(K.shape[0])).multiply(mask).max() < 1e-9
    lmax = mg.gershgorin_lmax(K, Dinv)
    ev = np.linalg.eigvals((Dinv @ K).toarray())
    assert ev.real.max() <= lmax * (1 + 1e-12)


def test_vcycle_symmetric_and_effective():
    st, K = svn_operator(N=32)
    levels = mg.build_hierarchy(K, 32, coarse_N=8)
    assert len(levels) == 3
    rng = np.random.default_rng(1)
    y, z = rng.standard_normal(K.shape[0]), rng.standard_normal(K.shape[0])
    My, Mz = mg.vcycle(levels, y), mg.vcycle(levels, z)
    assert abs(z @ My - y @ Mz) <= 1e-12 * np.linalg.norm(My) * np.linalg.norm(z)
    b = rng.standard_normal(K.shape[0])
    _, it_pc, _ = mg.fgmres(K, b, M=lambda r: mg.vcycle(levels, r), rtol=1e-8)
    _, it_j, _ = mg.fgmres(K, b, M=levels[0].Dinv, rtol=1e-8, maxit=2000)
    assert it_pc < it_j / 3, (it_pc, it_j)


def test_fgmres_textbook_properties():
    rng = np.random.default_rng(3)
    n = 60
    vals = np.repeat([1.0, 2.0, 5.0, 9.0], n // 4)
    A = sp.diags(vals).tocsr()
    b = rng.standard_normal(n)
    x, it, _ = mg.fgmres(A, b, rtol=1e-12)
    assert it <= 4
    assert np.abs(x - b / vals).max() < 1e-10
    st, K = svn_operator(N=12)
    b = rng.standard_normal(K.shape[0])
    lu = spla.splu(K.tocsc())
    x, it, _ = mg.fgmres(K, b, M=lu.solve, rtol=1e-10)
    assert it == 1
    x, it, est = mg.fgmres(K, b, M=mg.block_diag_inverse(K), rtol=1e-9, restart=20, maxit=3000)
    xe = lu.solve(b)
    assert np.linalg.norm(b - K @ x) <= 1.01e-9 * np.linalg.norm(b)
    assert it > 20          # went through at least one restart



def test_power_lmax_converges_to_eigs():
    import scipy.sparse.linalg as spla2
    st, K = svn_operator(N=16)
    Dinv = mg.block_diag_inverse(K)
    true = spla2.eigs((Dinv @ K).tocsr(), k=1, which="LR", return_eigenvectors=False, tol=1e-10).real.max()
    assert abs(mg.power_lmax(K, Dinv, 16, iters=100, safety=1.0) / true - 1) < 1e-3
    est = mg.power_lmax(K, Dinv, 16, iters=15, safety=1.0)
    assert 0.8 * true <= est <= 1.01 * true
