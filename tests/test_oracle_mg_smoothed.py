"""Pins of the oracle's smoothed prolongator P_s = (I - omega D^-1 A) P
(smoothed aggregation: Vanek, Mandel, Brezina, Computing 56, 1996) applied to
the bilinear prolongation, and of the coarse operators it gives (no GPU).

  * closed form: for the separable operator A = (K1 x K1) x I2 with K1 the 1-D
    second-difference matrix tridiag(-1, 2, -1), D^-1 = I/4 and every column
    of A P is (K1 p) x (K1 p) with p = (1/2, 1, 1/2), so away from the
    boundary the column of coarse node (I, J) is
        P_s[2I + a, 2J + b] = p(a) p(b) - (omega / 4) u(a) u(b),
    u = K1 p = (-1/2, 0, 1, 0, -1/2) on offsets -2..2 -- a flipped sign or a
    missing D^-1 fails it;
  * width: with a 9-point fine operator, P^T A P couples coarse nodes at most
    one apart (3 x 3 blocks) and P_s^T A P_s at most two apart (5 x 5
    blocks): the supports of P columns (+-1 fine node) and of P_s columns
    (+-2) fix this;
  * effect: on svN linearisations at Newton iterates of the synthetic recipe
    (64^2), one smoothed level cuts the FGMRES iterations of the V-cycle
    preconditioner (degree-6 Chebyshev) by at least 15 %.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import mg
from oracle.fem import Step
from oracle.newton import newton

P1 = {-1: 0.5, 0: 1.0, 1: 0.5}
U1 = {-2: -0.5, -1: 0.0, 0: 1.0, 1: 0.0, 2: -0.5}


def separable_operator(N):
    n = N - 1
    K1 = sp.diags([-np.ones(n - 1), 2.0 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1])
    return sp.kron(sp.kron(K1, K1), sp.identity(2)).tocsr()


def closed_form_mismatch(smooth, N=16, omega=0.3):
    A = separable_operator(N)
    Dinv = mg.block_diag_inverse(A)
    Ps = smooth(A, Dinv, mg.prolongation(N // 2), omega)
    Ps = Ps.toarray()
    fi, ci = mg.interior_index(N), mg.interior_index(N // 2)
    worst = 0.0
    for J in range(2, N // 2 - 1):
        for I in range(2, N // 2 - 1):
            for k in range(2):
                col = Ps[:, 2 * ci[J, I] + k]
                exp = np.zeros_like(col)
                for db in range(-2, 3):
                    for da in range(-2, 3):
                        val = P1.get(da, 0.0) * P1.get(db, 0.0) - 0.25 * omega * U1[da] * U1[db]
                        exp[2 * fi[2 * J + db, 2 * I + da] + k] = val
                worst = max(worst, float(np.abs(col - exp).max()))
    return worst


def test_smoothed_prolongation_closed_form():
    assert closed_form_mismatch(mg.smoothed_prolongation) < 1e-14
    assert closed_form_mismatch(mg.smoothed_prolongation, omega=mg.sa_omega(3.7)) < 1e-14


@pytest.mark.parametrize("wrong", [
    lambda A, Dinv, P, w: (P + w * (Dinv @ (A @ P))).tocsr(),        # sign flipped
    lambda A, Dinv, P, w: (P - w * (A @ P)).tocsr(),                  # D^-1 dropped
    lambda A, Dinv, P, w: (P - w * (Dinv @ (A @ (A @ P)))).tocsr(),   # A applied twice
])
def test_planted_mistakes_fail_the_closed_form(wrong):
    assert closed_form_mismatch(wrong) > 1e-3


def block_reach(Ac, Nc):
    """Largest |dI|, |dJ| between coupled coarse nodes."""
    ci = mg.interior_index(Nc)
    node_ij = {}
    for j in range(1, Nc):
        for i in range(1, Nc):
            node_ij[ci[j, i]] = (i, j)
    C = sp.coo_matrix(Ac)
    di = dj = 0
    for r, c in zip(C.row, C.col):
        (i0, j0), (i1, j1) = node_ij[r // 2], node_ij[c // 2]
        di, dj = max(di, abs(i0 - i1)), max(dj, abs(j0 - j1))
    return di, dj


def svn_linearisation(N, newton_iters):
    p = W.config(2, N=N)
    st = Step(p)
    r = newton(p, tol=1e-12, max_newton=newton_iters)
    K = st.svn_matrix(r.v, r.pi)
    b = -st.to_free(st.residual(r.v))
    return K, b


def test_smoothed_coarse_operator_is_a_5x5_block_stencil():
    N = 32
    K, _ = svn_linearisation(N, 3)
    plain = mg.build_hierarchy(K, N, coarse_N=8, power_iters=15)
    smooth = mg.build_hierarchy(K, N, coarse_N=8, power_iters=15, smooth_levels=1)
    assert block_reach(plain[1].A, N // 2) == (1, 1)
    assert block_reach(smooth[1].A, N // 2) == (2, 2)
    # the coarse operator stays symmetric positive definite
    Ac = smooth[1].A
    assert abs(Ac - Ac.T).max() <= 1e-12 * abs(Ac).max()
    assert np.linalg.eigvalsh(Ac.toarray()).min() > 0


@pytest.mark.parametrize("newton_iters", [5, 10])
def test_smoothed_prolongator_cuts_fgmres_iterations(newton_iters):
    N = 64
    K, b = svn_linearisation(N, newton_iters)
    its = {}
    for sl in (0, 1):
        levels = mg.build_hierarchy(K, N, coarse_N=4, power_iters=15, smooth_levels=sl)
        _, its[sl], _ = mg.fgmres(K, b, M=lambda x: mg.vcycle(levels, x, degree=6, lo=0.02), rtol=1e-5,
                                  restart=100)
    assert its[1] <= 0.85 * its[0], its
