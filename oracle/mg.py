"""Multigrid-preconditioned FGMRES pieces, textbook forms (FP64, CPU).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper solves each Newton linearisation with FGMRES preconditioned by
algebraic multigrid with 3 smoothing steps and a direct coarsest-level solve
(Section 5.4).  The fast path keeps FGMRES and the V-cycle structure but uses
the structured grid's geometric hierarchy; this module states each piece in
its plain form so the CUDA kernels can be compared against it:

  * prolongation P: bilinear interpolation from N/2 to N cells on interior
    (free) nodes, per velocity component; restriction is P^T;
  * Galerkin coarse operator A_c = P^T A P;
  * 2x2 block-Jacobi D (one block per node) and the Gershgorin bound
    lambda_max(D^-1 A) <= max_i sum_j |(D^-1 A)_ij|;
  * Chebyshev iteration on [lo * lmax, lmax] (Saad, "Iterative Methods for
    Sparse Linear Systems", 2nd ed., Alg. 12.1);
  * V-cycle: pre-smooth, restrict the residual, recurse, prolong, post-smooth,
    dense Cholesky on the coarsest level;
  * FGMRES with right preconditioning (Saad, Alg. 9.6), modified Gram-Schmidt
    and Givens rotations;
  * optionally, on the finest levels, the smoothed prolongator of smoothed
    aggregation (Vanek, Mandel, Brezina, "Algebraic multigrid by smoothed
    aggregation for second and fourth order elliptic problems", Computing 56,
    1996): P_s = (I - omega D^-1 A) P with omega = 4 / (3 lambda_max(D^-1 A)),
    here applied to the bilinear P; the Galerkin operator P_s^T A P_s then
    couples each coarse node to its 5 x 5 block neighbourhood.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp


def interior_index(N):
    """Map interior node (i, j), 1 <= i, j <= N-1, to its free-node number."""
    idx = -np.ones((N + 1, N + 1), dtype=np.int64)
    n = N - 1
    idx[1:N, 1:N] = np.arange(n * n).reshape(n, n)
    return idx


def prolongation(Nc):
    """Bilinear prolongation from Nc to 2 Nc cells on free dofs (2 per node)."""
    Nf = 2 * Nc
    fi, ci = interior_index(Nf), interior_index(Nc)
    rows, cols, vals = [], [], []

    def w1(i):
        return [(i // 2, 1.0)] if i % 2 == 0 else [((i - 1) // 2, 0.5), ((i + 1) // 2, 0.5)]

    for j in range(1, Nf):
        for i in range(1, Nf):
            for (I, wi) in w1(i):
                for (J, wj) in w1(j):
                    if ci[J, I] < 0:
                        continue
                    for k in range(2):
                        rows.append(2 * fi[j, i] + k)
                        cols.append(2 * ci[J, I] + k)
                        vals.append(wi * wj)
    nf, nc = 2 * (Nf - 1) ** 2, 2 * (Nc - 1) ** 2
    return sp.csr_matrix((vals, (rows, cols)), shape=(nf, nc))


def galerkin(A, P):
    """Coarse operator P^T A P."""
    return (P.T @ A @ P).tocsr()


def block_diag_inverse(A):
    """Inverse of the 2x2 node blocks of A, as a block-diagonal sparse matrix."""
    A = A.tocsr()
    n = A.shape[0] // 2
    d = A.diagonal()
    off = np.asarray(A[np.arange(0, 2 * n, 2), np.arange(1, 2 * n, 2)]).ravel()
    off2 = np.asarray(A[np.arange(1, 2 * n, 2), np.arange(0, 2 * n, 2)]).ravel()
    a, b, c, e = d[0::2], off, off2, d[1::2]
    det = a * e - b * c
    blocks = np.stack([np.stack([e, -b], -1), np.stack([-c, a], -1)], -2) / det[:, None, None]
    return sp.bsr_matrix((blocks, np.arange(n), np.arange(n + 1)),
                         shape=(2 * n, 2 * n)).tocsr()


def gershgorin_lmax(A, Dinv):
    """Upper bound of the spectrum of D^-1 A: its largest absolute row sum."""
    M = abs(Dinv @ A)
    return float(np.asarray(M.sum(axis=1)).max())


def checkerboard(N):
    """Deterministic start vector on the interior nodes of the N-cell grid:
    x[i, j] = ((-1)^(i+j), -(-1)^(i+j)) (high-frequency in both components)."""
    jj, ii = np.meshgrid(np.arange(1, N), np.arange(1, N), indexing="ij")
    s = (-1.0) ** (ii + jj)
    return np.stack([s, -s], -1).reshape(-1)


def power_lmax(A, Dinv, N, iters=15, safety=1.15):
    """Estimate of lambda_max(D^-1 A) by ``iters`` steps of the power method
    from the checkerboard vector: safety * |x_k| / |x_{k-1}| (no
    normalisation between steps)."""
    x = checkerboard(N)
    prev = x
    for _ in range(iters):
        prev, x = x, Dinv @ (A @ x)
    return safety * np.linalg.norm(x) / np.linalg.norm(prev)


def chebyshev(A, Dinv, b, x, degree, lmax, lo=0.1):
    """``degree`` steps of Chebyshev iteration for D^-1 A on [lo lmax, lmax].

    Saad Alg. 12.1 applied to the preconditioned system: theta, delta are the
    centre and half-width of the interval, sigma = theta/delta.
    """
    alpha, beta = lo * lmax, lmax
    theta, delta = 0.5 * (beta + alpha), 0.5 * (beta - alpha)
    sigma = theta / delta
    rho = 1.0 / sigma
    r = b - A @ x
    d = (Dinv @ r) / theta
    x = x + d
    for _ in range(degree - 1):
        r = r - A @ d
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * (Dinv @ r)
        rho = rho_new
        x = x + d
    return x


def sa_omega(lmax):
    """Damping of the prolongator smoother: 4 / (3 lambda_max(D^-1 A)), the
    choice of Vanek, Mandel and Brezina (1996)."""
    return 4.0 / (3.0 * lmax)


def smoothed_prolongation(A, Dinv, P, omega):
    """P_s = (I - omega D^-1 A) P: one damped block-Jacobi step applied to every
    column of P."""
    return (P - omega * (Dinv @ (A @ P))).tocsr()


@dataclasses.dataclass
class Level:
    A: sp.csr_matrix
    Dinv: sp.csr_matrix | None = None
    lmax: float = 0.0
    P: sp.csr_matrix | None = None        # from the next-coarser level to this one
    chol: object = None


def build_hierarchy(A0, N, coarse_N=8, lo=0.1, power_iters=0, safety=1.15, smooth_levels=0):
    """Galerkin hierarchy N, N/2, ... down to ``coarse_N`` cells.

    lambda_max(D^-1 A) per level: the Gershgorin bound (power_iters = 0) or
    the power-method estimate ``power_lmax``.  The prolongators into the
    ``smooth_levels`` finest levels are the smoothed ones of
    ``smoothed_prolongation`` (omega from ``sa_omega`` of that level's
    lambda_max estimate); the coarse operators stay Galerkin, P^T A P."""

    def estimate(lv, n):
        lv.Dinv = block_diag_inverse(lv.A)
        if power_iters > 0:
            lv.lmax = power_lmax(lv.A, lv.Dinv, n, power_iters, safety)
        else:
            lv.lmax = gershgorin_lmax(lv.A, lv.Dinv)

    levels = [Level(A0.tocsr())]
    n = N
    while n > coarse_N and n % 2 == 0:
        lv = levels[-1]
        estimate(lv, n)
        P = prolongation(n // 2)
        if len(levels) <= smooth_levels:
            P = smoothed_prolongation(lv.A, lv.Dinv, P, sa_omega(lv.lmax))
        lv.P = P
        levels.append(Level(galerkin(lv.A, P)))
        n //= 2
    levels[-1].chol = sla.cho_factor(levels[-1].A.toarray(), lower=True)
    return levels


def vcycle(levels, b, degree=3, lo=0.1, l=0):
    """One V-cycle z = M^-1 b with zero initial guess."""
    lv = levels[l]
    if l == len(levels) - 1:
        return sla.cho_solve(lv.chol, b)
    x = chebyshev(lv.A, lv.Dinv, b, np.zeros_like(b), degree, lv.lmax, lo)
    r = b - lv.A @ x
    xc = vcycle(levels, lv.P.T @ r, degree, lo, l + 1)
    x = x + lv.P @ xc
    return chebyshev(lv.A, lv.Dinv, b, x, degree, lv.lmax, lo)


def fgmres(A, b, M=None, rtol=1e-6, restart=100, maxit=1000, x0=None):
    """Right-preconditioned flexible GMRES (Saad Alg. 9.6).

    ``A`` and ``M`` are callables (or matrices); stops when the Givens
    residual estimate is <= rtol ||b||.  Returns (x, iterations, estimate).
    """
    Aop = A if callable(A) else (lambda v: A @ v)
    Mop = (lambda v: v) if M is None else (M if callable(M) else (lambda v: M @ v))
    n = b.shape[0]
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0, 0.0
    its = 0
    while True:
        r = b - Aop(x)
        beta = np.linalg.norm(r)
        if beta <= rtol * bnorm or its >= maxit:
            return x, its, beta
        V = [r / beta]
        Z = []
        H = np.zeros((restart + 1, restart))
        cs, sn = np.zeros(restart), np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        j_done = 0
        for j in range(restart):
            z = Mop(V[j])
            Z.append(z)
            w = Aop(z)
            for i in range(j + 1):
                H[i, j] = np.dot(w, V[i])
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            V.append(w / H[j + 1, j] if H[j + 1, j] != 0 else w)
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = math.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            j_done = j + 1
            if abs(g[j + 1]) <= rtol * bnorm or its >= maxit:
                break
        y = sla.solve_triangular(H[:j_done, :j_done], g[:j_done])
        x = x + np.column_stack(Z) @ y
        if abs(g[j_done]) <= rtol * bnorm or its >= maxit:
            return x, its, abs(g[j_done])
