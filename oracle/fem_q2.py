"""Q2 (biquadratic) velocity elements for the implicit VP momentum step (FP64, CPU).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper's implementation allows higher-order velocity elements and shows
Problem II with quadratic elements for v on a 2 km mesh (Section 5.1 and the
Problem II discussion of Section 5.3): the same number of velocity unknowns as
Q1 on the 1 km mesh.  This module is the Q2 counterpart of ``fem.Q1Mesh``:

  * N x N cells of width dx; each cell carries the 9 Lagrange nodes of the
    tensor-product quadratic basis at local coordinates {0, 1/2, 1}^2, so the
    velocity lives on the (2N+1) x (2N+1) grid of spacing dx/2 (node (I, J) at
    (I dx/2, J dx/2)); v = 0 on the boundary nodes;
  * 1-D basis on [0, 1] with nodes 0, 1/2, 1:
        L0 = 2 (x - 1/2)(x - 1),  L1 = -4 x (x - 1),  L2 = 2 x (x - 1/2);
  * 3 x 3 Gauss quadrature per cell (points 1/2 -+ sqrt(3/5)/2 and 1/2, weights
    5/18, 8/18, 5/18 on [0, 1]): exact for the mass matrix (degree 4 in each
    variable) and applied to every term of Phi_h, R and K, so that R = grad
    Phi_h and K_stdN = grad R hold exactly as for Q1 (reading R3);
  * H and A constant per cell (the paper pairs Q2 velocity with Q1-disc H and A
    in its time-dependent runs; the momentum step here takes cell values, and
    the transport of Q1-disc fields is not built);
  * the dual variable pi at the 9 quadrature points (3 symmetric components).

``Step2`` reuses every pointwise formula of ``fem.Step`` (tau, Delta, the
energy density, the svN / stdN coefficients, the dual step) and supplies the
element integrals with per-point weights.  Layouts: node fields
(2N+1, 2N+1, 2) indexed [J, I, k]; cell fields (N, N); quadrature fields
(N, N, 9, ...) with q = 3 qb + qa.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

from .fem import Step, tau_voigt_from_grad

_G = math.sqrt(3.0 / 5.0) / 2.0
GAUSS3 = (0.5 - _G, 0.5, 0.5 + _G)
WEIGHT3 = (5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0)
QPTS2 = tuple((GAUSS3[qa], GAUSS3[qb]) for qb in range(3) for qa in range(3))
QW2 = np.array([WEIGHT3[qa] * WEIGHT3[qb] for qb in range(3) for qa in range(3)])
# local node n = 3 b + a sits at fine node (2 i + a, 2 j + b) of cell (i, j)
LOCAL2 = tuple((a, b) for b in range(3) for a in range(3))


def lagrange2(x: float):
    """Quadratic Lagrange basis on [0, 1] (nodes 0, 1/2, 1) and its derivatives."""
    val = np.array([2 * (x - 0.5) * (x - 1), -4 * x * (x - 1), 2 * x * (x - 0.5)])
    der = np.array([4 * x - 3, -8 * x + 4, 4 * x - 1])
    return val, der


class Q2Mesh:
    """Reference-element tables of the uniform Q2 mesh with N x N cells
    (the same attributes as ``fem.Q1Mesh``, with 18 local dofs and 9 points)."""

    def __init__(self, N: int, L: float, e: float):
        self.N, self.L, self.e = N, L, e
        self.dx = L / N
        self.n1 = 2 * N + 1                       # nodes per side
        self.w = self.dx * self.dx * QW2          # per-point weights, (9,)
        nq = len(QPTS2)
        Nq = np.zeros((nq, 2, 18))
        Gq = np.zeros((nq, 2, 2, 18))
        for q, (xi, eta) in enumerate(QPTS2):
            lx, dlx = lagrange2(xi)
            ly, dly = lagrange2(eta)
            for n, (a, b) in enumerate(LOCAL2):
                for k in range(2):
                    Nq[q, k, 2 * n + k] = lx[a] * ly[b]
                    Gq[q, k, 0, 2 * n + k] = dlx[a] * ly[b] / self.dx
                    Gq[q, k, 1, 2 * n + k] = lx[a] * dly[b] / self.dx
        self.Nq, self.Gq = Nq, Gq
        self.Bq = np.stack([tau_voigt_from_grad(np.moveaxis(Gq[q], -1, 0), e).T for q in range(nq)])
        self.Dq = Gq[:, 0, 0, :] + Gq[:, 1, 1, :]
        n1 = self.n1
        jj, ii = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
        dofs = np.zeros((N, N, 18), dtype=np.int64)
        for n, (a, b) in enumerate(LOCAL2):
            node = (2 * jj + b) * n1 + (2 * ii + a)
            for k in range(2):
                dofs[..., 2 * n + k] = 2 * node + k
        self.dofs = dofs
        idx = np.arange(n1)
        inner = (idx >= 1) & (idx <= n1 - 2)
        self.free = np.repeat(np.outer(inner, inner).reshape(-1), 2)
        self.free_idx = np.nonzero(self.free)[0]

    def gather(self, u):
        """Node field (2N+1, 2N+1, 2) -> local dofs per cell (N, N, 18)."""
        N = self.N
        out = np.empty((N, N, 18))
        for n, (a, b) in enumerate(LOCAL2):
            out[..., 2 * n:2 * n + 2] = u[b:2 * N + b:2, a:2 * N + a:2, :]
        return out

    def scatter(self, ue):
        """Sum local-dof contributions (N, N, 18) into a node field."""
        N = self.N
        out = np.zeros((self.n1, self.n1, 2))
        for n, (a, b) in enumerate(LOCAL2):
            out[b:2 * N + b:2, a:2 * N + a:2, :] += ue[..., 2 * n:2 * n + 2]
        return out

    def at_qp(self, ue):
        return np.einsum("qkd,nmd->nmqk", self.Nq, ue)

    def tau_at_qp(self, ue):
        return np.einsum("qsd,nmd->nmqs", self.Bq, ue)

    def div_at_qp(self, ue):
        return np.einsum("qd,nmd->nmq", self.Dq, ue)

    def node_to_qp(self, u):
        return self.at_qp(self.gather(u))

    def zero_boundary(self, u):
        u = np.array(u, dtype=np.float64, copy=True)
        u[0, :, :] = 0.0
        u[-1, :, :] = 0.0
        u[:, 0, :] = 0.0
        u[:, -1, :] = 0.0
        return u


class Step2(Step):
    """One implicit step on Q2 velocity elements (see the module docstring)."""

    @staticmethod
    def direct_solver(K, b):
        # Q2 couples nodes two apart, so the Q1 nested dissection does not apply
        from .newton import superlu_solve
        return superlu_solve(K, b)

    def __init__(self, prob):
        super().__init__(prob, mesh=Q2Mesh(prob.N, prob.L, prob.const.e))

    def residual(self, v):
        """Assembled R(v) = A(v, .) - F(.) on the Q2 nodes, boundary rows zero."""
        m, c, dt = self.mesh, self.c, self.dt
        ve = m.gather(v)
        vq = m.at_qp(ve)
        t = m.tau_at_qp(ve)
        Dl = self.delta(t)
        w = self.vo_q - vq
        nw = np.linalg.norm(w, axis=-1)[..., None]
        rhoH = self.rhoH[..., None, None]
        P = self.P[..., None]
        W = m.w
        src = (rhoH * (vq - self.vn_q) - dt * c.Co * c.rho_o * nw * w + dt * self.cor - dt * self.tau_atm)
        re = np.einsum("qkd,nmqk->nmd", m.Nq, src * W[:, None])
        re += dt * np.einsum("qsd,nmqs->nmd", m.Bq, (P / Dl * W)[..., None] * t)
        re -= dt * np.einsum("qd,nmq->nmd", m.Dq, 0.5 * np.broadcast_to(P, Dl.shape) * W)
        return m.zero_boundary(m.scatter(re))

    def element_matrices(self, Cq, Oq):
        """K_e = sum_q w_q (rho H Nq^T Nq + Nq^T O Nq + Bq^T C Bq), (N, N, 18, 18)."""
        m = self.mesh
        W = m.w
        Ke = np.einsum("qka,nmqkl,qlb->nmab", m.Nq, Oq * W[:, None, None], m.Nq)
        Ke += np.einsum("qsa,nmqst,qtb->nmab", m.Bq, Cq * W[:, None, None], m.Bq)
        mass = np.einsum("q,qka,qkb->ab", W, m.Nq, m.Nq)
        Ke += self.rhoH[..., None, None] * mass
        return Ke

    def assemble(self, Ke):
        """Global sparse matrix on the free Q2 dofs (CSR)."""
        m = self.mesh
        n = 2 * m.n1 ** 2
        fmap = np.full(n, -1, dtype=np.int64)
        fmap[m.free_idx] = np.arange(m.free_idx.size)
        ld = fmap[m.dofs]
        keep = (ld[..., :, None] >= 0) & (ld[..., None, :] >= 0)
        rows = np.broadcast_to(ld[..., :, None], Ke.shape)[keep]
        cols = np.broadcast_to(ld[..., None, :], Ke.shape)[keep]
        nf = m.free_idx.size
        return sp.coo_matrix((Ke[keep], (rows, cols)), shape=(nf, nf)).tocsr()

    def from_free(self, x):
        out = np.zeros(2 * self.mesh.n1 ** 2)
        out[self.mesh.free_idx] = x
        return out.reshape(self.mesh.n1, self.mesh.n1, 2)
