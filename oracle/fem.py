"""Q1 finite-element definitions of the implicit VP momentum step (FP64, CPU).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Discretisation (Section 5.1): structured N x N quadrilateral mesh of
(0, L)^2, Q1 velocity at the (N+1)^2 nodes, Q0 thickness H and concentration
A on cells, homogeneous Dirichlet velocity on the boundary (Section 2).  All
integrals use 2 x 2 Gauss quadrature on every cell, so the residual below is
the exact gradient of the discrete energy and the standard-Newton Jacobian is
its exact Hessian (the paper leaves the quadrature of the non-polynomial
terms open).

Notation follows Sections 2-4:
  eps(v)  = (grad v + grad v^T)/2, eps' = eps - tr(eps) I / 2
  tau(v)  = e^{-1} eps'(v) + tr(eps(v)) I / 2                  (Section 4)
  Delta   = sqrt(Delta_min^2 + 2 tau:tau)                      (Eq. "Delta")
  P       = P* H exp(-C (1 - A))                               (Eq. "ice-strength")
  tau_atm = Ca rho_a |v_a| v_a, tau_ocean = Co rho_o |v_o - v| (v_o - v)   (Eq. "force")
Symmetric 2x2 tensors are handled as Voigt vectors t(X) = (Xxx, Xyy, sqrt2 Xxy)
so that X:Y = t(X).t(Y).  Tensor-valued state (the dual variable pi) is passed
in and out as components (xx, yy, xy).

Array layouts: node fields (N+1, N+1, 2) indexed [j, i, k]; cell fields
(N, N) indexed [j, i]; quadrature fields (N, N, 4, ...) with qp q = 2*qb + qa
at local coordinates (g[qa], g[qb]), g = 1/2 -+ 1/(2 sqrt 3).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

SQRT2 = math.sqrt(2.0)
GAUSS = (0.5 - 0.5 / math.sqrt(3.0), 0.5 + 0.5 / math.sqrt(3.0))
# local corner c = 2*b + a sits at node (i + a, j + b) of cell (i, j)
CORNERS = ((0, 0), (1, 0), (0, 1), (1, 1))
QPTS = tuple((GAUSS[qa], GAUSS[qb]) for qb in (0, 1) for qa in (0, 1))


def q1_shape(xi: float, eta: float):
    """Bilinear shape functions on the unit cell and their xi/eta derivatives."""
    val = np.array([(1 - xi) * (1 - eta), xi * (1 - eta), (1 - xi) * eta, xi * eta])
    dxi = np.array([-(1 - eta), (1 - eta), -eta, eta])
    deta = np.array([-(1 - xi), -xi, (1 - xi), xi])
    return val, dxi, deta


def strain_from_grad(g):
    """eps = sym(grad u) from g[..., k, d] = d u_k / d x_d -> (xx, yy, xy)."""
    return g[..., 0, 0], g[..., 1, 1], 0.5 * (g[..., 0, 1] + g[..., 1, 0])


def tau_voigt_from_grad(g, e):
    """Voigt vector of tau(u) = e^{-1} eps'(u) + tr(eps(u)) I / 2."""
    exx, eyy, exy = strain_from_grad(g)
    tr = exx + eyy
    dxx, dyy, dxy = exx - 0.5 * tr, eyy - 0.5 * tr, exy     # eps'
    txx = dxx / e + 0.5 * tr
    tyy = dyy / e + 0.5 * tr
    txy = dxy / e
    return np.stack([txx, tyy, SQRT2 * txy], axis=-1)


def voigt_to_comp(t):
    return np.stack([t[..., 0], t[..., 1], t[..., 2] / SQRT2], axis=-1)


def comp_to_voigt(c):
    return np.stack([c[..., 0], c[..., 1], c[..., 2] * SQRT2], axis=-1)


class Q1Mesh:
    """Reference-element tables of the uniform Q1 mesh with N x N cells.

    For every quadrature point q (uniform mesh, so the same on every cell):
      Nq[q]  (2, 8): velocity at q from the 8 local dofs (dof = 2 c + k)
      Gq[q]  (2, 2, 8): Gq[q, k, d] = d u_k / d x_d at q
      Bq[q]  (3, 8): t(tau(u)) at q
      Dq[q]  (8,):   div u at q
    and the quadrature weight w = dx^2 / 4.
    """

    def __init__(self, N: int, L: float, e: float):
        self.N, self.L, self.e = N, L, e
        self.dx = L / N
        self.w = self.dx * self.dx / 4.0
        Nq = np.zeros((4, 2, 8))
        Gq = np.zeros((4, 2, 2, 8))
        for q, (xi, eta) in enumerate(QPTS):
            val, dxi, deta = q1_shape(xi, eta)
            for c in range(4):
                for k in range(2):
                    Nq[q, k, 2 * c + k] = val[c]
                    Gq[q, k, 0, 2 * c + k] = dxi[c] / self.dx
                    Gq[q, k, 1, 2 * c + k] = deta[c] / self.dx
        self.Nq, self.Gq = Nq, Gq
        # t(tau(.)) and div(.) of each local basis function, by linearity
        self.Bq = np.stack([tau_voigt_from_grad(np.moveaxis(Gq[q], -1, 0), e).T
                            for q in range(4)])                    # (4, 3, 8)
        self.Dq = Gq[:, 0, 0, :] + Gq[:, 1, 1, :]                  # (4, 8)
        n1 = N + 1
        # global dof index of every local dof of every cell, (N, N, 8)
        jj, ii = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
        dofs = np.zeros((N, N, 8), dtype=np.int64)
        for c, (a, b) in enumerate(CORNERS):
            node = (jj + b) * n1 + (ii + a)
            for k in range(2):
                dofs[..., 2 * c + k] = 2 * node + k
        self.dofs = dofs
        node_i = np.arange(n1)
        inner = (node_i >= 1) & (node_i <= N - 1)
        free_node = np.outer(inner, inner).reshape(-1)
        self.free = np.repeat(free_node, 2)                         # bool, (2 (N+1)^2,)
        self.free_idx = np.nonzero(self.free)[0]

    # -- gather / scatter -------------------------------------------------
    def gather(self, u):
        """Node field (N+1, N+1, 2) -> local dofs per cell (N, N, 8)."""
        N = self.N
        out = np.empty((N, N, 8))
        for c, (a, b) in enumerate(CORNERS):
            out[..., 2 * c:2 * c + 2] = u[b:N + b, a:N + a, :]
        return out

    def scatter(self, ue):
        """Sum local-dof contributions (N, N, 8) into a node field (N+1, N+1, 2)."""
        N = self.N
        out = np.zeros((N + 1, N + 1, 2))
        for c, (a, b) in enumerate(CORNERS):
            out[b:N + b, a:N + a, :] += ue[..., 2 * c:2 * c + 2]
        return out

    def at_qp(self, ue):
        """Values (N, N, 4, 2) at the quadrature points."""
        return np.einsum("qkd,nmd->nmqk", self.Nq, ue)

    def tau_at_qp(self, ue):
        """Voigt t(tau(u)) (N, N, 4, 3) at the quadrature points."""
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


class Step:
    """Precomputed data of one implicit step (hot-path step a1).

    P = P* H exp(-C (1 - A)) and rho_ice H on cells; the atmospheric stress
    tau_atm = Ca rho_a |v_a| v_a at the quadrature points from the
    Q1-interpolated wind; the explicit Coriolis vector
    rho_ice H f_c e_r x (v^n - v_o) at the quadrature points (Eq. "F").
    """

    def __init__(self, prob, mesh: Q1Mesh | None = None):
        c = prob.const
        self.prob, self.c, self.dt = prob, c, prob.dt
        self.mesh = mesh or Q1Mesh(prob.N, prob.L, c.e)
        m = self.mesh
        self.P = c.Pstar * prob.h * np.exp(-c.C * (1.0 - prob.A))
        self.rhoH = c.rho_ice * prob.h
        self.vn = m.zero_boundary(prob.v_old)
        self.vn_q = m.node_to_qp(self.vn)
        self.vo_q = m.node_to_qp(prob.ocean)
        va_q = m.node_to_qp(prob.wind)
        self.tau_atm = c.Ca * c.rho_a * np.linalg.norm(va_q, axis=-1)[..., None] * va_q
        d = self.vn_q - self.vo_q
        er_cross = np.stack([-d[..., 1], d[..., 0]], axis=-1)        # e_r x d
        self.cor = c.f_c * self.rhoH[..., None, None] * er_cross

    # -- pointwise quantities --------------------------------------------
    def delta(self, t):
        """Delta = sqrt(Delta_min^2 + 2 tau:tau) from Voigt tau."""
        return np.sqrt(self.c.delta_min ** 2 + 2.0 * np.sum(t * t, axis=-1))

    # -- energy (Eq. "energy") -------------------------------------------
    def energy_terms(self, v):
        """The four terms of the integrand of Phi_h at every qp, times the weight.

        (rho H |v|^2 / 2, (-rho H v^n + dt cor - dt tau_atm) . v,
         dt P/2 (Delta - tr eps), dt Co rho_o |v_o - v|^3 / 3), each (N, N, 4).
        """
        m, c, dt = self.mesh, self.c, self.dt
        ve = m.gather(v)
        vq = m.at_qp(ve)
        t = m.tau_at_qp(ve)
        tr = m.div_at_qp(ve)
        Dl = self.delta(t)
        nw = np.linalg.norm(self.vo_q - vq, axis=-1)
        rhoH = self.rhoH[..., None]
        P = self.P[..., None]
        return (m.w * 0.5 * rhoH * np.sum(vq * vq, axis=-1),
                m.w * np.sum((-rhoH[..., None] * self.vn_q + dt * (self.cor - self.tau_atm)) * vq, axis=-1),
                m.w * dt * 0.5 * P * (Dl - tr),
                m.w * dt * c.Co * c.rho_o * nw ** 3 / 3.0)

    def energy_density(self, v):
        """Per-quadrature-point integrand of Phi_h times the weight, (N, N, 4)."""
        m, c, dt = self.mesh, self.c, self.dt
        ve = m.gather(v)
        vq = m.at_qp(ve)
        t = m.tau_at_qp(ve)
        tr = m.div_at_qp(ve)
        Dl = self.delta(t)
        w = self.vo_q - vq
        nw = np.linalg.norm(w, axis=-1)
        rhoH = self.rhoH[..., None]
        P = self.P[..., None]
        dens = (0.5 * rhoH * np.sum(vq * vq, axis=-1)
                - rhoH * np.sum(self.vn_q * vq, axis=-1)
                + dt * (0.5 * P * (Dl - tr) + c.Co * c.rho_o * nw ** 3 / 3.0)
                + dt * np.sum((self.cor - self.tau_atm) * vq, axis=-1))
        return m.w * dens

    def energy(self, v):
        """Phi_h(v), exactly rounded sum of the quadrature contributions."""
        return math.fsum(self.energy_density(v).ravel())

    def energy_scale(self, v):
        """Sum over qp of |each term|: the rounding scale of Phi_h(v)."""
        return math.fsum(sum(np.abs(t) for t in self.energy_terms(v)).ravel())

    # -- residual (Eqs. "Av=F", "A", "F", "sigma") --------------------------
    def residual(self, v):
        """Assembled R(v) = A(v, .) - F(.) as a node field, boundary rows zero."""
        m, c, dt = self.mesh, self.c, self.dt
        ve = m.gather(v)
        vq = m.at_qp(ve)
        t = m.tau_at_qp(ve)
        Dl = self.delta(t)
        w = self.vo_q - vq
        nw = np.linalg.norm(w, axis=-1)[..., None]
        rhoH = self.rhoH[..., None, None]
        P = self.P[..., None]
        # vector-valued source at qp, tested against N_c e_k
        src = (rhoH * (vq - self.vn_q) - dt * c.Co * c.rho_o * nw * w
               + dt * self.cor - dt * self.tau_atm)
        re = np.einsum("qkd,nmqk->nmd", m.Nq, src)
        # viscous-plastic term (P/Delta tau(v), tau(phi)) - (P/2, tr eps(phi))
        re += dt * np.einsum("qsd,nmqs->nmd", m.Bq, (P / Dl)[..., None] * t)
        re -= dt * np.einsum("qd,nmq->nmd", m.Dq, 0.5 * np.broadcast_to(P, Dl.shape))
        return m.zero_boundary(m.scatter(m.w * re))

    def residual_norm(self, v):
        r = self.residual(v)
        return math.sqrt(math.fsum((r * r).ravel()))

    # -- linearisations ---------------------------------------------------
    def ocean_tensor(self, v):
        """-dt tau_ocean'(v) as a 2x2 tensor per qp (Eq. "standardNewton2").

        O = dt Co rho_o (|w| I + w w^T / |w|), w = v_o - v; the rank-one term
        is dropped where |w| < 1e-14 m/s (its limit is bounded but direction
        dependent; it carries weight |w| -> 0).
        """
        m, c, dt = self.mesh, self.c, self.dt
        vq = m.node_to_qp(v)
        w = self.vo_q - vq
        nw = np.linalg.norm(w, axis=-1)
        safe = np.where(nw >= 1e-14, nw, 1.0)
        ww = np.einsum("...k,...l->...kl", w, w) / safe[..., None, None]
        ww = np.where((nw >= 1e-14)[..., None, None], ww, 0.0)
        eye = np.eye(2)
        return dt * c.Co * c.rho_o * (nw[..., None, None] * eye + ww)

    def svn_coefficients(self, v, pi):
        """Voigt 3x3 coefficient C per qp of the reduced svN operator.

        From Eq. "linearSVNewton" with tau x pi replaced per Eq. "modification"
        by (tau x pi + pi x tau) / (2 max(1, sqrt(2 pi:pi))), using the paper's
        convention (X x Y) Z = (X:Z) Y:
          C = dt [ (P/Delta) I - P / (Delta^2 m) (t_tau t_pi^T + t_pi t_tau^T) ].
        """
        m, dt = self.mesh, self.dt
        t = m.tau_at_qp(m.gather(v))
        Dl = self.delta(t)
        p = comp_to_voigt(pi)
        mm = np.maximum(1.0, np.sqrt(2.0 * np.sum(p * p, axis=-1)))
        P = np.broadcast_to(self.P[..., None], Dl.shape)
        eye = np.eye(3)
        sym = np.einsum("...a,...b->...ab", t, p) + np.einsum("...a,...b->...ab", p, t)
        return dt * ((P / Dl)[..., None, None] * eye
                     - (P / (Dl * Dl * mm))[..., None, None] * sym)

    def stdn_coefficients(self, v):
        """Voigt 3x3 coefficient of the standard Newton Jacobian (Eq. "standardNewton1").

        C = dt [ (P/Delta) I - 2 P / Delta^3 t_tau t_tau^T ].
        """
        m, dt = self.mesh, self.dt
        t = m.tau_at_qp(m.gather(v))
        Dl = self.delta(t)
        P = np.broadcast_to(self.P[..., None], Dl.shape)
        eye = np.eye(3)
        return dt * ((P / Dl)[..., None, None] * eye
                     - (2.0 * P / Dl ** 3)[..., None, None]
                     * np.einsum("...a,...b->...ab", t, t))

    def element_matrices(self, Cq, Oq):
        """K_e = sum_q w (rho H Nq^T Nq + Nq^T O Nq + Bq^T C Bq), (N, N, 8, 8)."""
        m = self.mesh
        Ke = np.einsum("qka,nmqkl,qlb->nmab", m.Nq, Oq, m.Nq)
        Ke += np.einsum("qsa,nmqst,qtb->nmab", m.Bq, Cq, m.Bq)
        mass = np.einsum("qka,qkb->ab", m.Nq, m.Nq)
        Ke += self.rhoH[..., None, None] * mass
        return m.w * Ke

    def assemble(self, Ke):
        """Global sparse matrix restricted to the free dofs (CSR): the element
        entries whose row and column dofs are both free, summed."""
        m = self.mesh
        n = 2 * (m.N + 1) ** 2
        fmap = np.full(n, -1, dtype=np.int64)
        fmap[m.free_idx] = np.arange(m.free_idx.size)
        ld = fmap[m.dofs]                                           # (N, N, 8) free index or -1
        keep = (ld[..., :, None] >= 0) & (ld[..., None, :] >= 0)
        rows = np.broadcast_to(ld[..., :, None], Ke.shape)[keep]
        cols = np.broadcast_to(ld[..., None, :], Ke.shape)[keep]
        nf = m.free_idx.size
        return sp.coo_matrix((Ke[keep], (rows, cols)), shape=(nf, nf)).tocsr()

    def svn_matrix(self, v, pi):
        """Reduced svN linearisation (Eq. "linearSVNewton" + Eq. "modification")."""
        return self.assemble(self.element_matrices(self.svn_coefficients(v, pi),
                                                   self.ocean_tensor(v)))

    def stdn_matrix(self, v):
        """Standard Newton Jacobian (Eqs. "standardNewton1", "standardNewton2")."""
        return self.assemble(self.element_matrices(self.stdn_coefficients(v),
                                                   self.ocean_tensor(v)))

    # -- dual variable (Eqs. "pi", "tautilde", "modification") -------------
    def pi_of(self, v):
        """pi = tau(v) / Delta(v) at every qp, components (xx, yy, xy)."""
        t = self.mesh.tau_at_qp(self.mesh.gather(v))
        return voigt_to_comp(t / self.delta(t)[..., None])

    def dual_step(self, v, dv, pi):
        """Newton step for pi after eliminating it (Eq. "tautilde").

        pi~ = -pi + tau/Delta + tau(dv)/Delta
              - [ (tau:tau(dv)) pi + (pi:tau(dv)) tau ] / (Delta^2 m),
        m = max(1, sqrt(2 pi:pi)): the last term of Eq. "tautilde" with the
        symmetrised, scaled tensor of Eq. "modification".
        """
        m = self.mesh
        t = m.tau_at_qp(m.gather(v))
        tt = m.tau_at_qp(m.gather(dv))
        Dl = self.delta(t)[..., None]
        p = comp_to_voigt(pi)
        mm = np.maximum(1.0, np.sqrt(2.0 * np.sum(p * p, axis=-1)))[..., None]
        tdt = np.sum(t * tt, axis=-1)[..., None]
        pdt = np.sum(p * tt, axis=-1)[..., None]
        dp = -p + t / Dl + tt / Dl - (tdt * p + pdt * t) / (Dl * Dl * mm)
        return voigt_to_comp(dp)

    # -- vector helpers -----------------------------------------------------
    def to_free(self, u):
        return np.asarray(u, dtype=np.float64).reshape(-1)[self.mesh.free_idx]

    def from_free(self, x):
        out = np.zeros(2 * (self.mesh.N + 1) ** 2)
        out[self.mesh.free_idx] = x
        return out.reshape(self.mesh.N + 1, self.mesh.N + 1, 2)
