"""Nested-dissection multifrontal Cholesky for the free-dof systems (FP64, CPU).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper solves each Newton linearisation directly (MUMPS) in its
iteration-count studies (Section 5.1).  SuperLU is enough up to a few hundred
thousand dofs; for the 2049^2-node workload (8.4M dofs) this module factors
the symmetric positive definite svN operator with a textbook multifrontal
Cholesky on a geometric nested-dissection ordering (George's nested
dissection of a grid graph; multifrontal assembly as in Duff & Reid and
Liu, "The multifrontal method for sparse matrix solution", SIAM Review 1992).

Grid and dofs: the free dofs belong to the m x m interior nodes (m = N - 1);
dof 2 (j m + i) + k is component k of interior node (i, j), which is the
order of ``Q1Mesh.free_idx``.  A Q1 operator couples a node to its eight
neighbours, so one line of nodes separates a rectangle into two.

Ordering: a rectangle of nodes is split by its middle column (or row, for
the longer side) into two halves and the separating line; the halves are
split recursively down to leaves of at most ``leaf`` x ``leaf`` nodes.  The
elimination tree is the tree of these splits: a leaf eliminates all of its
nodes, an inner node its separating line, after both halves.

Factorisation of one tree node with region R, eliminated set O (its line or
the whole leaf) and update set U = the nodes around R (they lie on the
separators of its ancestors, so they are eliminated later):

    F = [A_OO  A_OU]  +  sum over children c of  extend(U_c)
        [A_UO    0 ]
    L_OO = chol(F_OO),  L_UO = F_UO L_OO^-T,  U_R = F_UU - L_UO L_UO^T,

where A holds the operator's entries coupling O to O and U (entries coupling
O to R's interior were assembled at the fronts that eliminated it) and
extend(U_c) adds a child's update matrix into the rows and columns of F that
carry the same dofs.  The solve runs L y = b over the tree in elimination
order and L^T x = y in reverse.
"""
from __future__ import annotations

import dataclasses

import contextlib

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

try:                                   # optional: BLAS threads only for the large fronts
    from threadpoolctl import threadpool_limits
except ImportError:                    # pragma: no cover - then BLAS keeps its own setting
    threadpool_limits = None

# fronts with fewer rows than this run their dense kernels on one BLAS thread
# (thread start-up dominates small matrices); larger ones use all of them
BIG_FRONT = 1500


@dataclasses.dataclass
class Front:
    own: np.ndarray          # dofs eliminated here (sorted)
    upd: np.ndarray          # dofs of the update set (sorted)
    children: list           # indices of child fronts
    L_oo: np.ndarray | None = None
    L_uo: np.ndarray | None = None


def _dofs(i0, i1, j0, j1, m):
    """Dofs of the interior nodes i0 <= i < i1, j0 <= j < j1 (clipped), sorted."""
    i0, j0 = max(i0, 0), max(j0, 0)
    i1, j1 = min(i1, m), min(j1, m)
    if i0 >= i1 or j0 >= j1:
        return np.zeros(0, dtype=np.int64)
    jj, ii = np.meshgrid(np.arange(j0, j1), np.arange(i0, i1), indexing="ij")
    node = (jj * m + ii).ravel()
    return np.sort(np.concatenate([2 * node, 2 * node + 1]))


def _halo(i0, i1, j0, j1, m):
    """Dofs of the nodes around the rectangle (its eight-neighbour ring), sorted."""
    parts = [_dofs(i0 - 1, i1 + 1, j0 - 1, j0, m), _dofs(i0 - 1, i1 + 1, j1, j1 + 1, m),
             _dofs(i0 - 1, i0, j0, j1, m), _dofs(i1, i1 + 1, j0, j1, m)]
    return np.sort(np.concatenate(parts))


class NestedDissection:
    """Elimination tree of the m x m interior-node grid (fronts in postorder)."""

    def __init__(self, m: int, leaf: int = 8):
        self.m, self.n = m, 2 * m * m
        self.fronts: list[Front] = []
        self._build(0, m, 0, m, leaf)

    def _build(self, i0, i1, j0, j1, leaf):
        w, h = i1 - i0, j1 - j0
        if w <= 0 or h <= 0:
            return None
        if w <= leaf and h <= leaf:
            kids, own = [], _dofs(i0, i1, j0, j1, self.m)
        elif w >= h:
            c = (i0 + i1) // 2
            kids = [self._build(i0, c, j0, j1, leaf), self._build(c + 1, i1, j0, j1, leaf)]
            own = _dofs(c, c + 1, j0, j1, self.m)
        else:
            c = (j0 + j1) // 2
            kids = [self._build(i0, i1, j0, c, leaf), self._build(i0, i1, c + 1, j1, leaf)]
            own = _dofs(i0, i1, c, c + 1, self.m)
        self.fronts.append(Front(own=own, upd=_halo(i0, i1, j0, j1, self.m),
                                 children=[k for k in kids if k is not None]))
        return len(self.fronts) - 1

    # -- numeric ------------------------------------------------------------
    def factor(self, K: sp.spmatrix) -> "NestedDissection":
        """Cholesky factor of the SPD matrix K (n x n, the free-dof operator)."""
        K = sp.csr_matrix(K)
        if K.shape != (self.n, self.n):
            raise ValueError("matrix is %s, grid needs %d dofs" % (K.shape, self.n))
        # one line of nodes separates only if no entry couples nodes further apart
        # than the eight neighbours (true for Q1, not for Q2 elements)
        rn = np.repeat(np.arange(self.n), np.diff(K.indptr)) // 2
        cn = K.indices // 2
        if np.any(np.abs(rn % self.m - cn % self.m) > 1) or np.any(np.abs(rn // self.m - cn // self.m) > 1):
            raise ValueError("the matrix couples nodes beyond the eight-neighbour stencil")
        pos = np.full(self.n, -1, dtype=np.int64)
        updates: dict[int, np.ndarray] = {}
        # a front is "big" if it or any front below it is; the small subtrees
        # go first (postorder within them), then the big fronts in postorder
        big = []
        for f in self.fronts:
            big.append(f.own.size + f.upd.size >= BIG_FRONT or any(big[c] for c in f.children))
        small = threadpool_limits(1, user_api="blas") if threadpool_limits else contextlib.nullcontext()
        with small:
            for f_id, f in enumerate(self.fronts):
                if not big[f_id]:
                    self._front(K, f_id, f, pos, updates)
        for f_id, f in enumerate(self.fronts):
            if big[f_id]:
                self._front(K, f_id, f, pos, updates)
        return self

    def _front(self, K, f_id, f, pos, updates):
        """Assemble, factor and form the update matrix of one front."""
        nO = f.own.size
        idx = np.concatenate([f.own, f.upd])
        pos[idx] = np.arange(idx.size)
        F = np.zeros((idx.size, idx.size))
        # operator entries of the rows eliminated here, columns in O u U
        rows = K[f.own]
        r = np.repeat(np.arange(nO), np.diff(rows.indptr))
        c = pos[rows.indices]
        keep = c >= 0
        F[r[keep], c[keep]] = rows.data[keep]          # CSR rows hold each column once
        F[nO:, :nO] = F[:nO, nO:].T
        for ch in f.children:
            U = updates.pop(ch)
            p = pos[self.fronts[ch].upd]
            F[np.ix_(p, p)] += U
        pos[idx] = -1
        L_oo = sla.cholesky(F[:nO, :nO], lower=True, check_finite=False)
        L_uo = sla.solve_triangular(L_oo, F[:nO, nO:], lower=True, check_finite=False).T
        f.L_oo, f.L_uo = L_oo, np.ascontiguousarray(L_uo)
        if f.upd.size:
            updates[f_id] = F[nO:, nO:] - L_uo @ L_uo.T

    def solve(self, b: np.ndarray) -> np.ndarray:
        """x = K^-1 b with the factor of ``factor``."""
        y = np.array(b, dtype=np.float64, copy=True)
        for f in self.fronts:                                   # L y = b
            yo = sla.solve_triangular(f.L_oo, y[f.own], lower=True, check_finite=False)
            y[f.own] = yo
            if f.upd.size:
                y[f.upd] -= f.L_uo @ yo
        for f in reversed(self.fronts):                         # L^T x = y
            r = y[f.own]
            if f.upd.size:
                r = r - f.L_uo.T @ y[f.upd]
            y[f.own] = sla.solve_triangular(f.L_oo, r, lower=True, trans="T", check_finite=False)
        return y


def nd_solve(K: sp.spmatrix, b: np.ndarray, leaf: int = 8) -> np.ndarray:
    """Direct solve of the free-dof system K x = b of an N x N cell grid."""
    n = K.shape[0]
    m = int(round((n // 2) ** 0.5))
    if 2 * m * m != n:
        raise ValueError("K is not a free-dof operator of a square grid")
    return NestedDissection(m, leaf).factor(K).solve(b)
