"""Explicit upwind finite-volume transport of concentration A and thickness H.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The coupled model (Section 2, Eqs. "model:A" and "model:H") moves A and H
with the ice velocity, dA/dt + div(v A) = 0 and dH/dt + div(v H) = 0, with
A in [0, 1].  Section 3 advances them by an explicit step (an explicit Euler
step is named as the example) before the implicit momentum step, using the
velocity v^n of the previous time level; Section 5.1 discretises A and H as
cell-wise constants (Q0 finite volumes).  The paper fixes no flux formula,
no treatment of large Courant numbers and no limiter, so this module takes
the plainest readings:

  * face flux: first-order upwind, F_f = u_f |f| Q_up, where u_f is the
    outward normal velocity on the face, taken as the mean of the normal
    components at the face's two end nodes (the exact face average of the
    bilinear velocity), and Q_up the value of the cell the flow leaves;
  * boundary: v = 0 on the domain boundary (Section 2), so node velocities
    on the boundary are taken as zero, boundary faces carry no flux, and the
    inflow part of the boundary is empty;
  * explicit Euler, sub-cycled: with c_K = dt/dx * (sum of the outflow
    normal velocities of cell K) the step is split into
    n_sub = max(1, ceil(max_K c_K)) equal sub-steps, which keeps every
    sub-step positivity preserving (each new value is a convex combination
    of old values);
  * A is capped at 1 after the step (A in [0, 1]); H is left as it is.

Arrays: cell fields (N, N) indexed [j, i] (j = y); node velocity
(N+1, N+1, 2) indexed [j, i, k].
"""
from __future__ import annotations

import math

import numpy as np


def face_velocities(v: np.ndarray):
    """Normal velocities on the cell faces.

    Returns ``ux`` of shape (N, N+1): x-velocity on the vertical face at
    x_i between node rows j and j+1 (entry [j, i]); and ``uy`` of shape
    (N+1, N): y-velocity on the horizontal face at y_j between node columns
    i and i+1 (entry [j, i]).  Boundary node velocities count as zero."""
    vb = np.array(v, dtype=np.float64)
    vb[0], vb[-1], vb[:, 0], vb[:, -1] = 0.0, 0.0, 0.0, 0.0
    ux = 0.5 * (vb[:-1, :, 0] + vb[1:, :, 0])
    uy = 0.5 * (vb[:, :-1, 1] + vb[:, 1:, 1])
    return ux, uy


def courant(v: np.ndarray, dt: float, dx: float) -> np.ndarray:
    """c_K = dt/dx * sum over the faces of K of max(outward normal velocity, 0)."""
    ux, uy = face_velocities(v)
    out = (np.maximum(ux[:, 1:], 0.0) + np.maximum(-ux[:, :-1], 0.0)
           + np.maximum(uy[1:, :], 0.0) + np.maximum(-uy[:-1, :], 0.0))
    return (dt / dx) * out


def substeps(v: np.ndarray, dt: float, dx: float) -> int:
    c = float(np.max(courant(v, dt, dx))) if v.shape[0] > 1 else 0.0
    if not math.isfinite(c):
        raise ValueError("non-finite velocity")
    return max(1, int(math.ceil(c)))


def euler_substep(Q: np.ndarray, ux: np.ndarray, uy: np.ndarray, ds: float, dx: float) -> np.ndarray:
    """One explicit Euler step of length ds of dQ/dt + div(v Q) = 0."""
    N = Q.shape[0]
    Fx = np.zeros((N, N + 1))                 # flux in +x through the face at x_i
    for i in range(1, N):
        u = ux[:, i]
        Fx[:, i] = np.where(u > 0.0, u * Q[:, i - 1], u * Q[:, i])
    Fy = np.zeros((N + 1, N))                 # flux in +y through the face at y_j
    for j in range(1, N):
        u = uy[j, :]
        Fy[j, :] = np.where(u > 0.0, u * Q[j - 1, :], u * Q[j, :])
    # Q_K' = Q_K - ds/|K| * (outflow - inflow), |K| = dx^2, |f| = dx
    return Q - (ds / dx) * ((Fx[:, 1:] - Fx[:, :-1]) + (Fy[1:, :] - Fy[:-1, :]))


def transport(N: int, L: float, dt: float, v: np.ndarray, A: np.ndarray, H: np.ndarray):
    """Advance (A, H) over dt with velocity v; returns (A_new, H_new, n_sub)."""
    dx = L / N
    ux, uy = face_velocities(v)
    n = substeps(v, dt, dx)
    ds = dt / n
    A1, H1 = np.array(A, dtype=np.float64), np.array(H, dtype=np.float64)
    for _ in range(n):
        A1 = euler_substep(A1, ux, uy, ds, dx)
        H1 = euler_substep(H1, ux, uy, ds, dx)
    return np.minimum(A1, 1.0), H1, n
