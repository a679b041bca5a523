"""Pins of the oracle's modified svN operator and dual step in the scaled branch.

Eq. "modification" (Section 4.2) replaces tau(v_l) (x) pi_l, with the paper's
convention (X (x) Y) Z = (X : Z) Y, by

    [tau (x) pi + pi (x) tau] / (2 max(1, sqrt(2 pi:pi)))

in the operator of Eq. "linearSVNewton" and, "for consistency", in the last
term of Eq. "tautilde".  Where 2 pi:pi > 1 that is the unscaled symmetrised
term evaluated at pi_hat = pi / sqrt(2 pi:pi), which lies on the sphere
2 pi_hat:pi_hat = 1.  The checks below are written on full 2 x 2 tensors
(not the oracle's Voigt vectors), with pi_hat formed explicitly on states
where every quadrature point is in one branch, so no max() appears:

  * the bilinear form t(S1)^T C t(S2) of ``svn_coefficients`` equals
    dt [ (P/Delta) T1:T2 - (P/Delta^2) ((T:S1)(pi_hat:S2) + (pi_hat:S1)(T:S2)) ];
  * ``dual_step`` equals -pi + T/Delta + T~/Delta
    - ((T:T~) pi_hat + (pi_hat:T~) T) / Delta^2;
  * the two are the same elimination (Section 4.2): dt P times the part of the
    dual step that is linear in dv is C t(tau(dv)) at every point;
  * C(v, s pi) = C(v, pi) for s >= 1 once 2 pi:pi >= 1 (only the direction of
    pi enters the scaled branch).

Planted mistakes in a copy of the oracle (the factor 2 dropped from m, and the
unsymmetrised 2 (tau:tau~) pi / m kept) must fail the first two checks.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle.fem import Step, comp_to_voigt, voigt_to_comp

SQ2 = math.sqrt(2.0)


def problem(N=6, seed=3):
    return W.make_problem(N, seed=seed)


def random_velocity(N, seed, scale=0.1):
    rng = np.random.default_rng(seed)
    v = scale * rng.standard_normal((N + 1, N + 1, 2))
    v[0], v[-1], v[:, 0], v[:, -1] = 0, 0, 0, 0
    return v


def tensor(xx, yy, xy):
    """Full symmetric 2x2 tensor (..., 2, 2) from components."""
    out = np.empty(np.shape(xx) + (2, 2))
    out[..., 0, 0], out[..., 1, 1] = xx, yy
    out[..., 0, 1] = out[..., 1, 0] = xy
    return out


def ddot(X, Y):
    """X : Y for full 2x2 tensors."""
    return np.einsum("...ij,...ij->...", X, Y)


def voigt(X):
    """(Xxx, Xyy, sqrt2 Xxy), written here from the definition X:Y = t(X).t(Y)."""
    return np.stack([X[..., 0, 0], X[..., 1, 1], SQ2 * X[..., 0, 1]], axis=-1)


def pi_states(N, seed):
    """Two dual states: every point scaled (2 pi:pi in [1.5, 40]) or every point
    unscaled (2 pi:pi <= 0.8)."""
    rng = np.random.default_rng(seed)
    raw = rng.standard_normal((N, N, 4, 3))
    P = tensor(raw[..., 0], raw[..., 1], raw[..., 2])
    n2 = 2 * ddot(P, P)
    big_target = rng.uniform(1.5, 40.0, n2.shape)
    small_target = rng.uniform(0.05, 0.8, n2.shape)
    big = P * np.sqrt(big_target / n2)[..., None, None]
    small = P * np.sqrt(small_target / n2)[..., None, None]
    return big, small


def tau_tensor(st, v):
    tv = st.mesh.tau_at_qp(st.mesh.gather(v))             # oracle Voigt (pinned by FD tests)
    return tensor(tv[..., 0], tv[..., 1], tv[..., 2] / SQ2)


def delta_of(st, T):
    return np.sqrt(st.c.delta_min ** 2 + 2 * ddot(T, T))


def coefficient_error(step_cls, scaled):
    st = step_cls(problem())
    v = random_velocity(6, 5)
    big, small = pi_states(6, 17)
    Pi = big if scaled else small
    n2 = 2 * ddot(Pi, Pi)
    assert (n2 > 1).all() if scaled else (n2 < 1).all()
    Pihat = Pi / np.sqrt(n2)[..., None, None] if scaled else Pi
    T = tau_tensor(st, v)
    D = delta_of(st, T)
    Pq = np.broadcast_to(st.P[..., None], D.shape)
    C = st.svn_coefficients(v, np.stack([Pi[..., 0, 0], Pi[..., 1, 1], Pi[..., 0, 1]], -1))
    rng = np.random.default_rng(23)
    worst = 0.0
    for _ in range(4):
        r1, r2 = rng.standard_normal((2,) + D.shape + (3,))
        S1, S2 = tensor(*np.moveaxis(r1, -1, 0)), tensor(*np.moveaxis(r2, -1, 0))
        want = st.dt * ((Pq / D) * ddot(S1, S2)
                        - (Pq / D ** 2) * (ddot(T, S1) * ddot(Pihat, S2) + ddot(Pihat, S1) * ddot(T, S2)))
        got = np.einsum("...a,...ab,...b->...", voigt(S1), C, voigt(S2))
        scale = st.dt * (Pq / D) * np.sqrt(ddot(S1, S1) * ddot(S2, S2))
        worst = max(worst, float(np.max(np.abs(got - want) / scale)))
    return worst


def dual_error(step_cls, scaled):
    st = step_cls(problem())
    v = random_velocity(6, 4)
    dv = random_velocity(6, 9, scale=1.0)
    big, small = pi_states(6, 31)
    Pi = big if scaled else small
    n2 = 2 * ddot(Pi, Pi)
    Pihat = Pi / np.sqrt(n2)[..., None, None] if scaled else Pi
    T = tau_tensor(st, v)
    Tt = tau_tensor(st, dv)
    D = delta_of(st, T)[..., None, None]
    want = -Pi + T / D + Tt / D - (ddot(T, Tt)[..., None, None] * Pihat
                                    + ddot(Pihat, Tt)[..., None, None] * T) / D ** 2
    got_c = st.dual_step(v, dv, np.stack([Pi[..., 0, 0], Pi[..., 1, 1], Pi[..., 0, 1]], -1))
    got = tensor(got_c[..., 0], got_c[..., 1], got_c[..., 2])
    return float(np.max(np.abs(got - want)) / np.max(np.abs(want)))


class DroppedTwo(Step):
    """Planted mistake: m = max(1, sqrt(pi:pi)) (factor 2 dropped)."""

    def _m(self, pi):
        p = comp_to_voigt(pi)
        return np.maximum(1.0, np.sqrt(np.sum(p * p, axis=-1)))

    def svn_coefficients(self, v, pi):
        m, dt = self.mesh, self.dt
        t = m.tau_at_qp(m.gather(v))
        Dl = self.delta(t)
        p = comp_to_voigt(pi)
        mm = self._m(pi)
        P = np.broadcast_to(self.P[..., None], Dl.shape)
        sym = np.einsum("...a,...b->...ab", t, p) + np.einsum("...a,...b->...ab", p, t)
        return dt * ((P / Dl)[..., None, None] * np.eye(3) - (P / (Dl * Dl * mm))[..., None, None] * sym)

    def dual_step(self, v, dv, pi):
        m = self.mesh
        t = m.tau_at_qp(m.gather(v))
        tt = m.tau_at_qp(m.gather(dv))
        Dl = self.delta(t)[..., None]
        p = comp_to_voigt(pi)
        mm = self._m(pi)[..., None]
        dp = -p + t / Dl + tt / Dl - (np.sum(t * tt, -1)[..., None] * p + np.sum(p * tt, -1)[..., None] * t) / (
            Dl * Dl * mm)
        return voigt_to_comp(dp)


class Unsymmetrised(Step):
    """Planted mistake: the scaled but unsymmetrised term 2 (tau:tau~) pi / m."""

    def svn_coefficients(self, v, pi):
        m, dt = self.mesh, self.dt
        t = m.tau_at_qp(m.gather(v))
        Dl = self.delta(t)
        p = comp_to_voigt(pi)
        mm = np.maximum(1.0, np.sqrt(2.0 * np.sum(p * p, axis=-1)))
        P = np.broadcast_to(self.P[..., None], Dl.shape)
        # y = C x with (t (x) p) x = (t.x) p  ->  C = p t^T
        return dt * ((P / Dl)[..., None, None] * np.eye(3)
                     - (2 * P / (Dl * Dl * mm))[..., None, None] * np.einsum("...a,...b->...ab", p, t))

    def dual_step(self, v, dv, pi):
        m = self.mesh
        t = m.tau_at_qp(m.gather(v))
        tt = m.tau_at_qp(m.gather(dv))
        Dl = self.delta(t)[..., None]
        p = comp_to_voigt(pi)
        mm = np.maximum(1.0, np.sqrt(2.0 * np.sum(p * p, axis=-1)))[..., None]
        dp = -p + t / Dl + tt / Dl - 2 * np.sum(t * tt, -1)[..., None] * p / (Dl * Dl * mm)
        return voigt_to_comp(dp)


@pytest.mark.parametrize("scaled", [True, False])
def test_coefficients_match_tensor_form(scaled):
    assert coefficient_error(Step, scaled) < 1e-12


@pytest.mark.parametrize("scaled", [True, False])
def test_dual_step_matches_tensor_form(scaled):
    assert dual_error(Step, scaled) < 1e-12


@pytest.mark.parametrize("planted", [DroppedTwo, Unsymmetrised])
def test_planted_mistakes_fail_the_tensor_pins(planted):
    # both mistakes only show in the scaled branch (or in the split, which the
    # random, non-symmetric-direction pi exposes in either branch)
    assert coefficient_error(planted, True) > 1e-3
    assert dual_error(planted, True) > 1e-3


def test_dual_step_and_operator_are_one_elimination():
    st = Step(problem())
    v = random_velocity(6, 2)
    dv = random_velocity(6, 8, scale=1.0)
    for Pi in pi_states(6, 41):
        pi = np.stack([Pi[..., 0, 0], Pi[..., 1, 1], Pi[..., 0, 1]], -1)
        lin = comp_to_voigt(st.dual_step(v, dv, pi) - st.dual_step(v, np.zeros_like(dv), pi))
        C = st.svn_coefficients(v, pi)
        ttd = st.mesh.tau_at_qp(st.mesh.gather(dv))
        lhs = st.dt * st.P[..., None, None] * lin
        rhs = np.einsum("...ab,...b->...a", C, ttd)
        assert np.max(np.abs(lhs - rhs)) <= 1e-12 * np.max(np.abs(rhs))


def test_scaled_branch_depends_only_on_the_direction_of_pi():
    st = Step(problem())
    v = random_velocity(6, 7)
    big, _ = pi_states(6, 53)
    pi = np.stack([big[..., 0, 0], big[..., 1, 1], big[..., 0, 1]], -1)
    C1 = st.svn_coefficients(v, pi)
    for s in (1.0, 2.5, 1e3):
        C2 = st.svn_coefficients(v, s * pi)
        assert np.max(np.abs(C2 - C1)) <= 1e-13 * np.max(np.abs(C1))
    # on the sphere 2 pi:pi = 1 both branches give the same operator
    n = np.sqrt(2 * np.sum(comp_to_voigt(pi) ** 2, -1))[..., None]
    on = pi / n
    C_on = st.svn_coefficients(v, on)
    C_out = st.svn_coefficients(v, on * (1 + 1e-12))
    assert np.max(np.abs(C_on - C_out)) <= 1e-10 * np.max(np.abs(C_on))
