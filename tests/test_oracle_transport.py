"""Pins of the oracle's explicit upwind transport of A and H (Sections 2, 3, 5.1).

Each pin is fixed by the conservation law or by a closed form, not by the
oracle's own formula: a swapped upwind direction, a wrong face index, a
missing 1/dx or a sign error each fail at least one of them.
"""
import numpy as np
import pytest

from oracle.transport import transport, courant, face_velocities, substeps
import workloads as W


def interior_field(N, fx, fy):
    v = np.zeros((N + 1, N + 1, 2))
    v[1:-1, 1:-1, 0] = fx
    v[1:-1, 1:-1, 1] = fy
    return v


def test_zero_velocity_is_identity():
    rng = np.random.default_rng(0)
    N = 12
    A, H = rng.uniform(0.2, 1.0, (N, N)), rng.uniform(0.1, 3.0, (N, N))
    A1, H1, n = transport(N, 1.0, 10.0, np.zeros((N + 1, N + 1, 2)), A, H)
    assert n == 1 and np.array_equal(A1, A) and np.array_equal(H1, H)


def test_boundary_velocities_are_ignored():
    # v = 0 on the boundary (Section 2): boundary node values must not matter
    rng = np.random.default_rng(1)
    N = 10
    v = interior_field(N, rng.normal(size=(N - 1, N - 1)), rng.normal(size=(N - 1, N - 1)))
    w = v.copy()
    w[0], w[-1], w[:, 0], w[:, -1] = 5.0, -3.0, 7.0, 2.0
    A, H = rng.uniform(0.2, 0.9, (N, N)), rng.uniform(0.1, 3.0, (N, N))
    a = transport(N, 1.0, 0.05, v, A, H)
    b = transport(N, 1.0, 0.05, w, A, H)
    assert a[2] == b[2] and np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("scale", [0.05, 3.0])
def test_mass_is_conserved(scale):
    # div-form with zero boundary flux: sum of H |K| is invariant (A too while
    # the cap at 1 is inactive); also with sub-cycling (scale 3 -> n_sub > 1)
    rng = np.random.default_rng(2)
    N = 16
    v = interior_field(N, scale * rng.normal(size=(N - 1, N - 1)), scale * rng.normal(size=(N - 1, N - 1)))
    A, H = rng.uniform(0.001, 0.01, (N, N)), rng.uniform(0.1, 3.0, (N, N))
    A1, H1, n = transport(N, 16.0, 1.0, v, A, H)
    assert (n > 1) == (scale > 1)
    assert abs(H1.sum() - H.sum()) <= 1e-13 * H.sum()
    assert A1.max() < 1.0
    assert abs(A1.sum() - A.sum()) <= 1e-13 * A.sum()


def test_unit_courant_shift():
    # uniform u with u dt/dx = 1: upwind moves every interior cell value one
    # cell downstream, Q'(j, i) = Q(j, i - 1) (u > 0) or Q(j, i + 1) (u < 0)
    rng = np.random.default_rng(3)
    N = 12
    H = rng.uniform(0.1, 3.0, (N, N))
    A = rng.uniform(0.1, 1.0, (N, N))
    for u, di in ((1.0, -1), (-1.0, +1)):
        v = interior_field(N, u, 0.0)
        A1, H1, n = transport(N, float(N), 1.0, v, A, H)      # dx = 1, dt = 1
        assert n == 1
        rows = slice(1, N - 1)               # faces with both end nodes interior
        cols = np.arange(1, N - 1)
        np.testing.assert_allclose(H1[rows, cols], H[rows, cols + di], rtol=1e-15, atol=0)
        np.testing.assert_allclose(A1[rows, cols], A[rows, cols + di], rtol=1e-15, atol=0)
    # the same along y
    v = interior_field(N, 0.0, 1.0)
    _, H1, _ = transport(N, float(N), 1.0, v, A, H)
    np.testing.assert_allclose(H1[1:N - 1, 1:N - 1], H[0:N - 2, 1:N - 1], rtol=1e-15, atol=0)


def test_linear_flow_closed_form():
    # v = (a x, b y): div v = a + b, so a constant field c becomes
    # c (1 - (a + b) dt) on cells whose faces all have interior end nodes
    N, L, dt = 16, 32.0, 0.01
    a, b, c = 0.3, 0.7, 0.8
    x = np.linspace(0.0, L, N + 1)
    X, Y = np.meshgrid(x, x, indexing="xy")
    v = np.zeros((N + 1, N + 1, 2))
    v[..., 0], v[..., 1] = a * X, b * Y
    A1, H1, n = transport(N, L, dt, v, np.full((N, N), c), np.full((N, N), c))
    assert n == 1
    np.testing.assert_allclose(H1[1:N - 1, 1:N - 1], c * (1 - (a + b) * dt), rtol=1e-14)
    np.testing.assert_allclose(A1[1:N - 1, 1:N - 1], c * (1 - (a + b) * dt), rtol=1e-14)


def test_two_by_two_by_hand():
    # one interior node (1, 1) with velocity (p, q) > 0; each interior face
    # has it and a boundary node as end points, so every interior normal
    # velocity is p/2 (vertical faces) or q/2 (horizontal).  Flow leaves SW,
    # passes SE and NW, and collects in NE:
    #   SW' = SW - k (p + q)/2 SW
    #   SE' = SE + k (p/2 SW - q/2 SE)
    #   NW' = NW + k (q/2 SW - p/2 NW)
    #   NE' = NE + k (p/2 NW + q/2 SE),                        k = dt/dx
    p, q, dt, L = 0.3, 0.2, 0.5, 4.0
    v = np.zeros((3, 3, 2))
    v[1, 1] = (p, q)
    H = np.array([[1.0, 2.0], [3.0, 4.0]])          # [j, i]: SW, SE / NW, NE
    A = np.array([[0.5, 0.6], [0.7, 0.8]])
    A1, H1, n = transport(2, L, dt, v, A, H)
    k = dt / (L / 2)
    for Q, Q1 in ((H, H1), (A, A1)):
        SW, SE, NW, NE = Q[0, 0], Q[0, 1], Q[1, 0], Q[1, 1]
        expect = np.array([[SW - k * (p + q) / 2 * SW, SE + k * (p / 2 * SW - q / 2 * SE)],
                           [NW + k * (q / 2 * SW - p / 2 * NW), NE + k * (p / 2 * NW + q / 2 * SE)]])
        np.testing.assert_allclose(Q1, expect, rtol=1e-15)
    assert n == 1


def test_cap_and_convergence():
    # flow into the SW cell of a 2x2 grid: A there would exceed 1 and is
    # capped, H grows (mass kept)
    v = np.zeros((3, 3, 2))
    v[1, 1] = (-0.4, -0.4)
    A, H = np.ones((2, 2)), np.ones((2, 2))
    A1, H1, n = transport(2, 2.0, 0.5, v, A, H)
    assert A1[0, 0] == 1.0 and H1[0, 0] > 1.0 and abs(H1.sum() - 4.0) < 1e-15
    assert A1[1, 1] < 1.0 and A1[0, 1] == 1.0 and A1[1, 0] == 1.0


def test_courant_and_positivity_under_subcycling():
    rng = np.random.default_rng(4)
    N = 16
    v = interior_field(N, 4.0 * rng.normal(size=(N - 1, N - 1)), 4.0 * rng.normal(size=(N - 1, N - 1)))
    c = courant(v, 1.0, 1.0)
    # brute force: per cell, the outflow through each of its four faces
    ux, uy = face_velocities(v)
    brute = np.zeros((N, N))
    for j in range(N):
        for i in range(N):
            brute[j, i] = max(ux[j, i + 1], 0) + max(-ux[j, i], 0) + max(uy[j + 1, i], 0) + max(-uy[j, i], 0)
    np.testing.assert_allclose(c, brute, rtol=1e-15)
    np.testing.assert_allclose(courant(v, 0.5, 2.0), 0.25 * brute, rtol=1e-15)   # c = dt/dx * outflow
    n = substeps(v, 1.0, 1.0)
    assert n == int(np.ceil(brute.max())) and n >= 3
    A, H = rng.uniform(0.0, 1.0, (N, N)), rng.uniform(0.0, 2.0, (N, N))
    A1, H1, _ = transport(N, float(N), 1.0, v, A, H)
    assert A1.min() >= 0.0 and H1.min() >= 0.0


def test_problem_two_fields():
    # Section 5.3's fields: ocean 0.01 m/s rotation about the centre, wind
    # zero at the cyclone centre and at day 4, initial H in [0.29, 0.31]
    p = W.problem_two(64)
    assert np.all(p.A == 1.0) and 0.29 <= p.h.min() and p.h.max() <= 0.31
    assert np.allclose(p.ocean[32, 32], 0.0) and abs(np.abs(p.ocean).max() - 0.01) < 1e-15
    assert np.abs(W.problem_two_wind(64, 4 * 86400.0)).max() == 0.0
    # centre at t = 2 d: 256 + 102.4 km on the diagonal (node 366.4 km / 8 km: between nodes)
    w = W.problem_two_wind(64, 2 * 86400.0)
    speed = np.sqrt((w ** 2).sum(-1))
    assert 10.9 < speed.max() <= 15 * 100 / 50 / np.e + 1e-9


def test_problem_two_steps_conserve_ice_volume():
    # the coupled oracle time stepping (Section 3: transport with v^n, then
    # the momentum step) keeps sum H |K| (no flux across the boundary, where
    # v = 0) while the ice moves; A stays in [0, 1]
    from oracle.newton import newton
    N = 16
    p = W.problem_two(N)
    v, H, A = p.v_old.copy(), p.h.copy(), p.A.copy()
    vol0 = H.sum()
    for n in range(3):
        A, H, _ = transport(N, p.L, p.dt, v, A, H)
        q = W.Problem(N=N, L=p.L, const=p.const, h=H, A=A, wind=W.problem_two_wind(N, (n + 1) * p.dt),
                      ocean=p.ocean, v_old=v, dt=p.dt)
        r = newton(q, tol=1e-8)
        assert r.converged
        v = r.v
        assert abs(H.sum() - vol0) <= 1e-14 * vol0
        assert 0.0 <= A.min() and A.max() <= 1.0
    assert np.abs(H - p.h).max() > 0.0
