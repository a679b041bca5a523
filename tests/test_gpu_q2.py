"""Parity of the CUDA Q2 (biquadratic velocity) path with the Q2 oracle.

Element-by-element comparisons through the C ABI (svn_q2_*) on seeded inputs
at N = 8, 14 (a ragged edge of the 32 x 4 cell blocks) and 40 cells: the
residual, the energy at several step lengths, the linearisation through its
operator (svN coefficient in both branches of Eq. "modification"), the dual
update, and the full damped-Newton step (FP64 Q1 preconditioner: <= 1e-8
relative L2 at tolerance 1e-10, Newton counts within +-1; mixed-precision
preconditioner: <= 1e-6).  Tolerances as for the Q1 parity tests.
"""
import numpy as np
import pytest

import workloads as W
from oracle.fem_q2 import Step2
from oracle.newton import newton

pytestmark = pytest.mark.gpu

SIZES = [(8, 0), (14, 1), (40, 2)]


def dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def relmax(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def rand_v(N, seed, scale=0.05):
    rng = np.random.default_rng(seed)
    v = np.zeros((2 * N + 1, 2 * N + 1, 2))
    v[1:-1, 1:-1] = scale * rng.standard_normal((2 * N - 1, 2 * N - 1, 2))
    return v


def make(p, **kw):
    from paper_2204_10822_gb300 import Q2Solver
    c = p.const
    s = Q2Solver(p.N, p.L, rho_ice=c.rho_ice, rho_a=c.rho_a, rho_o=c.rho_o, Ca=c.Ca, Co=c.Co, f_c=c.f_c,
                 Pstar=c.Pstar, C=c.C, e=c.e, delta_min=c.delta_min, **kw)
    s.set_forcing(dev(p.h), dev(p.A), dev(p.wind), dev(p.ocean), dev(p.v_old))
    return s


@pytest.mark.parametrize("N,seed", SIZES)
def test_q2_residual_parity(N, seed):
    p = W.make_problem_q2(N, seed=seed, v_old=rand_v(N, seed + 7, 0.02))
    st = Step2(p)
    s = make(p)
    v = rand_v(N, seed)
    R, nrm = s.residual(p.dt, dev(v))
    Ro = st.residual(v)
    assert relmax(host(R), Ro) < 1e-11, relmax(host(R), Ro)
    assert abs(nrm - st.residual_norm(v)) <= 1e-12 * st.residual_norm(v)


@pytest.mark.parametrize("N,seed", SIZES[:2])
def test_q2_energy_parity(N, seed):
    p = W.make_problem_q2(N, seed=seed)
    st = Step2(p)
    s = make(p)
    v, dv = rand_v(N, seed), rand_v(N, seed + 1)
    alphas = [0.0, 1.0, 0.5, 0.125]
    phi, scale = s.energy(p.dt, dev(v), dev(dv), alphas)
    for a, f in zip(alphas, phi):
        ref = st.energy(v + a * dv)
        assert abs(f - ref) <= 1e-13 * st.energy_scale(v + a * dv), (a, f, ref)


@pytest.mark.parametrize("N,seed", SIZES)
def test_q2_linearize_apply_parity(N, seed):
    p = W.make_problem_q2(N, seed=seed)
    st = Step2(p)
    s = make(p)
    v = rand_v(N, seed)
    rng = np.random.default_rng(seed + 3)
    pi = 0.4 * rng.standard_normal((N, N, 9, 3))        # both branches of the scaling
    s.linearize(p.dt, dev(v), dev(pi))
    K = st.svn_matrix(v, pi)
    x = rand_v(N, seed + 5, 1.0)
    y = host(s.apply(dev(x)))
    yo = st.from_free(K @ st.to_free(x))
    assert relmax(y, yo) < 1e-11, relmax(y, yo)


@pytest.mark.parametrize("N,seed", SIZES[:2])
def test_q2_dual_update_parity(N, seed):
    p = W.make_problem_q2(N, seed=seed)
    st = Step2(p)
    s = make(p)
    v, dv = rand_v(N, seed), rand_v(N, seed + 1)
    rng = np.random.default_rng(seed + 4)
    pi = 0.4 * rng.standard_normal((N, N, 9, 3))
    out = host(s.dual_update(p.dt, dev(v), dev(dv), 0.5, dev(pi)))
    ref = pi + 0.5 * st.dual_step(v, dv, pi)
    assert relmax(out, ref) < 1e-12, relmax(out, ref)


@pytest.mark.parametrize("N", [8, 16])
def test_q2_step_parity_fp64(N):
    p = W.make_problem_q2(N, seed=0)
    res = newton(p, tol=1e-10, step=Step2(p))
    assert res.converged
    s = make(p, cheb_degree=4, cheb_lo=0.05, coarse_N=4)
    v, stats = s.step(p.dt, 1e-10)
    err = np.linalg.norm(host(v) - res.v) / np.linalg.norm(res.v)
    assert err <= 1e-8, err
    assert abs(stats["newton_iters"] - res.newton_iters) <= 1, (stats["newton_iters"], res.newton_iters)
    vs, pis = s.get_state()
    pc = Step2(p).pi_of(host(vs))
    assert relmax(host(pis), pc) < 1e-5


def test_q2_step_parity_mixed():
    N = 16
    p = W.make_problem_q2(N, seed=3)
    res = newton(p, tol=1e-10, step=Step2(p))
    s = make(p, precision="mixed", cheb_degree=4, cheb_lo=0.05)
    v, stats = s.step(p.dt, 1e-10)
    err = np.linalg.norm(host(v) - res.v) / np.linalg.norm(res.v)
    assert err <= 1e-6, err
    assert abs(stats["newton_iters"] - res.newton_iters) <= 1
