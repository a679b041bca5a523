"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Element-by-element comparisons on seeded inputs at sizes that span several
thread-block tiles and a ragged tail (N = 16, 40, 64), for every step of the
hot path: residual, energy, linearisation + Jacobian apply, Galerkin coarse
operators, dual update, V-cycle, FGMRES, and the full damped-Newton step.

Tolerances (FP64, derived from the arithmetic): element-wise results are
compared relative to the largest entry of the oracle's result, at 1e-11 for
single-pass quantities (a few hundred flops per entry, condition of the
viscous term ~1e3) and 1e-9 for multi-pass ones (V-cycle).  The solution of
the implicit step is unique (Phi strictly convex), so the full step is
compared by its relative L2 error, <= 1e-8 at nonlinear tolerance 1e-10, with
Newton counts within +-1.
"""
import dataclasses

import numpy as np
import pytest

import workloads as W
from oracle import mg
from oracle.fem import Step
from oracle.newton import newton

pytestmark = pytest.mark.gpu


def torch_mod():
    import torch
    return torch


def dev(a):
    torch = torch_mod()
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def make_solver(p, **kw):
    from paper_2204_10822_gb300 import Solver
    c = p.const
    s = Solver(p.N, p.L, rho_ice=c.rho_ice, rho_a=c.rho_a, rho_o=c.rho_o, Ca=c.Ca, Co=c.Co, f_c=c.f_c,
               Pstar=c.Pstar, C=c.C, e=c.e, delta_min=c.delta_min, **kw)
    s.set_forcing(dev(p.h), dev(p.A), dev(p.wind), dev(p.ocean), dev(p.v_old))
    return s


def rand_v(N, seed, scale=0.05):
    rng = np.random.default_rng(seed)
    v = np.zeros((N + 1, N + 1, 2))
    v[1:-1, 1:-1] = scale * rng.standard_normal((N - 1, N - 1, 2))
    return v


def relmax(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


PROBS = [(16, 0), (40, 1), (64, 2)]


@pytest.mark.parametrize("N,seed", PROBS)
def test_residual_parity(N, seed):
    p = W.make_problem(N, seed=seed, v_old=rand_v(N, seed + 7, 0.02))
    st = Step(p)
    s = make_solver(p)
    v = rand_v(N, seed)
    R, nrm = s.residual(p.dt, dev(v))
    Ro = st.residual(v)
    assert relmax(host(R), Ro) < 1e-11
    assert abs(nrm - st.residual_norm(v)) <= 1e-12 * st.residual_norm(v)


@pytest.mark.parametrize("N,seed", PROBS[:2])
def test_energy_parity(N, seed):
    p = W.make_problem(N, seed=seed)
    st = Step(p)
    s = make_solver(p)
    v, dv = rand_v(N, seed), rand_v(N, seed + 1)
    alphas = [1.0, 0.5, 0.25, 0.0]
    phi, scale = s.energy(p.dt, dev(v), dev(dv), alphas)
    for a, f in zip(alphas, phi):
        fo = st.energy(v + a * dv)
        assert abs(f - fo) <= 1e-14 * st.energy_scale(v + a * dv), (a, f, fo)
    assert abs(scale - st.energy_scale(v + dv)) <= 1e-12 * scale


@pytest.mark.parametrize("N,seed", PROBS)
def test_linearize_apply_parity(N, seed):
    p = W.make_problem(N, seed=seed)
    st = Step(p)
    s = make_solver(p)
    v = rand_v(N, seed)
    rng = np.random.default_rng(seed + 3)
    pi = 0.4 * rng.standard_normal((N, N, 4, 3))        # includes 2 pi:pi > 1 (scaled branch)
    s.linearize(p.dt, dev(v), dev(pi))
    K = st.svn_matrix(v, pi)
    x = rand_v(N, seed + 5, 1.0)
    y = host(s.apply(dev(x)))
    yo = st.from_free(K @ st.to_free(x))
    assert relmax(y, yo) < 1e-11


def test_galerkin_levels_parity():
    N = 64
    p = W.make_problem(N, seed=4)
    st = Step(p)
    s = make_solver(p, coarse_N=8)
    v = rand_v(N, 4)
    pi = st.pi_of(v)
    s.linearize(p.dt, dev(v), dev(pi))
    levels = mg.build_hierarchy(st.svn_matrix(v, pi), N, coarse_N=8)
    assert len(levels) == 4
    for l in range(1, 4):
        n = N >> l
        x = rand_v(n, 10 + l, 1.0)
        y = host(s.apply(dev(x), level=l))
        yo = np.zeros_like(x)
        yo[1:-1, 1:-1] = (levels[l].A @ x[1:-1, 1:-1].reshape(-1)).reshape(n - 1, n - 1, 2)
        assert relmax(y, yo) < 1e-11, l


@pytest.mark.parametrize("N,seed", PROBS)
def test_dual_update_parity(N, seed):
    p = W.make_problem(N, seed=seed)
    st = Step(p)
    s = make_solver(p)
    v, dv = rand_v(N, seed), rand_v(N, seed + 2)
    rng = np.random.default_rng(seed + 4)
    pi = 0.4 * rng.standard_normal((N, N, 4, 3))
    alpha = 0.75
    out = host(s.dual_update(p.dt, dev(v), dev(dv), alpha, dev(pi)))
    exp = pi + alpha * st.dual_step(v, dv, pi)
    assert relmax(out, exp) < 1e-12


def test_vcycle_parity_fp64():
    N = 64
    p = W.make_problem(N, seed=5)
    st = Step(p)
    for iters, fuse, deg in ((0, 0, 3), (15, 0, 3), (15, 1, 3), (15, 1, 4)):   # bound, fusion, degree
        s = make_solver(p, coarse_N=8, cheb_degree=deg, cheb_lo=0.1, lmax_iters=iters, cheb_fuse=fuse)
        v = rand_v(N, 5)
        pi = st.pi_of(v)
        s.linearize(p.dt, dev(v), dev(pi))
        levels = mg.build_hierarchy(st.svn_matrix(v, pi), N, coarse_N=8, power_iters=iters)
        r = rand_v(N, 6, 1.0)
        z = host(s.precondition(dev(r)))
        zo = st.from_free(mg.vcycle(levels, st.to_free(r), degree=deg, lo=0.1))
        assert relmax(z, zo) < 1e-9, (iters, fuse, deg)


def test_vcycle_parity_level_degrees():
    # degree 4 on the finest level, 7 on the coarser ones (cheb_degree_coarse):
    # the oracle's V-cycle steps with a per-level degree
    import scipy.linalg as sla
    N = 64
    p = W.make_problem(N, seed=7)
    st = Step(p)
    s = make_solver(p, coarse_N=8, cheb_degree=4, cheb_degree_coarse=7, cheb_lo=0.1, lmax_iters=15)
    v = rand_v(N, 7)
    pi = st.pi_of(v)
    s.linearize(p.dt, dev(v), dev(pi))
    levels = mg.build_hierarchy(st.svn_matrix(v, pi), N, coarse_N=8, power_iters=15)

    def cycle(b, l):
        lv = levels[l]
        if l == len(levels) - 1:
            return sla.cho_solve(lv.chol, b)
        deg = 4 if l == 0 else 7
        x = mg.chebyshev(lv.A, lv.Dinv, b, np.zeros_like(b), deg, lv.lmax, 0.1)
        x = x + lv.P @ cycle(lv.P.T @ (b - lv.A @ x), l + 1)
        return mg.chebyshev(lv.A, lv.Dinv, b, x, deg, lv.lmax, 0.1)

    r = rand_v(N, 9, 1.0)
    z = host(s.precondition(dev(r)))
    zo = st.from_free(cycle(st.to_free(r), 0))
    assert relmax(z, zo) < 1e-9


@pytest.mark.parametrize("fuse", [2, 3, 5])
def test_vcycle_parity_mixed_sweeps(fuse):
    # FP32 V-cycle (mixed precision) against the oracle's FP64 V-cycle, with the
    # two-step sweeps done by the shared-memory tile kernel (cheb_fuse = 2), the
    # row-streaming kernel (3) or the TMA-staged kernel (5) on every level; FP32
    # rounding of the stencil and the arithmetic bounds the difference
    N = 64
    p = W.make_problem(N, seed=11)
    st = Step(p)
    s = make_solver(p, precision="mixed", coarse_N=8, cheb_degree=4, cheb_lo=0.1, lmax_iters=15, cheb_fuse=fuse)
    v = rand_v(N, 11)
    pi = st.pi_of(v)
    s.linearize(p.dt, dev(v), dev(pi))
    levels = mg.build_hierarchy(st.svn_matrix(v, pi), N, coarse_N=8, power_iters=15)
    r = rand_v(N, 12, 1.0)
    z = host(s.precondition(dev(r)))
    zo = st.from_free(mg.vcycle(levels, st.to_free(r), degree=4, lo=0.1))
    assert relmax(z, zo) < 1e-4, relmax(z, zo)


@pytest.mark.parametrize("N", [1024, 2048])
def test_streaming_sweep_matches_tile_sweep(N):
    # at the sizes where the row-streaming (default) and TMA-staged kernels run
    # (finest levels, and their power mode for lambda_max) they compute the same
    # V-cycle as the tile kernel up to FP32 summation order
    p = W.make_problem(N, seed=13)
    v = rand_v(N, 13)
    out = []
    for fuse in (2, 1, 4):
        s = make_solver(p, precision="mixed", cheb_degree=6, cheb_lo=0.02, cheb_fuse=fuse)
        s.linearize(p.dt, dev(v), dev(np.zeros(s.pi_shape)))      # pi = 0 is a valid dual state
        out.append(host(s.precondition(dev(rand_v(N, 14, 1.0)))))
        s.close()
    assert relmax(out[1], out[0]) < 1e-5, relmax(out[1], out[0])
    assert relmax(out[2], out[0]) < 1e-5, relmax(out[2], out[0])


def test_sweep_wait_bound_reports_timeout():
    # a one-poll bound makes every TMA-staged block give up at its first wait
    # (the copies it just issued cannot have landed); the step must fail with
    # SVN_ERR_TIMEOUT, the device must stay usable, and a handle with the
    # default bound must then solve the same step
    from paper_2204_10822_gb300 import SvnError
    p = W.config(0, N=64)
    s = make_solver(p, precision="mixed", cheb_fuse=5, wait_polls=1)
    with pytest.raises(SvnError) as e:
        s.step(p.dt, 1e-8)
    assert e.value.status == "SVN_ERR_TIMEOUT", e.value
    s.close()
    s = make_solver(p, precision="mixed", cheb_fuse=5)
    _, st = s.step(p.dt, 1e-8)
    assert st["status"] == "SVN_OK"


def test_krylov_solve_parity():
    N = 64
    p = W.make_problem(N, seed=6)
    st = Step(p)
    s = make_solver(p, coarse_N=8, cheb_degree=3, cheb_lo=0.05)
    v = rand_v(N, 6)
    pi = st.pi_of(v)
    s.linearize(p.dt, dev(v), dev(pi))
    K = st.svn_matrix(v, pi)
    b = rand_v(N, 8, 1.0)
    x, its = s.krylov_solve(dev(b), 1e-8)
    xf, bf = st.to_free(host(x)), st.to_free(b)
    assert np.linalg.norm(bf - K @ xf) <= 1.05e-8 * np.linalg.norm(bf)
    levels = mg.build_hierarchy(K, N, coarse_N=8, power_iters=15)
    _, its_o, _ = mg.fgmres(K, bf, M=lambda r: mg.vcycle(levels, r, degree=3, lo=0.05), rtol=1e-8, restart=30)
    assert abs(its - its_o) <= 1, (its, its_o)


@pytest.mark.parametrize("N,fused", [(16, 1), (64, 1), (64, 0)])
def test_step_parity_fp64(N, fused):
    p = W.config(0, N=N)
    res = newton(p, tol=1e-10)
    s = make_solver(p, fused_trial=fused)
    v, stats = s.step(p.dt, 1e-10)
    v = host(v)
    err = np.linalg.norm(v - res.v) / np.linalg.norm(res.v)
    assert err <= 1e-8, err
    assert abs(stats["newton_iters"] - res.newton_iters) <= 1, (stats["newton_iters"], res.newton_iters)
    assert stats["status"] == "SVN_OK"


@pytest.mark.parametrize("fp32,fuse", [(1, 1), (0, 1), (1, 3)])
def test_step_parity_mixed(fp32, fuse):
    p = W.config(0, N=64)
    res = newton(p, tol=1e-10)
    s = make_solver(p, precision="mixed", vcycle_fp32=fp32, cheb_fuse=fuse)
    v, stats = s.step(p.dt, 1e-10)
    err = np.linalg.norm(host(v) - res.v) / np.linalg.norm(res.v)
    assert err <= 1e-6, err
    assert abs(stats["newton_iters"] - res.newton_iters) <= 1


def test_step_nonzero_v_old_and_state_roundtrip():
    N = 40
    p = W.make_problem(N, seed=9, v_old=rand_v(N, 3, 0.05))
    res = newton(p, tol=1e-10)
    s = make_solver(p)
    v, stats = s.step(p.dt, 1e-10)
    assert np.linalg.norm(host(v) - res.v) <= 1e-8 * np.linalg.norm(res.v)
    vs, pis = s.get_state()
    st = Step(p)
    # at convergence pi = tau(v)/Delta(v) (Eq. "pi")
    assert relmax(host(pis), st.pi_of(host(vs))) < 1e-5
    s.set_state(vs, pis)
    v2, stats2 = s.step(p.dt, 1e-10)
    assert stats2["newton_iters"] == 0


def test_mass_only_limit_one_newton_step():
    N = 16
    c = dataclasses.replace(W.Constants(), Pstar=0.0, Co=0.0)
    p = W.make_problem(N, seed=1, const=c, v_old=rand_v(N, 2))
    res = newton(p, tol=1e-12)
    s = make_solver(p, krylov_rtol=1e-14)      # exact linear solve: the step is linear
    v, stats = s.step(p.dt, 1e-12)
    assert stats["newton_iters"] == 1
    assert np.linalg.norm(host(v) - res.v) <= 1e-10 * np.linalg.norm(res.v)


def test_error_paths():
    from paper_2204_10822_gb300 import SvnError
    N = 16
    p = W.make_problem(N, seed=0)
    s = make_solver(p)
    bad = p.h.copy()
    bad[3, 4] = np.nan
    with pytest.raises(SvnError) as e:
        s.set_forcing(dev(bad), dev(p.A), dev(p.wind), dev(p.ocean), dev(p.v_old))
    assert e.value.status == "SVN_ERR_NONFINITE"
    neg = p.h.copy()
    neg[0, 0] = -1.0
    with pytest.raises(SvnError) as e:
        s.set_forcing(dev(neg), dev(p.A), dev(p.wind), dev(p.ocean), dev(p.v_old))
    assert e.value.status == "SVN_ERR_ARG"
    with pytest.raises(SvnError) as e:
        s.step(p.dt, 1e-10)          # forcing was rejected: state error
    assert e.value.status == "SVN_ERR_STATE"
    s2 = make_solver(p, max_newton=2)
    v, stats = s2.step(p.dt, 1e-14, raise_on_error=False)
    assert stats["status"] == "SVN_ERR_NO_CONVERGENCE"
    assert stats["newton_iters"] == 2 and np.isfinite(host(v)).all()
    with pytest.raises(SvnError):
        from paper_2204_10822_gb300 import Solver
        Solver(15)                   # odd N


def test_minimum_grid_and_restarted_fgmres():
    # N = 8 (smallest grid, one multigrid level above the 4x4 coarsest) and a
    # restart length of 4 that forces several FGMRES restarts
    for N, kw in ((8, {}), (32, dict(restart=4, krylov_rtol=1e-9, max_krylov=2000))):
        p = W.config(0, N=N)
        res = newton(p, tol=1e-10)
        s = make_solver(p, **kw)
        v, st = s.step(p.dt, 1e-10)
        assert np.linalg.norm(host(v) - res.v) <= 1e-8 * np.linalg.norm(res.v), N
        assert abs(st["newton_iters"] - res.newton_iters) <= 1


def test_line_search_exhaustion_is_reported():
    # stdN on the 32^2 base workload: the oracle first rejects the unit step at
    # Newton iteration 3 (it accepts alpha = 1/8 there), so with no halvings
    # allowed the oracle and the GPU path must both stop at that iteration with
    # a line-search failure (Section 5.1's backtracking, exhausted), after the
    # same residual history, and leave a finite iterate
    p = W.config(0, N=32)
    ref = newton(p, tol=1e-10, method="stdn", max_newton=200, max_halvings=0)
    assert ref.status == "linesearch" and ref.newton_iters == 3
    s = make_solver(p, method=1, krylov_rtol=1e-11, max_krylov=2000, max_halvings=0)
    v, st = s.step(p.dt, 1e-10, raise_on_error=False)
    assert st["status"] == "SVN_ERR_LINESEARCH", st["status"]
    assert st["newton_iters"] == ref.newton_iters
    np.testing.assert_allclose(st["res_hist"], ref.res_hist, rtol=1e-6)
    assert np.isfinite(host(v)).all()


def test_standard_newton_matches_oracle_stdn():
    # stdN (Section 4.1) on the GPU against the oracle's stdN.  Its damped phase
    # is chaotic: in the oracle itself, perturbing every Newton direction by a
    # relative 1e-12 moves the count from 59 to 62-63, because a line-search
    # halving decision flips after about 15 iterations.  So the first 10 step
    # lengths must agree exactly and the residuals along them closely; then
    # the converged solution (unique) and a count band, well above svN's
    # (Section 5.2).
    p = W.config(0, N=32)
    ref = newton(p, tol=1e-10, method="stdn", max_newton=200)
    assert ref.converged
    s = make_solver(p, method=1, krylov_rtol=1e-11, max_krylov=2000)
    v, st = s.step(p.dt, 1e-10, raise_on_error=False)
    assert st["status"] == "SVN_OK"
    k = 10
    assert st["alpha_hist"][:k] == ref.alphas[:k], (st["alpha_hist"][:k], ref.alphas[:k])
    np.testing.assert_allclose(st["res_hist"][:k + 1], ref.res_hist[:k + 1], rtol=1e-6)
    assert np.linalg.norm(host(v) - ref.v) <= 1e-8 * np.linalg.norm(ref.v)
    svn = newton(p, tol=1e-10)
    assert 3 * svn.newton_iters <= st["newton_iters"] <= 2 * ref.newton_iters, (st["newton_iters"], ref.newton_iters)
