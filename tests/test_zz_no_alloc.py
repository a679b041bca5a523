"""The allocation-free residual entry point (svn_residual_noalloc).

It exists for callers that cannot call cudaMalloc (a host model that owns the
whole device through its own pool, or a runtime that keeps its footprint
fixed after start-up).  It must give the same R(v) and ||R|| as the handle-
based svn_residual, within the residual tolerance of the parity tests, on two
calls in a row (the second call reuses the shared device array that the first
one left behind), whether it runs alone in a fresh process or after the
other tests.  The file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def _rand_v(N, seed, scale=0.05):
    rng = np.random.default_rng(seed)
    v = np.zeros((N + 1, N + 1, 2))
    v[1:-1, 1:-1] = scale * rng.standard_normal((N - 1, N - 1, 2))
    return v


def test_residual_noalloc_matches_handle_entry_point():
    import torch
    from paper_2204_10822_gb300 import Solver, capi
    lib = capi.lib()
    stream = torch.cuda.current_stream()
    for N, seed in ((64, 3), (40, 5)):           # two calls in a row, different grids
        p = W.make_problem(N, seed=seed, v_old=_rand_v(N, seed + 1, 0.02))
        ins = [_dev(x) for x in (p.h, p.A, p.wind, p.ocean, p.v_old)]
        v = _dev(_rand_v(N, seed + 2))
        s = Solver(N, p.L)
        s.set_forcing(*ins)
        R_ref, n_ref = s.residual(p.dt, v)
        R = torch.zeros_like(R_ref)
        nrm = ctypes.c_double()
        g = capi.SvnGrid(N, p.L)
        rc = lib.svn_residual_noalloc(ctypes.byref(g), ctypes.byref(s.params), p.dt,
                                      *[x.data_ptr() for x in ins], v.data_ptr(), R.data_ptr(),
                                      ctypes.byref(nrm), ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0
        Rr, Rn = R_ref.cpu().numpy(), R.cpu().numpy()
        assert np.abs(Rn - Rr).max() <= 1e-11 * np.abs(Rr).max()
        assert abs(nrm.value - n_ref) <= 1e-12 * n_ref
        s.close()


def test_residual_noalloc_rejects_oversized_grid():
    from paper_2204_10822_gb300 import capi, default_params
    lib = capi.lib()
    g = capi.SvnGrid(2 * 256, 512e3)          # above SVN_NOALLOC_MAX_N
    prm = default_params()
    dummy = ctypes.c_void_p(1)
    rc = lib.svn_residual_noalloc(ctypes.byref(g), ctypes.byref(prm), 1800.0, *([dummy] * 7), None, None)
    assert rc == -1
