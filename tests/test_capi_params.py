"""Host-side argument checks of the C ABI (no GPU needed: svn_create validates
the grid and the parameters before it touches the device)."""
import ctypes

import pytest

from paper_2204_10822_gb300 import capi

SVN_OK, SVN_ERR_ARG = 0, -1


@pytest.fixture(scope="module", autouse=True)
def built_library():
    from paper_2204_10822_gb300 import build
    build.build()


def defaults():
    p = capi.SvnParams()
    assert capi.lib().svn_default_params(ctypes.byref(p)) == SVN_OK
    return p


def test_defaults_match_the_header():
    p = defaults()
    # paper constants (Table "tab:params"; P* read as 27.5 kN/m^2) and solver defaults
    assert (p.rho_ice, p.rho_a, p.rho_o, p.Ca, p.Co, p.Pstar, p.C, p.e) == (900.0, 1.3, 1026.0, 1.2e-3, 5.5e-3,
                                                                          27500.0, 20.0, 2.0)
    assert p.delta_min == 2e-9 and p.max_newton == 200 and p.max_halvings == 30
    assert p.krylov_rtol == 1e-6 and p.restart == 30 and p.cheb_degree == 3 and p.coarse_N == 4
    assert p.precision == capi.SVN_FP64 and p.method == 0 and p.cheb_fuse == 1 and p.cheb_degree_coarse == 0
    assert p.lmax_iters == 15 and p.lmax_safety == 1.15 and p.use_graphs == 1 and p.vcycle_fp32 == 1
    assert p.retry_alpha == 1.0 / 64.0 and p.wait_polls == 0 and p.q2_smooth_degree == 3
    assert p.ew_tail == 0.5


def create(grid, params):
    lib = capi.lib()
    h = ctypes.c_void_p()
    rc = lib.svn_create(ctypes.byref(grid), ctypes.byref(params), None, ctypes.byref(h))
    msg = lib.svn_last_error(h).decode() if h.value else ""
    if h.value:
        lib.svn_destroy(h)
    return rc, msg


@pytest.mark.parametrize("field,value,needle", [
    ("cheb_fuse", 6, "cheb_fuse"), ("wait_polls", -1, "wait_polls"), ("method", 2, "method"), ("cheb_degree", 0, "cheb_degree"),
    ("cheb_degree", 17, "cheb_degree"), ("restart", 0, "restart"), ("restart", 201, "restart"),
    ("cheb_degree_coarse", 17, "cheb_degree_coarse"), ("cheb_degree_coarse", -1, "cheb_degree_coarse"),
    ("lmax_safety", 0.5, "lmax_safety"), ("lmax_iters", 61, "lmax_iters"), ("cheb_lo", 1.0, "cheb_lo"),
    ("coarse_N", 1, "coarse_N"), ("precision", 7, "precision"), ("max_newton", 201, "max_newton"),
    ("max_halvings", -1, "max_halvings"), ("e", 0.0, "physical"), ("delta_min", 0.0, "physical"),
    ("retry_alpha", -0.5, "retry_alpha"), ("retry_alpha", 2.0, "retry_alpha"),
    ("learned_rule", 5, "learned_rule"), ("learned_rule", -1, "learned_rule"),
    ("q2_smooth_degree", 17, "q2_smooth_degree"), ("ew_tail", -0.1, "ew_tail"), ("ew_tail", 1.5, "ew_tail")])
def test_bad_parameter_is_rejected(field, value, needle):
    p = defaults()
    setattr(p, field, value)
    rc, msg = create(capi.SvnGrid(64, 512e3), p)
    assert rc == SVN_ERR_ARG and needle in msg, (rc, msg)


@pytest.mark.parametrize("N,L", [(7, 512e3), (6, 512e3), (16386, 512e3), (64, 0.0), (64, float("inf"))])
def test_bad_grid_is_rejected(N, L):
    rc, msg = create(capi.SvnGrid(N, L), defaults())
    assert rc == SVN_ERR_ARG and msg, (rc, msg)


def test_null_arguments():
    lib = capi.lib()
    assert lib.svn_create(None, None, None, None) == SVN_ERR_ARG
    assert lib.svn_destroy(None) == SVN_ERR_ARG
    assert lib.svn_step(None, 1.0, 1e-8, None, None) == SVN_ERR_ARG
    assert lib.svn_transport(None, 1.0, None) == SVN_ERR_ARG
    assert lib.svn_advance(None, 1.0, 1e-4, None, None, None, None, None) == SVN_ERR_ARG
