"""ctypes declarations of the C ABI in ``include/svn.h`` (argument marshalling only).

Loading fails loudly when ``libsvn.so`` is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsvn.so")

SVN_MAX_NEWTON = 200
SVN_FP64, SVN_MIXED = 0, 1
STATUS = {0: "SVN_OK", -1: "SVN_ERR_ARG", -2: "SVN_ERR_CUDA", -3: "SVN_ERR_OOM", -4: "SVN_ERR_NONFINITE",
          -5: "SVN_ERR_NO_CONVERGENCE", -6: "SVN_ERR_LINESEARCH", -7: "SVN_ERR_KRYLOV", -8: "SVN_ERR_TIMEOUT",
          -9: "SVN_ERR_STATE"}

c_int, c_double, c_void_p = ctypes.c_int, ctypes.c_double, ctypes.c_void_p
P_double = ctypes.POINTER(ctypes.c_double)


class SvnGrid(ctypes.Structure):
    _fields_ = [("N", c_int), ("L", c_double)]


class SvnParams(ctypes.Structure):
    _fields_ = [(n, c_double) for n in ("rho_ice", "rho_a", "rho_o", "Ca", "Co", "f_c", "Pstar", "C", "e",
                                        "delta_min")] + [
        ("max_newton", c_int), ("max_halvings", c_int), ("ls_floor", c_double),
        ("krylov_rtol", c_double), ("restart", c_int), ("max_krylov", c_int), ("precision", c_int),
        ("cheb_degree", c_int), ("cheb_lo", c_double), ("coarse_N", c_int), ("eisenstat_walker", c_int),
        ("learned", c_int), ("use_graphs", c_int), ("reorth_always", c_int),
        ("ew_eta_max", c_double), ("lmax_iters", c_int), ("lmax_safety", c_double),
        ("learned_rule", c_int), ("method", c_int), ("mg_rebuild", c_int), ("cheb_fuse", c_int),
        ("fused_trial", c_int),
        ("vcycle_fp32", c_int),
        ("cheb_degree_coarse", c_int),
        ("retry_alpha", c_double), ("wait_polls", c_int), ("q2_smooth_degree", c_int),
        ("ew_tail", c_double)]


class SvnStats(ctypes.Structure):
    _fields_ = [("status", c_int), ("newton_iters", c_int), ("krylov_iters_total", c_int),
                ("halvings_total", c_int), ("learned_used", c_int), ("learned_fallback", c_int),
                ("res0", c_double), ("res_final", c_double), ("rel_res_final", c_double), ("seconds", c_double),
                ("krylov_per_newton", c_int * SVN_MAX_NEWTON),
                ("res_hist", c_double * (SVN_MAX_NEWTON + 1)),
                ("alpha_hist", c_double * SVN_MAX_NEWTON),
                ("direction_retries", c_int), ("learned_alpha", c_double)]

    def to_dict(self) -> dict:
        n = self.newton_iters
        return {"status": STATUS.get(self.status, self.status), "newton_iters": n,
                "krylov_iters_total": self.krylov_iters_total, "halvings_total": self.halvings_total,
                "learned_used": self.learned_used, "learned_fallback": self.learned_fallback,
                "res0": self.res0, "res_final": self.res_final, "rel_res_final": self.rel_res_final,
                "seconds": self.seconds, "krylov_per_newton": list(self.krylov_per_newton[:n]),
                "res_hist": list(self.res_hist[:n + 1]), "alpha_hist": list(self.alpha_hist[:n]),
                "direction_retries": self.direction_retries, "learned_alpha": self.learned_alpha}


_SIGS = {
    "svn_default_params": (c_int, [ctypes.POINTER(SvnParams)]),
    "svn_create": (c_int, [ctypes.POINTER(SvnGrid), ctypes.POINTER(SvnParams), c_void_p, ctypes.POINTER(c_void_p)]),
    "svn_destroy": (c_int, [c_void_p]),
    "svn_last_error": (ctypes.c_char_p, [c_void_p]),
    "svn_set_forcing": (c_int, [c_void_p] + [c_void_p] * 5),
    "svn_set_forcing_host": (c_int, [c_void_p] + [c_void_p] * 5),
    "svn_step": (c_int, [c_void_p, c_double, c_double, c_void_p, ctypes.POINTER(SvnStats)]),
    "svn_step_host": (c_int, [c_void_p, c_double, c_double, c_void_p, ctypes.POINTER(SvnStats)]),
    "svn_transport": (c_int, [c_void_p, c_double, ctypes.POINTER(c_int)]),
    "svn_get_ice": (c_int, [c_void_p, c_void_p, c_void_p]),
    "svn_advance": (c_int, [c_void_p, c_double, c_double, c_void_p, c_void_p, c_void_p, ctypes.POINTER(SvnStats),
                            ctypes.POINTER(c_int)]),
    "svn_get_state": (c_int, [c_void_p, c_void_p, c_void_p]),
    "svn_set_state": (c_int, [c_void_p, c_void_p, c_void_p]),
    "svn_residual": (c_int, [c_void_p, c_double, c_void_p, c_void_p, P_double]),
    "svn_energy": (c_int, [c_void_p, c_double, c_void_p, c_void_p, P_double, c_int, P_double, P_double]),
    "svn_linearize": (c_int, [c_void_p, c_double, c_void_p, c_void_p]),
    "svn_apply": (c_int, [c_void_p, c_int, c_void_p, c_void_p]),
    "svn_precondition": (c_int, [c_void_p, c_void_p, c_void_p]),
    "svn_krylov_solve": (c_int, [c_void_p, c_void_p, c_void_p, c_double, ctypes.POINTER(c_int)]),
    "svn_dual_update": (c_int, [c_void_p, c_double, c_void_p, c_void_p, c_double, c_void_p]),
    "svn_profile": (c_int, [c_void_p, c_int]),
    "svn_profile_read": (c_int, [c_void_p, c_int, P_double, ctypes.POINTER(ctypes.c_longlong)]),
    "svn_kernel_launches": (ctypes.c_ulonglong, []),
    "svn_batch_create": (c_int, [c_int, ctypes.POINTER(SvnGrid), ctypes.POINTER(SvnParams), c_int,
                                 ctypes.POINTER(c_void_p)]),
    "svn_batch_destroy": (c_int, [c_void_p]),
    "svn_batch_last_error": (ctypes.c_char_p, [c_void_p]),
    "svn_batch_size": (c_int, [c_void_p]),
    "svn_batch_instance": (c_void_p, [c_void_p, c_int]),
    "svn_batch_step": (c_int, [c_void_p, c_double, c_double, ctypes.POINTER(c_void_p), ctypes.POINTER(SvnStats)]),
    "svn_autotune": (c_int, [c_void_p, c_double, c_int, ctypes.POINTER(c_int), c_int, P_double, c_int, P_double]),
    "svn_set_smoother": (c_int, [c_void_p, c_int, c_int, c_double]),
    "svn_autotune_kernels": (c_int, [c_void_p, c_double, c_int, ctypes.POINTER(c_int), c_int, P_double, c_int,
                                     ctypes.POINTER(c_int), c_int, P_double]),
    "svn_get_params": (c_int, [c_void_p, ctypes.POINTER(SvnParams)]),
    "svn_q2_create": (c_int, [ctypes.POINTER(SvnGrid), ctypes.POINTER(SvnParams), c_void_p,
                              ctypes.POINTER(c_void_p)]),
    "svn_q2_destroy": (c_int, [c_void_p]),
    "svn_q2_last_error": (ctypes.c_char_p, [c_void_p]),
    "svn_q2_set_forcing": (c_int, [c_void_p] + [c_void_p] * 5),
    "svn_q2_step": (c_int, [c_void_p, c_double, c_double, c_void_p, ctypes.POINTER(SvnStats)]),
    "svn_q2_residual": (c_int, [c_void_p, c_double, c_void_p, c_void_p, ctypes.POINTER(c_double)]),
    "svn_q2_energy": (c_int, [c_void_p, c_double, c_void_p, c_void_p, ctypes.POINTER(c_double), c_int,
                              ctypes.POINTER(c_double), ctypes.POINTER(c_double)]),
    "svn_q2_linearize": (c_int, [c_void_p, c_double, c_void_p, c_void_p]),
    "svn_q2_apply": (c_int, [c_void_p, c_void_p, c_void_p]),
    "svn_q2_dual_update": (c_int, [c_void_p, c_double, c_void_p, c_void_p, c_double, c_void_p]),
    "svn_q2_get_state": (c_int, [c_void_p, c_void_p, c_void_p]),
    "svn_net_create": (c_int, [c_int, c_int, c_void_p, ctypes.POINTER(c_void_p)]),
    "svn_net_destroy": (c_int, [c_void_p]),
    "svn_net_last_error": (ctypes.c_char_p, [c_void_p]),
    "svn_net_num_params": (ctypes.c_longlong, [c_void_p]),
    "svn_net_set_params": (c_int, [c_void_p, c_void_p, ctypes.c_longlong]),
    "svn_net_get_params": (c_int, [c_void_p, c_void_p, ctypes.c_longlong]),
    "svn_net_get_grads": (c_int, [c_void_p, c_void_p, ctypes.c_longlong]),
    "svn_net_set_sample": (c_int, [c_void_p, c_int, c_int] + [c_void_p] * 6),
    "svn_net_forward": (c_int, [c_void_p, c_int, c_void_p]),
    "svn_net_train_step": (c_int, [c_void_p, c_int, ctypes.c_float, c_int, ctypes.POINTER(ctypes.c_float)]),
    "svn_attach_net": (c_int, [c_void_p, c_void_p]),
    "svn_set_learned": (c_int, [c_void_p, c_int]),
    "svn_residual_noalloc": (c_int, [ctypes.POINTER(SvnGrid), ctypes.POINTER(SvnParams), c_double] +
                             [c_void_p] * 7 + [P_double, c_void_p]),
}

KCLASS = {"apply": 0, "cheb": 1, "multidot": 2, "update": 3, "element": 4, "residual": 5, "energy": 6,
          "dual": 7, "rap": 8, "vcycle": 9}

_lib = None


def lib() -> ctypes.CDLL:
    """The loaded svN library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libsvn.so not found at %s: run paper_2204_10822_gb300/build.py "
                              "(the svN solver has no CPU fallback)" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_symbols() -> list[str]:
    return sorted(_SIGS)
