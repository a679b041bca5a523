"""Thin Python binding of the svN C ABI (argument marshalling only).

Device calls take CUDA float64 tensors; ``*_host`` calls take NumPy arrays.
Array layouts are those of ``include/svn.h``:
  cells (N, N) [j, i]; node vectors (N+1, N+1, 2) [j, i, k];
  dual state (N, N, 4, 3) [j, i, q, c].
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import capi


class SvnError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s: %s" % (capi.STATUS.get(code, code), msg))
        self.code = code
        self.status = capi.STATUS.get(code, str(code))


PARAM_NAMES = frozenset(name for name, _ in capi.SvnParams._fields_)


def default_params(**overrides) -> capi.SvnParams:
    """The library's defaults with `overrides` applied; an unknown name is an
    error (a misspelt setting would otherwise be ignored)."""
    unknown = sorted(set(overrides) - PARAM_NAMES)
    if unknown:
        raise TypeError("unknown svn_params field(s): %s" % ", ".join(unknown))
    p = capi.SvnParams()
    capi.lib().svn_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        if k == "precision" and isinstance(v, str):
            v = {"fp64": capi.SVN_FP64, "mixed": capi.SVN_MIXED}[v]
        setattr(p, k, v)
    return p


def _check_numel(t, numel, name):
    """The C ABI reads and writes exactly `numel` float64 values through a bare
    pointer: a buffer of another size is refused here, before any call."""
    n = int(t.numel()) if hasattr(t, "numel") and callable(t.numel) else int(np.size(t))
    if numel is not None and n != numel:
        raise ValueError("%s: expected %d float64 values, got %d" % (name, numel, n))


def _ptr(t, numel=None, name="array") -> int:
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError("%s: expected a contiguous CUDA float64 tensor" % name)
    _check_numel(t, numel, name)
    return t.data_ptr()


def _hptr(a, numel=None, name="array"):
    a = np.ascontiguousarray(a, dtype=np.float64)
    _check_numel(a, numel, name)
    return a.ctypes.data, a


def _host_out(out, numel, name="out"):
    """A caller-supplied host result buffer: written in place, so it must be a
    C-contiguous, writable float64 array of exactly `numel` values."""
    if not (isinstance(out, np.ndarray) and out.dtype == np.float64 and out.flags.c_contiguous
            and out.flags.writeable):
        raise TypeError("%s: expected a writable C-contiguous float64 NumPy array" % name)
    _check_numel(out, numel, name)
    return out.ctypes.data


class Solver:
    """One svN solver instance for an N x N grid of side L on the current device."""

    def __init__(self, N: int, L: float = 512e3, stream=None, **params):
        import torch
        self.N, self.L = int(N), float(L)
        self.nc, self.nv, self.npi = self.N * self.N, 2 * (self.N + 1) ** 2, 12 * self.N * self.N
        self.lib = capi.lib()
        self.params = default_params(**params)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        g = capi.SvnGrid(self.N, self.L)
        h = ctypes.c_void_p()
        rc = self.lib.svn_create(ctypes.byref(g), ctypes.byref(self.params),
                                 ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        self.h = h
        if rc != 0:
            msg = self.lib.svn_last_error(h).decode() if h.value else ""
            if h.value:
                self.lib.svn_destroy(h)
            self.h = None
            raise SvnError(rc, msg)

    def close(self):
        if getattr(self, "h", None):
            self.lib.svn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc: int):
        if rc != 0:
            raise SvnError(rc, self.lib.svn_last_error(self.h).decode())

    # -- shapes --------------------------------------------------------------
    @property
    def node_shape(self):
        return (self.N + 1, self.N + 1, 2)

    @property
    def pi_shape(self):
        return (self.N, self.N, 4, 3)

    def _vec(self):
        import torch
        return torch.zeros(self.node_shape, dtype=torch.float64, device="cuda")

    # -- step ----------------------------------------------------------------
    def _forcing_sizes(self):
        return ((self.nc, "h"), (self.nc, "A"), (self.nv, "wind"), (self.nv, "ocean"), (self.nv, "v_old"))

    def set_forcing(self, h, A, wind, ocean, v_old):
        ptrs = [_ptr(x, n, nm) for x, (n, nm) in zip((h, A, wind, ocean, v_old), self._forcing_sizes())]
        self._check(self.lib.svn_set_forcing(self.h, *ptrs))

    def set_forcing_host(self, h, A, wind, ocean, v_old):
        keep = [_hptr(x, n, nm) for x, (n, nm) in zip((h, A, wind, ocean, v_old), self._forcing_sizes())]
        self._check(self.lib.svn_set_forcing_host(self.h, *[k[0] for k in keep]))

    def step(self, dt: float, tol: float, out=None, raise_on_error: bool = True):
        out = self._vec() if out is None else out
        st = capi.SvnStats()
        rc = self.lib.svn_step(self.h, dt, tol, _ptr(out, self.nv, "out"), ctypes.byref(st))
        if rc != 0 and raise_on_error:
            self._check(rc)
        return out, st.to_dict()

    def step_host(self, dt: float, tol: float, out: np.ndarray | None = None, raise_on_error: bool = True):
        out = np.zeros(self.node_shape) if out is None else out
        st = capi.SvnStats()
        rc = self.lib.svn_step_host(self.h, dt, tol, _host_out(out, self.nv), ctypes.byref(st))
        if rc != 0 and raise_on_error:
            self._check(rc)
        return out, st.to_dict()

    # -- time stepping of the coupled system --------------------------------
    def transport(self, dt: float) -> int:
        """Explicit upwind transport of the handle's h and A over dt with v^n;
        returns the number of sub-steps."""
        n = ctypes.c_int()
        self._check(self.lib.svn_transport(self.h, dt, ctypes.byref(n)))
        return n.value

    def ice(self):
        """Current (h, A) as device tensors of shape (N, N)."""
        import torch
        hc = torch.zeros((self.N, self.N), dtype=torch.float64, device="cuda")
        A = torch.zeros_like(hc)
        self._check(self.lib.svn_get_ice(self.h, _ptr(hc, self.nc, "h"), _ptr(A, self.nc, "A")))
        return hc, A

    def advance(self, dt: float, tol: float, wind=None, ocean=None, out=None, raise_on_error: bool = True):
        """One time step: transport of h and A with v^n, new wind / ocean
        (None keeps the current field), implicit momentum step; the solution
        becomes v^n of the next call.  Returns (v, stats with "substeps")."""
        out = self._vec() if out is None else out
        st = capi.SvnStats()
        n = ctypes.c_int()
        rc = self.lib.svn_advance(self.h, dt, tol, _ptr(wind, self.nv, "wind") if wind is not None else None,
                                  _ptr(ocean, self.nv, "ocean") if ocean is not None else None,
                                  _ptr(out, self.nv, "out"), ctypes.byref(st), ctypes.byref(n))
        if rc != 0 and raise_on_error:
            self._check(rc)
        d = st.to_dict()
        d["substeps"] = n.value
        return out, d

    def get_state(self):
        import torch
        v = self._vec()
        pi = torch.zeros(self.pi_shape, dtype=torch.float64, device="cuda")
        self._check(self.lib.svn_get_state(self.h, _ptr(v, self.nv, "v"), _ptr(pi, self.npi, "pi")))
        return v, pi

    def set_state(self, v, pi):
        self._check(self.lib.svn_set_state(self.h, _ptr(v, self.nv, "v"), _ptr(pi, self.npi, "pi")))

    # -- hot-path components ---------------------------------------------------
    def residual(self, dt: float, v):
        R = self._vec()
        nrm = ctypes.c_double()
        self._check(self.lib.svn_residual(self.h, dt, _ptr(v, self.nv, "v"), _ptr(R, self.nv, "R"),
                                          ctypes.byref(nrm)))
        return R, nrm.value

    def energy(self, dt: float, v, dv, alphas):
        k = len(alphas)
        al = (ctypes.c_double * k)(*alphas)
        phi = (ctypes.c_double * k)()
        scale = ctypes.c_double()
        self._check(self.lib.svn_energy(self.h, dt, _ptr(v, self.nv, "v"), _ptr(dv, self.nv, "dv"), al, k, phi,
                                        ctypes.byref(scale)))
        return list(phi), scale.value

    def linearize(self, dt: float, v, pi):
        self._check(self.lib.svn_linearize(self.h, dt, _ptr(v, self.nv, "v"), _ptr(pi, self.npi, "pi")))

    def apply(self, x, level: int = 0):
        import torch
        n = 2 * ((self.N >> level) + 1) ** 2 if level >= 0 else None
        y = torch.zeros_like(x)
        self._check(self.lib.svn_apply(self.h, level, _ptr(x, n, "x"), _ptr(y, n, "y")))
        return y

    def precondition(self, r):
        import torch
        z = torch.zeros_like(r)
        self._check(self.lib.svn_precondition(self.h, _ptr(r, self.nv, "r"), _ptr(z, self.nv, "z")))
        return z

    def krylov_solve(self, b, rtol: float):
        import torch
        x = torch.zeros_like(b)
        its = ctypes.c_int()
        self._check(self.lib.svn_krylov_solve(self.h, _ptr(b, self.nv, "b"), _ptr(x, self.nv, "x"), rtol,
                                              ctypes.byref(its)))
        return x, its.value

    # -- autotuner ---------------------------------------------------------------
    def autotune(self, dt: float, probe_newton: int = 4, degrees=(2, 3, 4, 6), los=(0.02, 0.05)):
        """Pick the fastest Chebyshev (degree, lo) for this grid and forcing."""
        d = (ctypes.c_int * len(degrees))(*degrees)
        l = (ctypes.c_double * len(los))(*los)
        best = ctypes.c_double()
        self._check(self.lib.svn_autotune(self.h, dt, probe_newton, d, len(degrees), l, len(los),
                                          ctypes.byref(best)))
        p = capi.SvnParams()
        self._check(self.lib.svn_get_params(self.h, ctypes.byref(p)))
        self.params = p
        return {"cheb_degree": p.cheb_degree, "cheb_lo": p.cheb_lo, "ms": best.value}

    def autotune_kernels(self, dt: float, probe_newton: int = 4, degrees=(4, 6), los=(0.02,), fuses=(1, 2, 4),
                         cache: str | None = None):
        """Pick the fastest (sweep kernel, Chebyshev degree, lo) for this grid and
        forcing.  With `cache` (a JSON file path), a result stored for this grid
        size and precision is applied without timing; a new one is stored."""
        import json
        import os
        key = "%d/%d" % (self.N, self.params.precision)
        if cache and os.path.exists(cache):
            with open(cache) as f:
                stored = json.load(f).get(key)
            if stored:
                self._check(self.lib.svn_set_smoother(self.h, stored["cheb_fuse"], stored["cheb_degree"],
                                                      stored["cheb_lo"]))
                p = capi.SvnParams()
                self._check(self.lib.svn_get_params(self.h, ctypes.byref(p)))
                self.params = p
                return dict(stored, cached=True)
        d = (ctypes.c_int * len(degrees))(*degrees)
        l = (ctypes.c_double * len(los))(*los)
        fz = (ctypes.c_int * len(fuses))(*fuses)
        best = ctypes.c_double()
        self._check(self.lib.svn_autotune_kernels(self.h, dt, probe_newton, d, len(degrees), l, len(los), fz,
                                                  len(fuses), ctypes.byref(best)))
        p = capi.SvnParams()
        self._check(self.lib.svn_get_params(self.h, ctypes.byref(p)))
        self.params = p
        res = {"cheb_fuse": p.cheb_fuse, "cheb_degree": p.cheb_degree, "cheb_lo": p.cheb_lo, "ms": best.value}
        if cache:
            data = {}
            if os.path.exists(cache):
                with open(cache) as f:
                    data = json.load(f)
            data[key] = res
            with open(cache, "w") as f:
                json.dump(data, f, indent=1)
        return dict(res, cached=False)

    # -- instrumentation -------------------------------------------------------
    def profile(self, enable: bool):
        self._check(self.lib.svn_profile(self.h, 1 if enable else 0))

    def profile_read(self, kclass: str):
        ms = ctypes.c_double()
        n = ctypes.c_longlong()
        self._check(self.lib.svn_profile_read(self.h, capi.KCLASS[kclass], ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    @staticmethod
    def kernel_launches() -> int:
        return int(capi.lib().svn_kernel_launches())

    def dual_update(self, dt: float, v, dv, alpha: float, pi):
        self._check(self.lib.svn_dual_update(self.h, dt, _ptr(v, self.nv, "v"), _ptr(dv, self.nv, "dv"), alpha,
                                             _ptr(pi, self.npi, "pi")))
        return pi


class Batch:
    """An ensemble of independent instances (any grid sizes), stepped concurrently."""

    def __init__(self, Ns, L: float = 512e3, host_threads: int = 8, **params):
        import torch
        self.lib = capi.lib()
        self.Ns = [int(n) for n in Ns]
        self.L = float(L)
        self.params = default_params(**params)
        grids = (capi.SvnGrid * len(self.Ns))(*[capi.SvnGrid(n, self.L) for n in self.Ns])
        h = ctypes.c_void_p()
        torch.cuda.current_stream().synchronize()
        rc = self.lib.svn_batch_create(len(self.Ns), grids, ctypes.byref(self.params), host_threads, ctypes.byref(h))
        self.b = h
        if rc != 0:
            msg = self.lib.svn_batch_last_error(h).decode() if h.value else ""
            if h.value:
                self.lib.svn_batch_destroy(h)
            self.b = None
            raise SvnError(rc, msg)
        self.handles = [ctypes.c_void_p(self.lib.svn_batch_instance(self.b, i)) for i in range(len(self.Ns))]

    def close(self):
        if getattr(self, "b", None):
            self.lib.svn_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_forcing(self, i, h, A, wind, ocean, v_old):
        import torch
        torch.cuda.current_stream().synchronize()      # inputs are read on the instance's own stream
        N = self.Ns[i]
        nc, nv = N * N, 2 * (N + 1) ** 2
        rc = self.lib.svn_set_forcing(self.handles[i], _ptr(h, nc, "h"), _ptr(A, nc, "A"), _ptr(wind, nv, "wind"),
                                      _ptr(ocean, nv, "ocean"), _ptr(v_old, nv, "v_old"))
        if rc != 0:
            raise SvnError(rc, self.lib.svn_last_error(self.handles[i]).decode())

    def step(self, dt: float, tol: float, outs=None):
        import torch
        n = len(self.Ns)
        if outs is None:
            outs = [torch.zeros((N + 1, N + 1, 2), dtype=torch.float64, device="cuda") for N in self.Ns]
        torch.cuda.current_stream().synchronize()
        if len(outs) != n:
            raise ValueError("outs: expected %d buffers, got %d" % (n, len(outs)))
        ptrs = (ctypes.c_void_p * n)(*[_ptr(o, 2 * (N + 1) ** 2, "outs[%d]" % i)
                                       for i, (o, N) in enumerate(zip(outs, self.Ns))])
        stats = (capi.SvnStats * n)()
        rc = self.lib.svn_batch_step(self.b, dt, tol, ptrs, stats)
        if rc != 0:
            raise SvnError(rc, self.lib.svn_batch_last_error(self.b).decode())
        return outs, [s.to_dict() for s in stats]


class Q2Solver:
    """One svN solver on Q2 (biquadratic) velocity elements: N x N cells, node
    vectors on the (2N+1)^2 grid, dual state (N, N, 9, 3)."""

    def __init__(self, N: int, L: float = 512e3, stream=None, **params):
        import torch
        self.N, self.L = int(N), float(L)
        self.nc, self.nv, self.npi = self.N * self.N, 2 * (2 * self.N + 1) ** 2, 27 * self.N * self.N
        self.lib = capi.lib()
        self.params = default_params(**params)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        g = capi.SvnGrid(self.N, self.L)
        h = ctypes.c_void_p()
        rc = self.lib.svn_q2_create(ctypes.byref(g), ctypes.byref(self.params),
                                    ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        self.h = h
        if rc != 0:
            msg = self.lib.svn_q2_last_error(h).decode() if h.value else ""
            if h.value:
                self.lib.svn_q2_destroy(h)
            self.h = None
            raise SvnError(rc, msg)

    def close(self):
        if getattr(self, "h", None):
            self.lib.svn_q2_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc: int):
        if rc != 0:
            raise SvnError(rc, self.lib.svn_q2_last_error(self.h).decode())

    @property
    def node_shape(self):
        return (2 * self.N + 1, 2 * self.N + 1, 2)

    @property
    def pi_shape(self):
        return (self.N, self.N, 9, 3)

    def _vec(self):
        import torch
        return torch.zeros(self.node_shape, dtype=torch.float64, device="cuda")

    def set_forcing(self, h, A, wind, ocean, v_old):
        self._check(self.lib.svn_q2_set_forcing(self.h, _ptr(h, self.nc, "h"), _ptr(A, self.nc, "A"),
                                                _ptr(wind, self.nv, "wind"), _ptr(ocean, self.nv, "ocean"),
                                                _ptr(v_old, self.nv, "v_old")))

    def step(self, dt: float, tol: float, out=None, raise_on_error: bool = True):
        out = self._vec() if out is None else out
        st = capi.SvnStats()
        rc = self.lib.svn_q2_step(self.h, dt, tol, _ptr(out, self.nv, "out"), ctypes.byref(st))
        if rc != 0 and raise_on_error:
            self._check(rc)
        return out, st.to_dict()

    def residual(self, dt: float, v):
        R = self._vec()
        nrm = ctypes.c_double()
        self._check(self.lib.svn_q2_residual(self.h, dt, _ptr(v, self.nv, "v"), _ptr(R, self.nv, "R"),
                                             ctypes.byref(nrm)))
        return R, nrm.value

    def energy(self, dt: float, v, dv, alphas):
        k = len(alphas)
        al = (ctypes.c_double * k)(*alphas)
        phi = (ctypes.c_double * k)()
        scale = ctypes.c_double()
        self._check(self.lib.svn_q2_energy(self.h, dt, _ptr(v, self.nv, "v"), _ptr(dv, self.nv, "dv"), al, k, phi,
                                           ctypes.byref(scale)))
        return list(phi), scale.value

    def linearize(self, dt: float, v, pi):
        self._check(self.lib.svn_q2_linearize(self.h, dt, _ptr(v, self.nv, "v"), _ptr(pi, self.npi, "pi")))

    def apply(self, x):
        import torch
        y = torch.zeros_like(x)
        self._check(self.lib.svn_q2_apply(self.h, _ptr(x, self.nv, "x"), _ptr(y, self.nv, "y")))
        return y

    def dual_update(self, dt: float, v, dv, alpha: float, pi):
        self._check(self.lib.svn_q2_dual_update(self.h, dt, _ptr(v, self.nv, "v"), _ptr(dv, self.nv, "dv"), alpha,
                                                _ptr(pi, self.npi, "pi")))
        return pi

    def get_state(self):
        import torch
        v = self._vec()
        pi = torch.zeros(self.pi_shape, dtype=torch.float64, device="cuda")
        self._check(self.lib.svn_q2_get_state(self.h, _ptr(v, self.nv, "v"), _ptr(pi, self.npi, "pi")))
        return v, pi
