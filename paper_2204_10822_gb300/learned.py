"""Learned Newton initial guess: binding of the svn_net C ABI and the trainer.

The network, its loss, gradients and Adam updates all run in the library's
CUDA kernels; this module only moves arguments.  Training pairs are produced
by the solver itself: trajectories of implicit steps (translating vortex over
fixed ice), each pair (h, A, wind at t_{n+1}, ocean, v^n) -> v^{n+1}.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import capi
from .solver import Solver, SvnError, _ptr


class Net:
    """U-Net on a G x G cell grid with `batch` training slots."""

    def __init__(self, G: int = 256, batch: int = 8, stream=None):
        import torch
        self.lib = capi.lib()
        self.G, self.batch = G, batch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        rc = self.lib.svn_net_create(G, batch, ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        self.h = h
        if rc != 0:
            msg = self.lib.svn_net_last_error(h).decode() if h.value else ""
            if h.value:
                self.lib.svn_net_destroy(h)
            self.h = None
            raise SvnError(rc, msg)
        self.nparam = int(self.lib.svn_net_num_params(self.h))

    def close(self):
        if getattr(self, "h", None):
            self.lib.svn_net_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != 0:
            raise SvnError(rc, self.lib.svn_net_last_error(self.h).decode())

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        if p.size != self.nparam:
            raise ValueError("params: expected %d float32 values, got %d" % (self.nparam, p.size))
        self._check(self.lib.svn_net_set_params(self.h, p.ctypes.data, self.nparam))

    def get_params(self):
        p = np.empty(self.nparam, dtype=np.float32)
        self._check(self.lib.svn_net_get_params(self.h, p.ctypes.data, self.nparam))
        return p

    def grads(self):
        g = np.empty(self.nparam, dtype=np.float32)
        self._check(self.lib.svn_net_get_grads(self.h, g.ctypes.data, self.nparam))
        return g

    def set_sample(self, slot, N, h, A, wind, ocean, v_old, v_target=None):
        import torch
        torch.cuda.current_stream().synchronize()
        nc, nv = N * N, 2 * (N + 1) ** 2
        self._check(self.lib.svn_net_set_sample(self.h, slot, N, _ptr(h, nc, "h"), _ptr(A, nc, "A"),
                                                _ptr(wind, nv, "wind"), _ptr(ocean, nv, "ocean"),
                                                _ptr(v_old, nv, "v_old"),
                                                _ptr(v_target, nv, "v_target") if v_target is not None else None))

    def forward(self, nb):
        out = np.empty((nb, self.G, self.G, 16), dtype=np.float32)
        self._check(self.lib.svn_net_forward(self.h, nb, out.ctypes.data))
        return out

    def train_step(self, nb, lr, apply=True):
        loss = ctypes.c_float()
        self._check(self.lib.svn_net_train_step(self.h, nb, lr, 1 if apply else 0, ctypes.byref(loss)))
        return float(loss.value)

    def attach(self, solver: Solver, on: bool = True):
        solver._check(self.lib.svn_attach_net(solver.h, self.h))
        solver._check(self.lib.svn_set_learned(solver.h, 1 if on else 0))


def he_init(seed: int, nparam: int | None = None) -> np.ndarray:
    """He-normal initial weights (std sqrt(2 / (9 Cin))), zero biases, seeded."""
    layers = [(16, 32), (32, 32), (32, 64), (64, 64), (64, 128), (128, 128), (128, 256), (256, 256),
              (384, 128), (128, 128), (192, 64), (64, 64), (96, 32), (32, 32), (32, 16)]
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = [rng.standard_normal(co * 9 * ci) * math.sqrt(2.0 / (9 * ci)) for ci, co in layers]
    parts += [np.zeros(co) for _, co in layers]
    p = np.concatenate(parts).astype(np.float32)
    assert nparam is None or p.size == nparam
    return p


def generate_pairs(G: int, n_traj: int, steps: int, seed0: int, dt: float = 1800.0, **solver_kw):
    """Solver-generated training pairs on G x G cells (device tensors)."""
    import torch

    import workloads as W
    L = 512e3
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    s = Solver(G, L, **solver_kw)
    pairs, stats = [], []
    ocean = t(W.ocean_gyre(G, L))
    for k in range(n_traj):
        seed = seed0 + k
        h, A = W.ice_fields(G, L, seed)
        hd, Ad = t(h), t(A)
        v = torch.zeros((G + 1, G + 1, 2), dtype=torch.float64, device="cuda")
        for n in range(steps):
            wind = t(W.rankine_vortex(G, L, W.translating_centre(L, seed, (n + 1) * dt)))
            s.set_forcing(hd, Ad, wind, ocean, v)
            vn, st = s.step(dt, 1e-8, raise_on_error=False)
            stats.append(st)
            if st["status"] != "SVN_OK":
                break
            pairs.append(dict(h=hd, A=Ad, wind=wind, ocean=ocean, v_old=v, v=vn.clone()))
            v = vn.clone()
    s.close()
    return pairs, stats


def train(net: Net, pairs, epochs: int, lr: float = 1e-3, seed: int = 0, lr_final: float | None = None):
    """Adam on minibatches of `net.batch` pairs; cosine learning-rate decay."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = len(pairs)
    losses = []
    total = epochs * max(1, n // net.batch)
    step = 0
    lr_final = lr * 0.05 if lr_final is None else lr_final
    for _ in range(epochs):
        order = rng.permutation(n)
        for b0 in range(0, n - net.batch + 1, net.batch):
            idx = order[b0:b0 + net.batch]
            for slot, i in enumerate(idx):
                q = pairs[i]
                net.set_sample(slot, net.G, q["h"], q["A"], q["wind"], q["ocean"], q["v_old"], q["v"])
            a = lr_final + 0.5 * (lr - lr_final) * (1 + math.cos(math.pi * step / max(total, 1)))
            losses.append(net.train_step(len(idx), a))
            step += 1
    return losses
