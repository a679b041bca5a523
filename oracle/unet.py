"""Plain PyTorch CPU forward/backward of the learned-start network.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  The paper has no
learned component; this is the reference for the network the library trains
on the GPU (see the "Learned initial guess" block of include/svn.h):

  * 4-level U-Net on a G x G cell grid: per level two 3x3 convolutions
    (zero padding 1) + ReLU with 32, 64, 128, 256 channels, 2x2 average
    pooling between levels, nearest-neighbour x2 upsampling and channel
    concatenation [upsampled, skip] on the way up, a 3x3 head to 16 channels
    of which channels 0 and 1 are the velocity / 0.2 m/s;
  * inputs: block averages over the N/G x N/G cells of an N-cell problem of
    h / 2, (A - 0.9) / 0.1 (cells) and of wind / 15, ocean / 0.1,
    v_old / 0.2 (nodes of the block, v_old zero on the boundary), padded to
    16 channels with zeros;
  * loss 0.5 mean over pixels and the two used channels of (out - target)^2,
    target = mean of the velocity over each cell's four corner nodes / 0.2;
  * parameter vector: each convolution's weights as [Cout][3 ky + kx][Cin] in
    layer order, then all biases in layer order.

Computed in FP64 with torch.nn.functional primitives (conv2d, avg_pool2d,
interpolate, cat) as steps; autograd supplies the gradients.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as F

# (cin, cout, relu) per convolution, in order; shapes of the U-Net tensors
LAYERS = [(16, 32, True), (32, 32, True), (32, 64, True), (64, 64, True), (64, 128, True), (128, 128, True),
          (128, 256, True), (256, 256, True), (384, 128, True), (128, 128, True), (192, 64, True), (64, 64, True),
          (96, 32, True), (32, 32, True), (32, 16, False)]
SCALES = dict(h=2.0, A_off=0.9, A=0.1, wind=15.0, ocean=0.1, v=0.2)


def num_params():
    return sum(co * 9 * ci for ci, co, _ in LAYERS) + sum(co for _, co, _ in LAYERS)


def split_params(p):
    """Parameter vector -> list of (weight (Cout, Cin, 3, 3), bias (Cout,)) torch tensors."""
    p = torch.as_tensor(np.asarray(p, dtype=np.float64))
    ws, off = [], 0
    for ci, co, _ in LAYERS:
        w = p[off:off + co * 9 * ci].reshape(co, 3, 3, ci).permute(0, 3, 1, 2)   # [co][ky][kx][ci] -> OIHW
        ws.append(w)
        off += co * 9 * ci
    out = []
    for (ci, co, _), w in zip(LAYERS, ws):
        out.append((w, p[off:off + co]))
        off += co
    return out


def he_init(seed: int) -> np.ndarray:
    """He-normal weights, zero biases, from a seeded generator (an input, not method arithmetic)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = [rng.standard_normal(co * 9 * ci) * np.sqrt(2.0 / (9 * ci)) for ci, co, _ in LAYERS]
    parts += [np.zeros(co) for _, co, _ in LAYERS]
    return np.concatenate(parts).astype(np.float32)


def features(N, G, h, A, wind, ocean, v_old):
    """(16, G, G) network input from a problem on N x N cells (N = f G)."""
    f = N // G
    hb = h.reshape(G, f, G, f).mean(axis=(1, 3))
    Ab = A.reshape(G, f, G, f).mean(axis=(1, 3))
    vo = np.array(v_old, dtype=np.float64)
    vo[0], vo[-1], vo[:, 0], vo[:, -1] = 0, 0, 0, 0

    def node_block(u):
        out = np.empty((G, G, 2))
        for J in range(G):
            for I in range(G):
                out[J, I] = u[J * f:(J + 1) * f + 1, I * f:(I + 1) * f + 1].reshape(-1, 2).mean(axis=0)
        return out

    w, o, v = node_block(wind), node_block(ocean), node_block(vo)
    X = np.zeros((16, G, G))
    X[0] = hb / SCALES["h"]
    X[1] = (Ab - SCALES["A_off"]) / SCALES["A"]
    X[2:4] = np.moveaxis(w, -1, 0) / SCALES["wind"]
    X[4:6] = np.moveaxis(o, -1, 0) / SCALES["ocean"]
    X[6:8] = np.moveaxis(v, -1, 0) / SCALES["v"]
    return X


def target(v):
    """(2, N, N) cell-centred training target from node velocity (N+1, N+1, 2)."""
    vv = np.array(v, dtype=np.float64)
    vv[0], vv[-1], vv[:, 0], vv[:, -1] = 0, 0, 0, 0
    c = 0.25 * (vv[:-1, :-1] + vv[1:, :-1] + vv[:-1, 1:] + vv[1:, 1:])
    return np.moveaxis(c, -1, 0) / SCALES["v"]


def forward(params, X):
    """U-Net forward; X: (B, 16, G, G) -> (B, 16, G, G)."""
    P = split_params(params) if not isinstance(params, list) else params
    x = torch.as_tensor(X, dtype=torch.float64)

    def conv(k, t):
        w, b = P[k]
        y = F.conv2d(t, w, b, padding=1)
        return F.relu(y) if LAYERS[k][2] else y

    e1 = conv(1, conv(0, x))
    e2 = conv(3, conv(2, F.avg_pool2d(e1, 2)))
    e3 = conv(5, conv(4, F.avg_pool2d(e2, 2)))
    b = conv(7, conv(6, F.avg_pool2d(e3, 2)))
    up = lambda t: F.interpolate(t, scale_factor=2, mode="nearest")
    d3 = conv(9, conv(8, torch.cat([up(b), e3], 1)))
    d2 = conv(11, conv(10, torch.cat([up(d3), e2], 1)))
    d1 = conv(13, conv(12, torch.cat([up(d2), e1], 1)))
    return conv(14, d1)


def loss_and_grads(params, X, T):
    """0.5 mean((out[:, :2] - T)^2) and its gradient w.r.t. the parameter vector."""
    p = torch.tensor(np.asarray(params, dtype=np.float64), requires_grad=True)
    out = forward(split_params_tensor(p), X)
    d = out[:, :2] - torch.as_tensor(T, dtype=torch.float64)
    loss = 0.5 * (d * d).mean()
    loss.backward()
    return float(loss.detach()), p.grad.numpy()


def split_params_tensor(p):
    ws, off = [], 0
    for ci, co, _ in LAYERS:
        ws.append(p[off:off + co * 9 * ci].reshape(co, 3, 3, ci).permute(0, 3, 1, 2))
        off += co * 9 * ci
    out = []
    for (ci, co, _), w in zip(LAYERS, ws):
        out.append((w, p[off:off + co]))
        off += co
    return out


def prolong(Y, N):
    """Cell-centred prediction (2, G, G) -> node velocity (N+1, N+1, 2) [m/s]:
    bilinear in the cell-centre lattice, clamped at the outer half cell, zero
    on the boundary."""
    G = Y.shape[-1]
    out = np.zeros((N + 1, N + 1, 2))
    for j in range(1, N):
        for i in range(1, N):
            cx = min(max(i * G / N - 0.5, 0.0), G - 1.0)
            cy = min(max(j * G / N - 0.5, 0.0), G - 1.0)
            x0, y0 = min(int(np.floor(cx)), G - 2), min(int(np.floor(cy)), G - 2)
            tx, ty = cx - x0, cy - y0
            for c in range(2):
                out[j, i, c] = SCALES["v"] * ((1 - ty) * ((1 - tx) * Y[c, y0, x0] + tx * Y[c, y0, x0 + 1])
                                              + ty * ((1 - tx) * Y[c, y0 + 1, x0] + tx * Y[c, y0 + 1, x0 + 1]))
    return out
