"""Pins of the oracle's learned-start network (no GPU).

  * the parameter layout [Cout][3 ky + kx][Cin] + torch conv2d equals a
    brute-force loop over pixels and taps (zero padding)
  * autograd gradients equal central finite differences (FP64)
  * features: constant fields give the scaled constants; prolongation of a
    linear cell-centred field is exact away from the clamped border.
"""
import numpy as np
import torch

from oracle import unet


def test_conv_layout_brute_force():
    rng = np.random.default_rng(0)
    ci, co, G = 16, 32, 5
    w = rng.standard_normal(co * 9 * ci)
    b = rng.standard_normal(co)
    x = rng.standard_normal((ci, G, G))
    W = torch.as_tensor(w).reshape(co, 3, 3, ci).permute(0, 3, 1, 2)
    y = torch.nn.functional.conv2d(torch.as_tensor(x)[None], W, torch.as_tensor(b), padding=1)[0].numpy()
    ref = np.zeros((co, G, G))
    wr = w.reshape(co, 9, ci)
    for o in range(co):
        for yy in range(G):
            for xx in range(G):
                s = b[o]
                for tap in range(9):
                    sy, sx = yy + tap // 3 - 1, xx + tap % 3 - 1
                    if 0 <= sy < G and 0 <= sx < G:
                        s += wr[o, tap] @ x[:, sy, sx]
                ref[o, yy, xx] = s
    assert np.abs(y - ref).max() < 1e-12


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    G = 16
    p = unet.he_init(3).astype(np.float64)
    p[-sum(co for _, co, _ in unet.LAYERS):] = 0.1 * rng.standard_normal(sum(co for _, co, _ in unet.LAYERS))
    X = rng.standard_normal((2, 16, G, G))
    T = rng.standard_normal((2, 2, G, G))
    loss, g = unet.loss_and_grads(p, X, T)
    for idx in rng.choice(len(p), size=6, replace=False):
        e = np.zeros_like(p)
        e[idx] = 1e-6
        lp, _ = unet.loss_and_grads(p + e, X, T)
        lm, _ = unet.loss_and_grads(p - e, X, T)
        fd = (lp - lm) / 2e-6
        assert abs(fd - g[idx]) <= 1e-5 * max(abs(g).max(), 1e-12), (idx, fd, g[idx])


def test_features_and_prolongation_closed_forms():
    N, G = 16, 8
    h = np.full((N, N), 1.4)
    A = np.full((N, N), 0.95)
    wind = np.tile([3.0, -6.0], (N + 1, N + 1, 1))
    ocean = np.tile([0.05, 0.02], (N + 1, N + 1, 1))
    vold = np.zeros((N + 1, N + 1, 2))
    X = unet.features(N, G, h, A, wind, ocean, vold)
    assert np.allclose(X[0], 0.7) and np.allclose(X[1], 0.5)
    assert np.allclose(X[2], 0.2) and np.allclose(X[3], -0.4)
    assert np.allclose(X[4], 0.5) and np.allclose(X[5], 0.2)
    assert np.allclose(X[6:], 0.0)
    # a linear field in cell-centre coordinates is reproduced at interior nodes
    Gc = 8
    yy, xx = np.meshgrid(np.arange(Gc) + 0.5, np.arange(Gc) + 0.5, indexing="ij")
    Y = np.stack([0.3 + 0.1 * xx - 0.05 * yy, -0.2 + 0.02 * xx + 0.07 * yy])
    out = unet.prolong(Y, 4 * Gc)
    for j in range(3, 4 * Gc - 2):
        for i in range(3, 4 * Gc - 2):
            x, y = i / 4.0, j / 4.0
            assert abs(out[j, i, 0] - 0.2 * (0.3 + 0.1 * x - 0.05 * y)) < 1e-12
            assert abs(out[j, i, 1] - 0.2 * (-0.2 + 0.02 * x + 0.07 * y)) < 1e-12
