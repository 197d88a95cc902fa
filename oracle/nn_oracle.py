"""FP64 reference of the warm-start network -- TEST INFRASTRUCTURE.

Plain numpy restatement of the encoder-decoder the CUDA library trains
(3x3 convolutions with zero padding, 2x2 average pooling, nearest 2x
upsampling, additive skips, ReLU, linear head) and of its gradients, for
checking the library's forward and backward kernels.  Only tests and the
benchmark's CPU leg import it.  Pinned by finite differences
(tests/test_oracle_pins.py::test_nn_oracle_gradients_match_finite_differences).

Parameter layout (same flat order as the library): for each of the 15
convolutions, W[cout][cin][3][3] then b[cout].
"""
from __future__ import annotations

import numpy as np

LAYERS = [(2, 32), (32, 32), (32, 64), (64, 64), (64, 128), (128, 128), (128, 128), (128, 128),
          (128, 128), (128, 128), (128, 64), (64, 64), (64, 32), (32, 32), (32, 1)]


def param_count():
    return sum(co * ci * 9 + co for ci, co in LAYERS)


def unpack(p):
    out, o = [], 0
    for ci, co in LAYERS:
        W = p[o:o + co * ci * 9].reshape(co, ci, 3, 3)
        o += co * ci * 9
        b = p[o:o + co]
        o += co
        out.append((W, b))
    return out


def conv(X, W, b):
    c, H, Wd = X.shape
    Xp = np.pad(X, ((0, 0), (1, 1), (1, 1)))
    Y = np.zeros((W.shape[0], H, Wd))
    for ky in range(3):
        for kx in range(3):
            Y += np.einsum("oc,chw->ohw", W[:, :, ky, kx], Xp[:, ky:ky + H, kx:kx + Wd])
    return Y + b[:, None, None]


def conv_bwd(X, W, dY):
    c, H, Wd = X.shape
    Xp = np.pad(X, ((0, 0), (1, 1), (1, 1)))
    dXp = np.zeros_like(Xp)
    dW = np.zeros_like(W)
    for ky in range(3):
        for kx in range(3):
            dW[:, :, ky, kx] = np.einsum("ohw,chw->oc", dY, Xp[:, ky:ky + H, kx:kx + Wd])
            dXp[:, ky:ky + H, kx:kx + Wd] += np.einsum("oc,ohw->chw", W[:, :, ky, kx], dY)
    return dXp[:, 1:-1, 1:-1], dW, dY.sum(axis=(1, 2))


def pool(X):
    return 0.25 * (X[:, 0::2, 0::2] + X[:, 1::2, 0::2] + X[:, 0::2, 1::2] + X[:, 1::2, 1::2])


def pool_bwd(dY):
    return 0.25 * np.repeat(np.repeat(dY, 2, axis=1), 2, axis=2)


def up(X):
    return np.repeat(np.repeat(X, 2, axis=1), 2, axis=2)


def up_bwd(dY):
    return dY[:, 0::2, 0::2] + dY[:, 1::2, 0::2] + dY[:, 0::2, 1::2] + dY[:, 1::2, 1::2]


def relu(x):
    return np.maximum(x, 0.0)


def features(occ, goal):
    H, W = occ.shape
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    d = np.hypot(xx - goal[0], yy - goal[1]) / np.hypot(H, W)
    return np.stack([(occ != 0).astype(np.float64), d])


def forward(p, occ, goal):
    L = unpack(np.asarray(p, np.float64))
    c = {"x": features(occ, goal)}
    e = []
    h = c["x"]
    for l in range(4):
        if l > 0:
            c[f"p{l}"] = pool(e[-1][1])
            h = c[f"p{l}"]
        a = relu(conv(h, *L[2 * l]))
        bb = relu(conv(a, *L[2 * l + 1]))
        c[f"ea{l}"], c[f"pre_a{l}"] = a, None
        e.append((a, bb))
    prev = e[3][1]
    d = []
    for j in range(3):
        lvl = 2 - j
        uu = up(prev)
        a = relu(conv(uu, *L[8 + 2 * j]) + e[lvl][1])
        bb = relu(conv(a, *L[9 + 2 * j]))
        d.append((uu, a, bb))
        prev = bb
    out = conv(prev, *L[14])[0]
    c.update(e=e, d=d, L=L)
    return out, c


def loss_and_grads(p, occ, goal, target):
    out, c = forward(p, occ, goal)
    L, e, d = c["L"], c["e"], c["d"]
    H, W = occ.shape
    m = (occ == 0).astype(np.float64)
    m[goal[1], goal[0]] = 0.0
    n = m.sum()
    diff = (out - target) * m
    loss = float((diff * diff).sum() / n)
    grads = [None] * 15
    dout = (2.0 * diff / n)[None]
    dprev, gw, gb = conv_bwd(d[2][2], L[14][0], dout)
    grads[14] = (gw, gb)
    dskip = {}
    for j in (2, 1, 0):
        lvl = 2 - j
        uu, a, bb = d[j]
        dprev = dprev * (bb > 0)
        da, gw, gb = conv_bwd(a, L[9 + 2 * j][0], dprev)
        grads[9 + 2 * j] = (gw, gb)
        da = da * (a > 0)
        dskip[lvl] = da
        du, gw, gb = conv_bwd(uu, L[8 + 2 * j][0], da)
        grads[8 + 2 * j] = (gw, gb)
        dprev = up_bwd(du)
    for l in (3, 2, 1, 0):
        a, bb = e[l]
        if l in dskip:
            dprev = dprev + dskip[l]
        dprev = dprev * (bb > 0)
        da, gw, gb = conv_bwd(a, L[2 * l + 1][0], dprev)
        grads[2 * l + 1] = (gw, gb)
        da = da * (a > 0)
        xin = c["x"] if l == 0 else c[f"p{l}"]
        dx, gw, gb = conv_bwd(xin, L[2 * l][0], da)
        grads[2 * l] = (gw, gb)
        if l > 0:
            dprev = pool_bwd(dx)
    flat = np.concatenate([np.concatenate([gw.ravel(), gb]) for gw, gb in grads])
    return loss, flat
