"""FP64 reference of the warm-start network (test infrastructure only).

The learned warm start is this project's addition to the method (the paper
iterates to convergence, Sec. V-C, and has no learned part). This module holds
the plain definition of the network the CUDA library trains, written in numpy
FP64 with its own forward and backward passes, so the GPU gradients can be
checked against it; its own backward is pinned by finite differences.

Parameter layout (shared convention with the library's C ABI, not code):
all conv weights W_l[co][ci][3][3] layer by layer, then all biases b_l[co].
Layers (C = base channels; 3x3 convs with zero padding, ReLU on all but the
last):
  0: 3->C, 1: C->C (skip s1), pool, 2: C->2C, 3: 2C->2C (skip s2), pool,
  4: 2C->2C, nearest up, concat [up, s2], 5: 4C->C, nearest up,
  concat [up, s1], 6: 2C->C, 7: C->1.
"""
from __future__ import annotations

import numpy as np


def layer_shapes(C: int):
    ci = [3, C, C, 2 * C, 2 * C, 4 * C, 2 * C, C]
    co = [C, C, 2 * C, 2 * C, 2 * C, C, C, 1]
    return list(zip(co, ci))


def unpack(params: np.ndarray, C: int):
    shapes = layer_shapes(C)
    Ws, bs, off = [], [], 0
    for co, ci in shapes:
        Ws.append(params[off:off + co * ci * 9].reshape(co, ci, 3, 3))
        off += co * ci * 9
    for co, _ in shapes:
        bs.append(params[off:off + co])
        off += co
    assert off == params.size
    return Ws, bs


def n_params(C: int) -> int:
    return sum(co * ci * 9 + co for co, ci in layer_shapes(C))


def conv(x, W, b):
    """out[b,o,y,x] = b[o] + sum_c,ky,kx W[o,c,ky,kx] x[b,c,y+ky-1,x+kx-1] (zero pad)."""
    H = x.shape[2]
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    out = np.zeros((x.shape[0], W.shape[0], H, H))
    for ky in range(3):
        for kx in range(3):
            out += np.einsum("oc,bchw->bohw", W[:, :, ky, kx], xp[:, :, ky:ky + H, kx:kx + H])
    return out + b[None, :, None, None]


def conv_grads(x, W, dout):
    """(dx, dW, db) of `conv` for upstream gradient dout."""
    H = x.shape[2]
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    dW = np.zeros_like(W)
    dxp = np.zeros_like(xp)
    for ky in range(3):
        for kx in range(3):
            dW[:, :, ky, kx] = np.einsum("bohw,bchw->oc", dout, xp[:, :, ky:ky + H, kx:kx + H])
            dxp[:, :, ky:ky + H, kx:kx + H] += np.einsum("oc,bohw->bchw", W[:, :, ky, kx], dout)
    return dxp[:, :, 1:-1, 1:-1], dW, dout.sum(axis=(0, 2, 3))


def pool(x):
    B, C, H, _ = x.shape
    return x.reshape(B, C, H // 2, 2, H // 2, 2).mean(axis=(3, 5))


def pool_grad(d):
    return np.repeat(np.repeat(d, 2, axis=2), 2, axis=3) / 4.0


def up(x):
    return np.repeat(np.repeat(x, 2, axis=2), 2, axis=3)


def up_grad(d):
    B, C, H, _ = d.shape
    return d.reshape(B, C, H // 2, 2, H // 2, 2).sum(axis=(3, 5))


def forward(params, C, x, keep=False):
    Ws, bs = unpack(params, C)
    relu = lambda z: np.maximum(z, 0.0)
    a1 = relu(conv(x, Ws[0], bs[0]))
    s1 = relu(conv(a1, Ws[1], bs[1]))
    p1 = pool(s1)
    a3 = relu(conv(p1, Ws[2], bs[2]))
    s2 = relu(conv(a3, Ws[3], bs[3]))
    p2 = pool(s2)
    a5 = relu(conv(p2, Ws[4], bs[4]))
    c1 = np.concatenate([up(a5), s2], axis=1)
    a6 = relu(conv(c1, Ws[5], bs[5]))
    c2 = np.concatenate([up(a6), s1], axis=1)
    a7 = relu(conv(c2, Ws[6], bs[6]))
    y = conv(a7, Ws[7], bs[7])
    if keep:
        return y, dict(x=x, a1=a1, s1=s1, p1=p1, a3=a3, s2=s2, p2=p2, a5=a5, c1=c1, a6=a6,
                       c2=c2, a7=a7)
    return y


def loss_and_grad(params, C, x, t):
    """MSE loss mean((y - t)^2) and its gradient with respect to params."""
    Ws, _ = unpack(params, C)
    y, a = forward(params, C, x, keep=True)
    loss = float(np.mean((y - t) ** 2))
    dy = 2.0 * (y - t) / y.size
    gW, gb = [None] * 8, [None] * 8
    da7, gW[7], gb[7] = conv_grads(a["a7"], Ws[7], dy)
    da7 = da7 * (a["a7"] > 0)
    dc2, gW[6], gb[6] = conv_grads(a["c2"], Ws[6], da7)
    C1 = a["a6"].shape[1]
    da6 = up_grad(dc2[:, :C1]) * (a["a6"] > 0)
    ds1 = dc2[:, C1:].copy()
    dc1, gW[5], gb[5] = conv_grads(a["c1"], Ws[5], da6)
    C2 = a["a5"].shape[1]
    da5 = up_grad(dc1[:, :C2]) * (a["a5"] > 0)
    ds2 = dc1[:, C2:].copy()
    dp2, gW[4], gb[4] = conv_grads(a["p2"], Ws[4], da5)
    ds2 = (ds2 + pool_grad(dp2)) * (a["s2"] > 0)
    da3, gW[3], gb[3] = conv_grads(a["a3"], Ws[3], ds2)
    da3 = da3 * (a["a3"] > 0)
    dp1, gW[2], gb[2] = conv_grads(a["p1"], Ws[2], da3)
    ds1 = (ds1 + pool_grad(dp1)) * (a["s1"] > 0)
    da1, gW[1], gb[1] = conv_grads(a["a1"], Ws[1], ds1)
    da1 = da1 * (a["a1"] > 0)
    _, gW[0], gb[0] = conv_grads(a["x"], Ws[0], da1)
    grad = np.concatenate([g.ravel() for g in gW] + [g.ravel() for g in gb])
    return loss, grad
