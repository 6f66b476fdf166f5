"""Plain numpy definition of the learned-guess network (test infrastructure).

A fully convolutional net of 3x3 convolutions with zero 'same' padding and dilation d:
    y[b, o, i, j] = bias[o] + sum_{c, ky, kx} W[o, c, ky, kx] x[b, c, i + d (ky-1), j + d (kx-1)]
ReLU after every layer but the last.  Loss: mean squared error over masked pixels,
    L = sum(mask (pred - target)^2) / sum(mask).
Backward written from the definition (the input gradient is the correlation of the output
gradient with the flipped kernel; the weight gradient correlates the output gradient with the
shifted input).  Adam follows Kingma & Ba (2015).  Pinned by finite differences and by a
hand-computed delta response in tests/test_oracle_net.py.
"""
from __future__ import annotations

import numpy as np


def conv2d(x, w, b, d):
    B, C, H, W = x.shape
    O = w.shape[0]
    xp = np.pad(x, ((0, 0), (0, 0), (d, d), (d, d)))
    out = np.zeros((B, O, H, W))
    for ky in range(3):
        for kx in range(3):
            patch = xp[:, :, ky * d:ky * d + H, kx * d:kx * d + W]
            out += np.einsum("oc,bchw->bohw", w[:, :, ky, kx], patch)
    return out + b[None, :, None, None]


def conv2d_backward(x, w, d, gout):
    """Gradients (gx, gw, gb) of sum(gout * conv2d(x, w, b, d))."""
    B, C, H, W = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (d, d), (d, d)))
    gxp = np.zeros_like(xp)
    gw = np.zeros_like(w)
    for ky in range(3):
        for kx in range(3):
            sl = (slice(None), slice(None), slice(ky * d, ky * d + H), slice(kx * d, kx * d + W))
            gw[:, :, ky, kx] = np.einsum("bohw,bchw->oc", gout, xp[sl])
            gxp[sl] += np.einsum("oc,bohw->bchw", w[:, :, ky, kx], gout)
    gx = gxp[:, :, d:d + H, d:d + W]
    gb = gout.sum(axis=(0, 2, 3))
    return gx, gw, gb


def forward(params, dils, x):
    """params: list of (W, b); returns the list of layer outputs (post-activation)."""
    acts = [x]
    h = x
    for li, ((w, b), d) in enumerate(zip(params, dils)):
        h = conv2d(h, w, b, d)
        if li < len(params) - 1:
            h = np.maximum(h, 0.0)
        acts.append(h)
    return acts


def loss_and_grad(params, dils, x, target, mask):
    acts = forward(params, dils, x)
    pred = acts[-1]
    msum = mask.sum()
    diff = (pred - target) * mask
    loss = (diff * diff).sum() / msum
    g = 2.0 * diff / msum
    grads = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        if li < len(params) - 1:
            g = g * (acts[li + 1] > 0)
        w, b = params[li]
        gx, gw, gb = conv2d_backward(acts[li], w, dils[li], g)
        grads[li] = (gw, gb)
        g = gx
    return loss, grads


def adam_update(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
