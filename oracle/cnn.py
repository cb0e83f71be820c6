"""CPU oracle of the subtree-level CNN (float64, numpy).

TEST INFRASTRUCTURE ONLY (like the rest of oracle/): the plain statement of
the network the GPU kernels train and run, used to check their forward
values and gradients.

Network: three 3x3 convolutions with zero padding (cross-correlation:
y[o, i, j] = b[o] + sum_{c, di, dj} w[o, c, di+1, dj+1] * x[c, i+di, j+dj]),
ReLU after the first two, softmax cross-entropy on the last (one class per
pixel), averaged over the pixels.  Arrays are channel-first per image:
x[batch, channel, row, col].

BF16 operands: the network's stated precision is BF16 weights and
activations with higher-precision accumulation.  `forward` and `backward`
take an optional rounding `rnd` (`bf16` below) applied to every operand of
a convolution that the network holds in BF16: the two hidden activations in
the forward pass, the loss gradient and the two masked hidden gradients in
the backward pass (the weights and the input are already BF16 values when
they are given).  Every other operation stays in float64.  Without `rnd`
the network is evaluated in plain float64.
"""
from __future__ import annotations

import numpy as np


def bf16(a):
    """Round to bfloat16 (1 sign, 8 exponent, 7 stored significand bits), as
    a float32 value is converted: to float32 first (nearest, ties to even),
    then the low 16 bits of the float32 pattern dropped with round to
    nearest, ties to even (finite inputs in float32's normal or subnormal
    range).  Returned as float64."""
    f = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    keep = (f + 0x7FFF + ((f >> 16) & 1)) & 0xFFFF0000
    return keep.astype(np.uint32).view(np.float32).astype(np.float64)


def _exact(a):
    return a


def conv3x3(x, w, b):
    """x [B, Cin, H, W], w [Cout, Cin, 3, 3], b [Cout] -> [B, Cout, H, W]."""
    B, C, H, W = x.shape
    xp = np.zeros((B, C, H + 2, W + 2))
    xp[:, :, 1:H + 1, 1:W + 1] = x
    y = np.zeros((B, w.shape[0], H, W)) + b[None, :, None, None]
    for di in range(3):
        for dj in range(3):
            patch = xp[:, :, di:di + H, dj:dj + W]                 # [B, C, H, W]
            y += np.einsum("oc,bchw->bohw", w[:, :, di, dj], patch)
    return y


def conv3x3_backward(x, w, dy):
    """Gradients of sum(dy * conv3x3(x, w, b)) w.r.t. x, w and b."""
    B, C, H, W = x.shape
    xp = np.zeros((B, C, H + 2, W + 2))
    xp[:, :, 1:H + 1, 1:W + 1] = x
    dw = np.zeros_like(w)
    dxp = np.zeros_like(xp)
    for di in range(3):
        for dj in range(3):
            patch = xp[:, :, di:di + H, dj:dj + W]
            dw[:, :, di, dj] = np.einsum("bohw,bchw->oc", dy, patch)
            dxp[:, :, di:di + H, dj:dj + W] += np.einsum("oc,bohw->bchw", w[:, :, di, dj], dy)
    db = dy.sum(axis=(0, 2, 3))
    return dxp[:, :, 1:H + 1, 1:W + 1], dw, db


def forward(params, x, rnd=None):
    """Returns (logits, cache); `rnd` rounds the hidden activations."""
    rnd = rnd or _exact
    w1, b1, w2, b2, w3, b3 = params
    z1 = conv3x3(x, w1, b1)
    a1 = rnd(np.maximum(z1, 0.0))
    z2 = conv3x3(a1, w2, b2)
    a2 = rnd(np.maximum(z2, 0.0))
    z3 = conv3x3(a2, w3, b3)
    return z3, (x, z1, a1, z2, a2)


def loss_and_dlogits(logits, labels):
    """Mean softmax cross-entropy over every pixel; labels [B, H, W] ints."""
    B, K, H, W = logits.shape
    m = logits.max(axis=1, keepdims=True)
    e = np.exp(logits - m)
    p = e / e.sum(axis=1, keepdims=True)
    onehot = np.zeros_like(p)
    for k in range(K):
        onehot[:, k] = labels == k
    npix = B * H * W
    loss = -np.sum(onehot * np.log(p)) / npix
    return loss, (p - onehot) / npix


def backward(params, cache, dlogits, rnd=None):
    """Gradients (dw1, db1, dw2, db2, dw3, db3) of the loss; `rnd` rounds
    the loss gradient and the masked hidden gradients."""
    rnd = rnd or _exact
    w1, b1, w2, b2, w3, b3 = params
    x, z1, a1, z2, a2 = cache
    da2, dw3, db3 = conv3x3_backward(a2, w3, rnd(dlogits))
    dz2 = rnd(da2 * (z2 > 0))
    da1, dw2, db2 = conv3x3_backward(a1, w2, dz2)
    dz1 = rnd(da1 * (z1 > 0))
    _, dw1, db1 = conv3x3_backward(x, w1, dz1)
    return dw1, db1, dw2, db2, dw3, db3


def init_params(rng, cin=4, ch=16, ncls=5):
    """He-style random initialisation."""
    def w(o, i):
        return rng.standard_normal((o, i, 3, 3)) * np.sqrt(2.0 / (9 * i))
    return [w(ch, cin), np.zeros(ch), w(ch, ch), np.zeros(ch), w(ncls, ch), np.zeros(ncls)]
