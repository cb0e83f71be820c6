"""Training data and training of the subtree CNN that drives the learned
subtree skip (the network predicts, per 16x16-finest subtree, the deepest
level the next step's threshold tree will need, and the subtree is encoded,
flagged and stored only down to it; see Sec. 2.1.2 for the significance
tree it stands in for).

Data come from simulations run on the GPU path itself: at sampled steps k
the input is the features of the state at t_k (level-(L-4) coefficients of
h, qx, qy, z over their s_max) and the label is the exact deepest level of
the closed threshold tree of the state at t_{k+1}.  Everything runs in the
library's kernels; this module only drives them.
"""
from __future__ import annotations

import numpy as np
import torch

from . import hwfv1 as H
from .sim import Simulation


def collect(cases, steps, every, warm=0, precision=64):
    """Run each (problem, fields) case for `steps` steps and, every `every`
    steps from step `warm` on, record (features(t_k), labels(t_{k+1})).

    Returns (x, y): x bf16 [n, S, S, 4] and y uint8 [n, S, S] on the GPU,
    S = 2^(L-4); every case must have the same L."""
    xs, ys = [], []
    for p, f in cases:
        sim = Simulation(p, f, precision=precision)
        S = 1 << (sim.L - 4)
        k = 0
        while k < steps:
            if k >= warm and (k - warm) % every == 0:
                sim.encode()
                sim.flag()
                x = torch.empty(S * S * 4, dtype=torch.bfloat16, device=sim.dev)
                sim.features_dev(x)
                sim.step()
                k += 1
                sim.encode()
                sim.flag()
                y = torch.empty(S * S, dtype=torch.uint8, device=sim.dev)
                sim.labels_dev(y)
                xs.append(x.view(S, S, 4))
                ys.append(y.view(S, S))
            else:
                n = every - ((k - warm) % every) if k >= warm else warm - k
                n = min(n, steps - k)
                sim.advance(max_steps=n)
                k += n
        sim.close()
    return torch.stack(xs), torch.stack(ys)


def augment(x, y):
    """The eight symmetries of the square, applied to samples x [n, S, S, 4]
    (rows j, columns i; channels h, qx, qy, z) and labels y [n, S, S].  The
    shallow-water equations are invariant under them when the momentum
    components follow: a mirror in i negates qx, a mirror in j negates qy,
    the transpose swaps qx and qy.  Returns 8n samples."""
    xs, ys = [], []
    for t in (0, 1):
        for fj in (0, 1):
            for fi in (0, 1):
                a, b = x, y
                if fi:
                    a, b = a.flip(2), b.flip(2)
                    a = a * torch.tensor([1, -1, 1, 1], dtype=a.dtype, device=a.device)
                if fj:
                    a, b = a.flip(1), b.flip(1)
                    a = a * torch.tensor([1, 1, -1, 1], dtype=a.dtype, device=a.device)
                if t:
                    a, b = a.transpose(1, 2)[..., [0, 2, 1, 3]], b.transpose(1, 2)
                xs.append(a.contiguous())
                ys.append(b.contiguous())
    return torch.cat(xs), torch.cat(ys)


def train(x, y, epochs=10, batch=8, lr=3e-3, seed=0, net=None):
    """Adam on mean softmax cross-entropy (BF16 tensor-core kernels).
    Returns (net handle, last mini-batch loss)."""
    if net is None:
        net = H.hwfv1_skipnet_create(seed)
    n, S = x.shape[0], x.shape[1]
    batch = max(1, min(batch, n))
    loss = H.hwfv1_skipnet_train(net, x.contiguous().view(-1), y.contiguous().view(-1), n, S, S, batch,
                                 epochs, lr, seed)
    return net, loss


def predict_levels(net, x, margin):
    """Predicted class (0..4 = deepest level - (L-4)) per pixel with the
    engine's rule: the smallest class whose cumulative probability reaches
    1 - margin.  Runs the network on the GPU; the rule is restated here in
    torch for reporting only."""
    n, S = x.shape[0], x.shape[1]
    logits = torch.empty(n * S * S * 16, dtype=torch.float32, device=x.device)
    H.hwfv1_skipnet_forward(net, x.contiguous().view(-1), n, S, S, logits)
    pr = torch.softmax(logits.view(n, S, S, 16)[..., :5], dim=-1)
    cum = pr.cumsum(-1)
    ok = cum[..., :4] >= 1.0 - margin
    cls = torch.where(ok.any(-1), ok.float().argmax(-1), torch.full_like(ok[..., 0], 4, dtype=torch.long))
    return cls.to(torch.uint8)


def under_prediction_rate(net, x, y, margin):
    """Fraction of subtrees whose predicted level is below the exact one."""
    return float((predict_levels(net, x, margin) < y).float().mean())
