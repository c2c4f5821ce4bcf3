"""Architecture comparison of Sec. 7 (Fig. 10) on synthetic records, through the C ABI.

The progressive residual network (Sec. 4.3) against two plain MLPs that take the whole
descriptor in the first layer -- shallow-wide (hidden widths 400, 400, 200, 200, 200) and
deep-narrow (22 hidden layers of 200) -- trained with Adam on the same minibatches of the
same records, validation log-MSE recorded every `eval_every` steps.  All arithmetic runs in
the library (rpnn_train_step, rpnn_dense_train_step, their forwards); this module sequences
the calls.
"""
from __future__ import annotations

import numpy as np
import torch

from . import api
from . import workloads as W


def _val_loss_dense(ctx, widths, params, desc, label, batch=8192):
    tot = 0.0
    for i in range(0, desc.shape[0], batch):
        g = ctx.dense_forward(widths, params, desc[i:i + batch])
        r = torch.log1p(g.double()) - torch.log1p(label[i:i + batch].double())
        tot += float((r * r).sum())
    return tot / desc.shape[0]


def compare(ctx: api.Context, train, val, steps: int = 300, batch: int = 1024, lr: float = 1e-3,
            eval_every: int = 100, seed: int = 0):
    """Returns {name: [(step, validation loss), ...]} for "rpnn", "shallow_wide" and
    "deep_narrow", and the parameter counts."""
    from . import train as T
    z, t = train
    zv, tv = val
    din = z[0].numel()
    g = torch.Generator(device="cpu").manual_seed(seed)
    order = [torch.randint(0, z.shape[0], (batch,), generator=g).to(z.device) for _ in range(steps)]
    out, counts = {}, {}
    # the progressive network
    p = torch.from_numpy(W.he_init(seed=11)).cuda()
    p.mul_(0.5)
    counts["rpnn"] = p.numel()
    m, v = torch.zeros_like(p), torch.zeros_like(p)
    ctx.set_weights(p)
    curve = [(0, T.val_loss(ctx, zv, tv))]
    for s, idx in enumerate(order, 1):
        ctx.train_step(z[idx].contiguous(), t[idx].contiguous(), p, m, v, s, lr=lr)
        if s % eval_every == 0:
            curve.append((s, T.val_loss(ctx, zv, tv)))
    out["rpnn"] = curve
    # the plain MLPs on the whole descriptor
    for name, widths in (("shallow_wide", W.SHALLOW_WIDE), ("deep_narrow", W.DEEP_NARROW)):
        p = torch.from_numpy(W.dense_he_init(widths, din, seed=11)).cuda()
        p.mul_(0.5)
        counts[name] = p.numel()
        m, v = torch.zeros_like(p), torch.zeros_like(p)
        curve = [(0, _val_loss_dense(ctx, widths, p, zv, tv))]
        for s, idx in enumerate(order, 1):
            ctx.dense_train_step(widths, z[idx].contiguous(), t[idx].contiguous(), p, m, v, s, lr=lr)
            if s % eval_every == 0:
                curve.append((s, _val_loss_dense(ctx, widths, p, zv, tv)))
        out[name] = curve
    return out, counts
