"""Comparisons of Sec. 7 (Fig. 10) on synthetic records, through the C ABI.

compare(): the progressive residual network (Sec. 4.3) against two plain MLPs that take the
whole descriptor in the first layer -- shallow-wide (hidden widths 400, 400, 200, 200, 200)
and deep-narrow (22 hidden layers of 200).
compare_stencils(): the progressive network fed by stencils of several resolutions over the
standard extent (n x n x (2n - 1) points; 5 x 5 x 9 is the paper's choice), each extracted
for the same records (positions, directions, lights and labels).
Every variant is trained with Adam on the same minibatches of the same records, validation
log-MSE recorded every `eval_every` steps.  All arithmetic runs in the library
(rpnn_train_step, rpnn_dense_train_step, rpnn_stencil_*, their forwards); this module
sequences the calls.
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


def stencil_records(ctx: api.Context, clouds, n_per_cloud: int, resolutions, seed: int = 1000,
                    rel_ci: float = 0.05, n_min: int = 32, n_max: int = 1024):
    """Path-traced records (Sec. 5.1) of each cloud with one descriptor set per stencil
    resolution: ({n: desc [N, 10, din(n)]}, label [N])."""
    descs = {n: [] for n in resolutions}
    labels = []
    for ci, dens in enumerate(clouds):
        vol = ctx.load_volume(torch.from_numpy(np.ascontiguousarray(dens)).cuda())
        ctx.build_mips(vol)
        x, d, wl, lab, _ = ctx.gen_records(vol, 0, n_per_cloud, seed + 7919 * ci, rel_ci, n_min, n_max)
        for n in resolutions:
            descs[n].append(ctx.stencil_descriptors(vol, n, x, d, wl))
        labels.append(lab)
        ctx.sync_status()
    return {n: torch.cat(v) for n, v in descs.items()}, torch.cat(labels)


def _val_loss_stencil(ctx, n, params, desc, label, batch=8192):
    tot = 0.0
    for i in range(0, desc.shape[0], batch):
        g = ctx.stencil_forward(n, params, desc[i:i + batch])
        r = torch.log1p(g.double()) - torch.log1p(label[i:i + batch].double())
        tot += float((r * r).sum())
    return tot / desc.shape[0]


def compare_stencils(ctx: api.Context, descs: dict, label, train_frac: float = 0.75, steps: int = 300,
                     batch: int = 1024, lr: float = 1e-3, eval_every: int = 100, seed: int = 0):
    """Trains the progressive network once per stencil resolution in `descs` (from
    stencil_records) on the same split and minibatches.  Returns ({n: [(step, validation
    loss), ...]}, {n: parameter count})."""
    N = label.shape[0]
    g = torch.Generator(device="cpu").manual_seed(seed)
    perm = torch.randperm(N, generator=g).to(label.device)
    n_tr = int(round(train_frac * N))
    tr, va = perm[:n_tr], perm[n_tr:]
    order = [tr[torch.randint(0, n_tr, (batch,), generator=g).to(label.device)] for _ in range(steps)]
    t_va = label[va].contiguous()
    out, counts = {}, {}
    for n, z in descs.items():
        din = z.shape[2]
        p = torch.from_numpy(W.he_init(seed=11, din=din)).cuda()
        p.mul_(0.5)
        counts[n] = p.numel()
        assert counts[n] == ctx.stencil_param_count(n)
        m, v = torch.zeros_like(p), torch.zeros_like(p)
        z_va = z[va].contiguous()
        curve = [(0, _val_loss_stencil(ctx, n, p, z_va, t_va))]
        for s, idx in enumerate(order, 1):
            ctx.stencil_train_step(n, z[idx].contiguous(), label[idx].contiguous(), p, m, v, s, lr=lr)
            if s % eval_every == 0:
                curve.append((s, _val_loss_stencil(ctx, n, p, z_va, t_va)))
        out[n] = curve
    return out, counts
