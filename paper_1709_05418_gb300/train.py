"""Training pipeline of Sec. 5 on the GPU, driven through the C ABI.

records():  path-traced (descriptor, L_i) records (Sec. 5.1) from seeded clouds,
            descriptors extracted on the GPU with each record's own light direction.
split():    75 % / 25 % non-overlapping train / validation split (Sec. 5.1).
fit():      minibatch Adam on the log-MSE loss (Sec. 5.2) with the library's own
            forward / backward kernels (rpnn_train_step); returns the loss history.
save_checkpoint() / load_checkpoint(): the FP32 master parameters, Adam moments, step,
            training precision and the GEMM autotuner's decisions, so a resumed run repeats
            the next step bit for bit.
Every step of the arithmetic runs in the CUDA library; this module only sequences
calls and holds tensors.
"""
from __future__ import annotations

import numpy as np
import torch

from . import api
from . import workloads as W


def records(ctx: api.Context, clouds, n_per_cloud: int, seed: int = 1000, rel_ci: float = 0.02,
            n_min: int = 64, n_max: int = 4096, chunk: int = 8192, albedo: float = 0.99, hg_g: float = 0.85,
            dtype=torch.float32):
    """Returns (desc [N,10,240] of `dtype` (FP32, or BF16 at half the memory), label [N]) for
    `n_per_cloud` records of each cloud (a list of FP32 density grids, numpy [nz][ny][nx])."""
    descs, labels = [], []
    for ci, dens in enumerate(clouds):
        vol = ctx.load_volume(torch.from_numpy(np.ascontiguousarray(dens)).cuda(), albedo, hg_g)
        ctx.build_mips(vol)
        for first in range(0, n_per_cloud, chunk):
            n = min(chunk, n_per_cloud - first)
            x, d, wl, lab, _ = ctx.gen_records(vol, first, n, seed + 7919 * ci, rel_ci, n_min, n_max)
            z = ctx.extract_descriptors(vol, x, d, wl, dtype=dtype)
            descs.append(z)
            labels.append(lab)
        ctx.sync_status()
    return torch.cat(descs), torch.cat(labels)


def split(desc, label, seed: int = 0, train_frac: float = 0.75):
    g = torch.Generator(device="cpu").manual_seed(seed)
    perm = torch.randperm(desc.shape[0], generator=g).to(desc.device)
    n_tr = int(round(train_frac * desc.shape[0]))
    tr, va = perm[:n_tr], perm[n_tr:]
    return (desc[tr].contiguous(), label[tr].contiguous()), (desc[va].contiguous(), label[va].contiguous())


def val_loss(ctx: api.Context, desc, label, batch: int = 8192) -> float:
    tot, n = 0.0, 0
    for i in range(0, desc.shape[0], batch):
        z, t = desc[i:i + batch], label[i:i + batch]
        g = ctx.mlp_forward(z, precision=api.BF16 if z.dtype == torch.bfloat16 else api.F32)
        r = torch.log1p(g.double()) - torch.log1p(t.double())
        tot += float((r * r).sum())
        n += z.shape[0]
    return tot / max(n, 1)


def fit(ctx: api.Context, train, val, params: torch.Tensor, steps: int, batch: int = 4096,
        lr: float = 1e-3, seed: int = 0, eval_every: int = 50):
    """Adam on minibatches of the training split; params (FP32, device) is updated in
    place.  Returns [(step, train_loss, val_loss or None)]."""
    desc, label = train
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    ctx.set_weights(params)
    g = torch.Generator(device="cpu").manual_seed(seed)
    hist = []
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    perm = torch.randperm(desc.shape[0], generator=g)
    pos = 0
    for step in range(1, steps + 1):
        if pos + batch > desc.shape[0]:
            perm = torch.randperm(desc.shape[0], generator=g)
            pos = 0
        idx = perm[pos:pos + batch].to(desc.device)
        pos += batch
        zb, tb = desc[idx].contiguous(), label[idx].contiguous()
        ctx.train_step(zb, tb, params, m, v, step, lr=lr, loss=loss)
        if step % eval_every == 0 or step == steps:
            hist.append((step, float(loss.item()), val_loss(ctx, *val) if val is not None else None))
    return hist


def blob_clouds(n: int, size: int = 64, seed0: int = 100):
    return [W.blob_cloud(size, nblobs=8, seed=seed0 + i) for i in range(n)]


def save_checkpoint(path, ctx: api.Context, params: torch.Tensor, m: torch.Tensor, v: torch.Tensor,
                    step: int, precision=api.F32):
    """Writes the training state: parameters, Adam moments, the last step taken, the
    training precision and the autotuner's table (its split-K choices fix the order of the
    weight-gradient sums)."""
    torch.save({"params": params.detach().cpu(), "m": m.detach().cpu(), "v": v.detach().cpu(),
                "step": int(step), "precision": int(precision), "autotune": ctx.autotune_table()}, path)


def load_checkpoint(path, ctx: api.Context, device="cuda"):
    """Restores a checkpoint into ctx (weights, training precision, tuning decisions);
    returns (params, m, v, step) on the device -- the next step is step + 1."""
    st = torch.load(path, map_location="cpu")
    params = st["params"].to(device)
    m = st["m"].to(device)
    v = st["v"].to(device)
    ctx.set_autotune_table(st["autotune"])
    ctx.set_train_precision(st["precision"])
    ctx.set_weights(params)
    return params, m, v, st["step"]
