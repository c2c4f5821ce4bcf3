"""CPU reference of the mixed-precision training arithmetic (test infrastructure).

The network of Sec. 4.3 and its chain rule (Sec. 5.2) in FP64 with torch's CPU autograd,
where every 200-wide layer's GEMM takes its two operands rounded to BF16 (round to nearest
even) in the forward and in both backward products -- the activation, the weight and the
incoming gradient -- exactly where the BF16 training kernels round them; biases, residual
sums, ReLU masks and the 1-wide output layer stay unrounded.  With rounding off it is the
plain FP64 network, which tests/test_oracle_mlp.py checks against the oracle."""
import numpy as np
import torch

from paper_1709_05418_gb300 import workloads as W


def _round(t, on):
    return t.to(torch.bfloat16).to(torch.float64) if on else t


class _Product(torch.autograd.Function):
    """a @ w^T with a [rows][K], w [N][K]; operands and incoming gradient rounded."""

    @staticmethod
    def forward(ctx, a, w, on):
        ctx.save_for_backward(a, w)
        ctx.on = on
        return _round(a, on) @ _round(w, on).T

    @staticmethod
    def backward(ctx, g):
        a, w = ctx.saved_tensors
        gb = _round(g, ctx.on)
        return gb @ _round(w, ctx.on), gb.T @ _round(a, ctx.on), None


def forward_backward(params, z, dout, bf16=True):
    """(g [q], flat parameter gradient of sum_i dout_i g_i), FP64 numpy."""
    P = W.split_params(np.asarray(params, np.float64))
    T = {k: torch.tensor(v, requires_grad=True) for k, v in P.items()}
    zz = torch.tensor(np.asarray(z, np.float64))
    o = None
    for k in range(1, 11):
        pre = _Product.apply(zz[:, k - 1, :], T[f"V{k}"], bf16)
        if o is not None:
            pre = pre + _Product.apply(o, T[f"W1_{k}"], bf16)
        f1 = torch.relu(pre + T[f"b1_{k}"])
        h = _Product.apply(f1, T[f"W2_{k}"], bf16) + T[f"b2_{k}"]
        if o is not None:
            h = h + o
        o = torch.relu(h)
    t0 = torch.relu(_Product.apply(o, T["T1"], bf16) + T["bT1"])
    t1 = torch.relu(_Product.apply(t0, T["T2"], bf16) + T["bT2"])
    g = torch.relu(t1 @ T["T3"].T + T["bT3"]).squeeze(1)
    (g * torch.tensor(np.asarray(dout, np.float64))).sum().backward()
    grads = {k: T[k].grad.numpy() for k in T}
    return g.detach().numpy(), W.join_params(grads)
