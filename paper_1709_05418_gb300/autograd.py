"""The RPNN (Sec. 4.3) as a differentiable PyTorch operation over the library's own
hand-written FP32 forward and backward kernels (Sec. 5.2 trains it by backpropagation).

    g = rpnn(params, z, ctx)      # params: [1,296,601] FP32, z: [Q][10][240] FP32 descriptors

The forward runs ``rpnn_mlp_forward`` with the given parameters; the backward runs
``rpnn_mlp_backward`` and returns dL/dparams (the descriptor is an input of the data, so no
gradient flows to it).  Both calls go through the C ABI; there is no PyTorch arithmetic on
the network path.
"""
from __future__ import annotations

import torch

from . import api


class RPNNFunction(torch.autograd.Function):
    @staticmethod
    def forward(fctx, params: torch.Tensor, desc: torch.Tensor, lib: "api.Context") -> torch.Tensor:
        if desc.dtype != torch.float32:
            raise TypeError("rpnn: training descriptors must be FP32")
        p = params.detach().contiguous()
        lib.set_weights(p)
        g = lib.mlp_forward(desc.contiguous(), precision=api.F32)
        fctx.save_for_backward(p, desc)
        fctx.lib = lib
        return g

    @staticmethod
    def backward(fctx, dg: torch.Tensor):
        p, desc = fctx.saved_tensors
        lib = fctx.lib
        lib.set_weights(p)                  # the library's weights may have changed since forward
        dp = lib.mlp_backward(desc.contiguous(), dg.detach().float().contiguous())
        return dp, None, None


def rpnn(params: torch.Tensor, desc: torch.Tensor, lib: "api.Context") -> torch.Tensor:
    """Network prediction g(z) for every row of ``desc``, differentiable in ``params``."""
    return RPNNFunction.apply(params, desc, lib)
