"""The RPNN (Sec. 4.3) as a differentiable PyTorch operation over the library's own
hand-written forward and backward kernels (Sec. 5.2 trains it by backpropagation).

    g = rpnn(params, z, ctx)      # params: [1,296,601] FP32, z: [Q][10][240] descriptors

The arithmetic follows the context's training precision (``ctx.set_train_precision``):
FP32 (the default) runs the FP32 CUDA-core forward on FP32 descriptors; BF16 runs the
tcgen05 tensor-core forward (BF16 operands, FP32 accumulation) on BF16 descriptors.  The
backward runs ``rpnn_mlp_backward`` in the same precision and returns dL/dparams (the
descriptor is an input of the data, so no gradient flows to it).  Both calls go through the
C ABI; there is no PyTorch arithmetic on the network path.  In BF16 the gradient is that of
the training GEMMs' forward, which rounds the same operands to BF16 as the inference kernel
but adds the biases in FP32 (the inference kernel carries them in the MMA as BF16), so the
two forwards agree to BF16 rounding, not bit for bit.
"""
from __future__ import annotations

import torch

from . import api


class RPNNFunction(torch.autograd.Function):
    @staticmethod
    def forward(fctx, params: torch.Tensor, desc: torch.Tensor, lib: "api.Context") -> torch.Tensor:
        bf16 = lib.train_precision == api.BF16
        want = torch.bfloat16 if bf16 else torch.float32
        if desc.dtype != want:
            raise TypeError(f"rpnn: {'BF16' if bf16 else 'FP32'} training takes {want} descriptors")
        p = params.detach().contiguous()
        lib.set_weights(p)
        g = lib.mlp_forward(desc.contiguous(), precision=api.BF16 if bf16 else api.F32)
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
