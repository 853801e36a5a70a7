"""PyTorch view of the likelihood: the NLL as a differentiable function.

TDMixNLL.apply(params, ctx) returns the NLL as a 0-d float64 tensor; its
backward multiplies the incoming gradient by the gradient the library's
adjoint kernel computed in the same evaluation (d NLL / d params for the
coefficients, resonance masses and widths, x and y).  Parameters on a CUDA
device stay there (stream-ordered evaluation); CPU tensors go through host
buffers.
"""
from __future__ import annotations

import numpy as np
import torch

from .tdmix import TDMix


class TDMixNLL(torch.autograd.Function):
    @staticmethod
    def forward(fctx, params: torch.Tensor, tdmix: TDMix):
        if params.dtype != torch.float64 or params.dim() != 1 or params.numel() != tdmix.n_params:
            raise ValueError("params must be a 1-d float64 tensor with one entry per model parameter")
        if params.is_cuda:
            p = params.detach().contiguous()
            out = torch.empty(1, dtype=torch.float64, device=p.device)
            grad = torch.empty(tdmix.n_params, dtype=torch.float64, device=p.device)
            tdmix.nll_device(p, out, grad)
            value = out[0]
        else:
            v, g = tdmix.nll(params.detach().numpy(), grad=True)
            value = torch.tensor(v, dtype=torch.float64)
            grad = torch.from_numpy(g)
        fctx.save_for_backward(grad)
        return value

    @staticmethod
    def backward(fctx, g):
        (grad,) = fctx.saved_tensors
        return g * grad, None


def nll(params: torch.Tensor, tdmix: TDMix) -> torch.Tensor:
    """Differentiable NLL of `tdmix` at `params`."""
    return TDMixNLL.apply(params, tdmix)


def as_numpy_objective(tdmix: TDMix):
    """(f, grad) callable on NumPy vectors for minimisers."""
    def fg(p: np.ndarray):
        v, g = tdmix.nll(p, grad=True)
        return v, g
    return fg
