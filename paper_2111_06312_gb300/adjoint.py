"""Gradients through the implicit design matrix (Sec. 3.3: the linear model
Y = M W on M = [X | N X | ... | N^L X], Eq. 6, is fine-tuned by gradient
descent from the closed-form start W* of Thm. 1).

The forward product M W and the backward product dW = M^T dY are the
library's isvd_apply / isvd_apply_T (right-to-left evaluation: X W_l first,
then the Horner chain over N); nothing is materialised.  PyTorch only
provides the autograd plumbing, the tensors and the stream.
"""
from __future__ import annotations

import torch

from . import isvd


class _ImplicitMatmul(torch.autograd.Function):
    """Y = M W with dL/dW = M^T dL/dY (M is a constant of the graph)."""

    @staticmethod
    def forward(ctx, W: torch.Tensor, op: isvd.Operator) -> torch.Tensor:
        if W.dtype != torch.float32:
            raise TypeError("implicit_matmul takes FP32 weights")
        ctx.op = op
        return op.apply(W.detach())

    @staticmethod
    def backward(ctx, dY: torch.Tensor):
        return ctx.op.apply(dY.detach().float(), transpose=True), None


def implicit_matmul(op: isvd.Operator, W: torch.Tensor) -> torch.Tensor:
    """M W for an implicit operator ``op`` (c x b weights -> r x b outputs)."""
    return _ImplicitMatmul.apply(W, op)


class ImplicitLinear(torch.nn.Module):
    """Linear model on the implicit design matrix: forward() = M W."""

    def __init__(self, op: isvd.Operator, W0: torch.Tensor):
        super().__init__()
        self.op = op
        self.weight = torch.nn.Parameter(W0.detach().clone().contiguous())

    def forward(self) -> torch.Tensor:
        return implicit_matmul(self.op, self.weight)


def one_hot_train(labels: torch.Tensor, train_mask: torch.Tensor, classes: int) -> torch.Tensor:
    """Y_lab: one-hot rows for training nodes, zero rows elsewhere (FP32)."""
    Y = torch.zeros((labels.numel(), classes), dtype=torch.float32, device=labels.device)
    idx = torch.nonzero(train_mask, as_tuple=False).reshape(-1)
    Y[idx, labels[idx]] = 1.0
    return Y


def closed_form_init(op: isvd.Operator, Y_lab: torch.Tensor, k: int, oversample: int = 10, iters: int = 4,
                     seed: int = 0, rcond: float = 1e-6):
    """W* = V S^+ U^T Y_lab from a rank-k iSVD of M (Alg. 1, then Thm. 1)."""
    U, S, V, info = op.svd(k, oversample, iters, seed=seed)
    W = isvd.closed_form(op, U, S, V, Y_lab, rcond=rcond)
    return W, (U, S, V, info)
