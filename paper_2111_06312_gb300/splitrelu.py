"""Split-ReLU graph network of Sec. 5.2, initialised from the SVD solution.

    message passing   H_{l+1} = [Â H_l Wp_l]_+ - [Â H_l Wn_l]_+,   H_0 = X
    output            H = sum_{l=0..L} [H_l Wop_l]_+ - [H_l Won_l]_+
    initialisation    Wp_l = I, Wn_l = -I, Wop_l = W*[dl : d(l+1)], Won_l = -Wop_l

With that start every Split-ReLU layer is linear (relu(t) - relu(-t) = t), so
the network equals the linear model [X | ÂX | ... | Â^L X] W* of Eq. 6 (Thm. 2)
and fine-tuning by cross-entropy starts from the closed-form fit.

The propagation Â H and its adjoint Â^T dH are the library's sparse products
(isvd_apply / isvd_apply_T on the operator N = Â); every split-ReLU layer,
forward and backward, is the library's too (isvd_split_relu_forward /
_backward: the d x d and d x y weight products on the tensor cores, the ReLUs
and their masks in the same calls).  PyTorch holds the parameters, runs Adam
and the cross-entropy.
"""
from __future__ import annotations

import torch

from . import isvd
from .adjoint import implicit_matmul


class _SplitReLU(torch.autograd.Function):
    """Z = [X Wp]_+ - [X Wn]_+ through the library (forward keeps the two
    pre-activations for the backward)."""

    @staticmethod
    def forward(ctx, X, Wp, Wn):
        L = isvd.lib()
        X = isvd._as_block(X.detach().float())
        Wp_c = Wp.detach().float().contiguous()
        Wn_c = Wn.detach().float().contiguous()
        n, d = X.shape
        e = Wp_c.shape[1]
        Z = isvd.new_block(n, e, device=X.device)
        Ap = isvd.new_block(n, e, device=X.device)
        An = isvd.new_block(n, e, device=X.device)
        isvd._check(L.isvd_split_relu_forward(isvd._ptr(X), X.stride(0), n, d, isvd._ptr(Wp_c), isvd._ptr(Wn_c), e,
                                              isvd._ptr(Z), Z.stride(0), isvd._ptr(Ap), isvd._ptr(An), Ap.stride(0),
                                              isvd._stream()), "isvd_split_relu_forward")
        ctx.save_for_backward(X, Wp_c, Wn_c, Ap, An)
        return Z

    @staticmethod
    def backward(ctx, dZ):
        L = isvd.lib()
        X, Wp, Wn, Ap, An = ctx.saved_tensors
        n, d = X.shape
        e = Wp.shape[1]
        dZ = isvd._as_block(dZ.float())
        dX = isvd.new_block(n, d, device=X.device) if ctx.needs_input_grad[0] else None
        dWp = torch.empty((d, e), dtype=torch.float32, device=X.device)
        dWn = torch.empty((d, e), dtype=torch.float32, device=X.device)
        nbytes = int(L.isvd_split_relu_work_bytes(n, d, e))
        work = torch.empty(nbytes, dtype=torch.uint8, device=X.device)
        isvd._check(L.isvd_split_relu_backward(isvd._ptr(X), X.stride(0), n, d, isvd._ptr(Wp), isvd._ptr(Wn), e,
                                               isvd._ptr(Ap), isvd._ptr(An), Ap.stride(0), isvd._ptr(dZ), dZ.stride(0),
                                               isvd._ptr(dX), dX.stride(0) if dX is not None else 0, isvd._ptr(dWp),
                                               isvd._ptr(dWn), isvd._ptr(work), nbytes, isvd._stream()),
                    "isvd_split_relu_backward")
        return dX, dWp, dWn


def split_relu(X: torch.Tensor, Wp: torch.Tensor, Wn: torch.Tensor) -> torch.Tensor:
    """[X Wp]_+ - [X Wn]_+ (Sec. 5.2): linear in X when Wp = -Wn."""
    return _SplitReLU.apply(X, Wp, Wn)


class SplitReLUNet(torch.nn.Module):
    """L message-passing layers and L + 1 output heads (Sec. 5.2).

    prop: the operator Â (``isvd.graph_operator(g, norm='sym', coeffs=[1.0])``);
    X: n x d features (FP32, CUDA); W_star: d(L+1) x y closed-form weights of
    the linear model on [X | ÂX | ... | Â^L X] (Thm. 1)."""

    def __init__(self, prop: isvd.Operator, X: torch.Tensor, W_star: torch.Tensor, L: int):
        super().__init__()
        n, d = X.shape
        if prop.shape != (n, n):
            raise ValueError("prop must be the n x n operator Â")
        if W_star.shape[0] != d * (L + 1):
            raise ValueError(f"W_star needs d(L+1) = {d * (L + 1)} rows")
        self.prop = prop
        self.L = L
        self.register_buffer("X", X.detach().float().contiguous())
        eye = torch.eye(d, dtype=torch.float32, device=X.device)
        self.Wp = torch.nn.ParameterList([torch.nn.Parameter(eye.clone()) for _ in range(L)])
        self.Wn = torch.nn.ParameterList([torch.nn.Parameter(-eye.clone()) for _ in range(L)])
        Ws = W_star.detach().float()
        self.Wop = torch.nn.ParameterList(
            [torch.nn.Parameter(Ws[d * l:d * (l + 1)].clone().contiguous()) for l in range(L + 1)])
        self.Won = torch.nn.ParameterList(
            [torch.nn.Parameter(-Ws[d * l:d * (l + 1)].clone().contiguous()) for l in range(L + 1)])

    def forward(self) -> torch.Tensor:
        H = self.X
        out = split_relu(H, self.Wop[0], self.Won[0])
        for l in range(self.L):
            P = implicit_matmul(self.prop, H)  # Â H through the library's SpMM
            H = split_relu(P, self.Wp[l], self.Wn[l])
            out = out + split_relu(H, self.Wop[l + 1], self.Won[l + 1])
        return out


def finetune(net: SplitReLUNet, labels: torch.Tensor, train_mask: torch.Tensor, epochs: int = 10,
             lr: float = 1e-3) -> list:
    """Cross-entropy fine-tuning on the training rows (Sec. 5.2 after
    Sec. 2.2's objective) with Adam; returns the loss per epoch."""
    opt = torch.optim.Adam(net.parameters(), lr=lr)
    idx = torch.nonzero(train_mask, as_tuple=False).reshape(-1)
    hist = []
    for _ in range(epochs):
        opt.zero_grad(set_to_none=True)
        loss = torch.nn.functional.cross_entropy(net()[idx], labels[idx])
        loss.backward()
        opt.step()
        hist.append(float(loss.item()))
    return hist
