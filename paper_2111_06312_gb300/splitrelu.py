"""Split-ReLU graph network of Sec. 5.2, initialised from the SVD solution.

    message passing   H_{l+1} = [Â H_l Wp_l]_+ - [Â H_l Wn_l]_+,   H_0 = X
    output            H = sum_{l=0..L} [H_l Wop_l]_+ - [H_l Won_l]_+
    initialisation    Wp_l = I, Wn_l = -I, Wop_l = W*[dl : d(l+1)], Won_l = -Wop_l

With that start every Split-ReLU layer is linear (relu(t) - relu(-t) = t), so
the network equals the linear model [X | ÂX | ... | Â^L X] W* of Eq. 6 (Thm. 2)
and fine-tuning by cross-entropy starts from the closed-form fit.

The propagation Â H and its adjoint Â^T dH are the library's sparse products
(isvd_apply / isvd_apply_T on the operator N = Â); the d x d and d x y weight
products and the ReLUs are PyTorch's (dense library GEMMs and elementwise ops).
"""
from __future__ import annotations

import torch

from . import isvd
from .adjoint import implicit_matmul


def split_relu(X: torch.Tensor, Wp: torch.Tensor, Wn: torch.Tensor) -> torch.Tensor:
    """[X Wp]_+ - [X Wn]_+ (Sec. 5.2): linear in X when Wp = -Wn."""
    return torch.relu(X @ Wp) - torch.relu(X @ Wn)


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
