"""Linear model on the implicit CONCAT matrix (Eq. 6, Sec. 3.3) on the GPU:
forward M W and backward M^T dY through autograd, against the FP64 oracle;
the closed-form start W* = V S^+ U^T Y (Thm. 1).  Dense features X (n x 128,
N(0,1)), Â normalisation, L = 2, 40 outputs: the ogbn-arxiv-sized shapes.
Tolerances (FP32): forward within 1e-5 and gradient within 1e-4 of the
output scale; closed form within 1e-5."""
import numpy as np
import pytest
import torch

import oracle
from paper_2111_06312_gb300 import adjoint, build, isvd, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    build.build()
    oracle.build()


def npy(t):
    return t.double().cpu().numpy()


def _ops(g, x):
    dev = torch.device("cuda")
    gop = isvd.Operator(g.n, g.rowptr, g.colidx, form="concat", norm="sym", X=x, L=2, device=dev)
    oop = oracle.graph_operator(g, form="concat", norm="sym", X=x.astype(np.float64), L=2)
    return gop, oop


@pytest.fixture(scope="module")
def sub():
    g, x, y, train = synth.workload_finetune_sub(2000)
    gop, oop = _ops(g, x)
    yield g, x, y, train, gop, oop
    gop.close()


@pytest.fixture(scope="module")
def full():
    g, x, y, train = synth.workload_finetune()
    gop, oop = _ops(g, x)
    yield g, x, y, train, gop, oop
    gop.close()


def _fwd_bwd(gop, W0, dY):
    W = W0.clone().requires_grad_(True)
    Y = adjoint.implicit_matmul(gop, W)
    (Y * dY).sum().backward()
    return Y.detach(), W.grad


@pytest.mark.parametrize("case", ["sub", "full"])
def test_forward_and_gradient_match_oracle(case, request):
    g, x, y, train, gop, oop = request.getfixturevalue(case)
    r, c = gop.shape
    assert (r, c) == (g.n, 3 * 128)
    gen = torch.Generator().manual_seed(7)
    W0 = (torch.randn((c, 40), generator=gen) * 0.1).cuda()
    dY = torch.randn((r, 40), generator=gen).cuda()
    Y, dW = _fwd_bwd(gop, W0, dY)
    Y_ref = oop.apply(npy(W0))
    dW_ref = oop.apply(npy(dY), transpose=True)
    assert np.abs(npy(Y) - Y_ref).max() <= 1e-5 * np.abs(Y_ref).max()
    assert np.abs(npy(dW) - dW_ref).max() <= 1e-4 * np.abs(dW_ref).max()


def test_adjoint_identity(sub):
    *_, gop, _ = sub
    r, c = gop.shape
    gen = torch.Generator().manual_seed(8)
    W = torch.randn((c, 16), generator=gen).cuda()
    H = torch.randn((r, 16), generator=gen).cuda()
    lhs = float((gop.apply(W).double() * H.double()).sum())
    rhs = float((W.double() * gop.apply(H, transpose=True).double()).sum())
    scale = float(gop.apply(W).double().norm() * H.double().norm())
    assert abs(lhs - rhs) <= 1e-5 * scale


def test_closed_form_matches_oracle(sub):
    g, x, y, train, gop, _ = sub
    labels = torch.as_tensor(y).cuda()
    mask = torch.as_tensor(train).cuda()
    Ylab = adjoint.one_hot_train(labels, mask, 40)
    W, (U, S, V, info) = adjoint.closed_form_init(gop, Ylab, k=40, oversample=10, iters=4, seed=3)
    assert isvd.info_dict(info)["status"] == "OK"
    W_ref = oracle.closed_form(npy(U), npy(S), npy(V), npy(Ylab))
    assert np.abs(npy(W) - W_ref).max() <= 1e-5 * np.abs(W_ref).max()


def test_closed_form_small_shapes_and_rcond(sub):
    """Ragged k and m (not multiples of the 32-wide tiles) and a cut-off that
    zeroes the smallest singular values."""
    *_, gop, _ = sub
    r, c = gop.shape
    gen = torch.Generator().manual_seed(9)
    for k, m in [(1, 1), (33, 7), (70, 65)]:
        U = torch.randn((r, k), generator=gen).cuda()
        V = torch.randn((c, k), generator=gen).cuda()
        S = torch.sort(torch.rand(k, generator=gen) + 1e-3, descending=True).values.cuda()
        Y = torch.randn((r, m), generator=gen).cuda()
        rc = 0.5
        W = isvd.closed_form(gop, U, S, V, Y, rcond=rc)
        W_ref = oracle.closed_form(npy(U), npy(S), npy(V), npy(Y), rcond=rc)
        assert np.abs(npy(W) - W_ref).max() <= 1e-5 * max(np.abs(W_ref).max(), 1e-30)


def test_finetune_from_closed_form_lowers_the_loss(sub):
    """A few epochs of gradient descent from W* on the training rows (the
    fine-tuning step that follows the closed form) lower the cross-entropy."""
    g, x, y, train, gop, _ = sub
    labels = torch.as_tensor(y).cuda()
    mask = torch.as_tensor(train).cuda()
    Ylab = adjoint.one_hot_train(labels, mask, 40)
    W0, _ = adjoint.closed_form_init(gop, Ylab, k=40, oversample=10, iters=4, seed=3)
    model = adjoint.ImplicitLinear(gop, W0)
    opt = torch.optim.Adam(model.parameters(), lr=1e-2)
    idx = torch.nonzero(mask).reshape(-1)
    losses = []
    for _ in range(6):
        opt.zero_grad()
        loss = torch.nn.functional.cross_entropy(model()[idx], labels[idx])
        loss.backward()
        opt.step()
        losses.append(float(loss.detach()))
    assert losses[-1] < losses[0]


def test_dense_contractions_run_on_tensor_cores(full):
    """The dense contractions of the fine-tuning step (Sec. 3.3, Eq. 6 with
    dense X): the forward X [W_0 | W_1 | W_2] and the weight gradient
    X^T [dY | N dY | N^2 dY] run on the tcgen05 kernels (the Q.B product and
    the A^T B contraction), and so do the closed form's U^T Y and V Z (Thm.
    1): the CUDA-core fallbacks are not launched."""
    from torch.profiler import ProfilerActivity, profile

    g, x, y, train, gop, oop = full
    W = torch.randn((384, 40), device="cuda")
    dY = torch.randn((g.n, 40), device="cuda")
    U, S, V, _ = gop.svd(40, 10, 2, 5)
    Yl = torch.randn((g.n, 40), device="cuda")
    torch.cuda.synchronize()
    with profile(activities=[ProfilerActivity.CUDA]) as prof:
        gop.apply(W)
        gop.apply(dY, transpose=True)
        isvd.closed_form(gop, U, S, V, Yl)
        torch.cuda.synchronize()
    names = [e.key for e in prof.key_averages()]
    assert any("gemm_tc_kernel" in k for k in names), names
    assert any("gram_ab_tc_kernel" in k for k in names), names
    assert not any("tn_partial_kernel" in k or "gemm_small_kernel" in k for k in names), names
