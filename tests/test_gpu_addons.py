"""Parity of the consumers and variants around the SVD with the FP64 oracle:
label re-use's adjacency Â - (D+I)^-1 (Sec. 5.3) in both operator forms, and
the network-embedding outputs L = U S^1/2, R = V S^1/2 with the pair scores
f(i, j) = <L_i, R_j> (Sec. 3.1).  Through the C ABI on the GPU."""
import numpy as np
import pytest
import torch

import oracle
from paper_2111_06312_gb300 import build, isvd, synth
from svd_checks import check_svd

pytestmark = pytest.mark.gpu
LAM = 0.05
C5 = oracle.ne_coefficients(5)
KERNELS = ["ring", "chunks", "rows", "slab"]


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    build.build()
    oracle.build()


def npy(t):
    return t.detach().double().cpu().numpy()


@pytest.fixture(scope="module")
def hub_graph():
    # hub rows above the split threshold; no self-loops (zero diagonal)
    return synth.chung_lu(3000, 24000, 78, max_degree=1500, isolated_self_loops=False)


# ---- Â - (D+I)^-1 --------------------------------------------------------------

@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("transpose", [False, True])
@pytest.mark.parametrize("b", [3, 42, 144])
def test_noself_poly_apply(hub_graph, kernel, transpose, b):
    g = hub_graph
    kw = dict(norm="sym_noself", coeffs=C5, ones_coeff=-LAM, adj_coeff=0.02)
    with isvd.graph_operator(g, **kw) as gpu:
        gpu.set_tuning(kernel=kernel, chunk_nnz=128)
        ref = oracle.graph_operator(g, **kw)
        G = isvd.gaussian(3, g.n, b)
        Y = gpu.apply(G, transpose=transpose)
        Yr = ref.apply(npy(G), transpose=transpose)
    assert np.abs(npy(Y) - Yr).max() <= 1e-5 * np.abs(Yr).max()


def test_noself_poly_apply_bf16(hub_graph):
    g = hub_graph
    kw = dict(norm="sym_noself", coeffs=C5, ones_coeff=-LAM)
    with isvd.graph_operator(g, **kw) as gpu:
        ref = oracle.graph_operator(g, **kw)
        G = isvd.gaussian(4, g.n, 72, dtype=torch.bfloat16)
        Y = gpu.apply(G)
        Yr = ref.apply(npy(G))
    assert np.abs(npy(Y) - Yr).max() <= 3e-2 * np.abs(Yr).max()


@pytest.mark.parametrize("dense", [False, True])
@pytest.mark.parametrize("transpose", [False, True])
def test_label_reuse_concat_apply(hub_graph, dense, transpose):
    """[Y | N0 Y | N0^2 Y] with N0 = Â - (D+I)^-1 and Y one-hot on the
    training rows (zero rows elsewhere), as dense or sparse X."""
    g = hub_graph
    classes = 7
    y, mask = synth.labels(g.n, classes, 0.5, 79)
    train = np.nonzero(mask)[0]
    Y = np.zeros((g.n, classes), np.float32)
    Y[train, y[train]] = 1.0
    if dense:
        Xg, Xo = Y, Y.astype(np.float64)
    else:
        rp = np.zeros(g.n + 1, np.int32)
        rp[1:] = np.cumsum(mask)
        ci = y[train].astype(np.int32)
        Xg = (classes, rp, ci, np.ones(len(ci), np.float32))
        Xo = (classes, rp, ci, np.ones(len(ci)))
    with isvd.graph_operator(g, form="concat", norm="sym_noself", X=Xg, L=2) as gpu:
        ref = oracle.graph_operator(g, form="concat", norm="sym_noself", X=Xo, L=2)
        r, c = gpu.shape
        assert (r, c) == ref.shape == (g.n, 3 * classes)
        G = isvd.gaussian(6, r if transpose else c, 19)
        out = gpu.apply(G, transpose=transpose)
        want = ref.apply(npy(G), transpose=transpose)
    assert np.abs(npy(out) - want).max() <= 1e-5 * np.abs(want).max()


def test_noself_svd(hub_graph):
    g = hub_graph
    kw = dict(norm="sym_noself", coeffs=C5, ones_coeff=-LAM)
    with isvd.graph_operator(g, **kw) as gpu:
        check_svd(gpu, oracle.graph_operator(g, **kw), 16, 10, 4, 80)


# ---- embeddings and pair scores ----------------------------------------------------

def test_embeddings_match_oracle(hub_graph):
    g = hub_graph
    with isvd.graph_operator(g, norm="sym", coeffs=C5, ones_coeff=-LAM) as gpu:
        U, S, V, _ = gpu.svd(24, 10, 3, 81)
    Lm, Rm = isvd.embeddings(U, S, V)
    Lr, Rr = oracle.embeddings(npy(U), npy(S), npy(V))
    for got, want in ((Lm, Lr), (Rm, Rr)):
        assert got.shape == want.shape
        assert np.all(np.abs(npy(got) - want) <= 3e-7 * np.abs(want))
    # in place: out == X
    Uc = U.clone()
    st = isvd.lib().isvd_embed(isvd._ptr(Uc), Uc.stride(0), Uc.shape[0], 24, isvd._ptr(S), isvd._ptr(Uc),
                               Uc.stride(0), isvd._stream())
    assert st == 0
    assert torch.equal(Uc, Lm)


@pytest.mark.parametrize("k", [1, 33, 144, 160])
def test_pair_scores_match_oracle(k):
    rows, cols, n_pairs = 3001, 2999, 20011
    rng = np.random.default_rng(82 + k)
    Lh = rng.standard_normal((rows, k)).astype(np.float32)
    Rh = rng.standard_normal((cols, k)).astype(np.float32)
    src = rng.integers(0, rows, n_pairs).astype(np.int32)
    dst = rng.integers(0, cols, n_pairs).astype(np.int32)
    src[:2] = (0, rows - 1)
    dst[:2] = (cols - 1, 0)
    Lm = isvd.new_block(rows, k)
    Rm = isvd.new_block(cols, k)
    Lm.copy_(torch.from_numpy(Lh))
    Rm.copy_(torch.from_numpy(Rh))
    f = isvd.pair_scores(Lm, Rm, torch.from_numpy(src), torch.from_numpy(dst))
    want = oracle.pair_scores(Lh, Rh, src, dst)
    bound = 1e-6 * np.sum(np.abs(Lh[src].astype(np.float64) * Rh[dst]), axis=1)
    assert np.all(np.abs(npy(f) - want) <= bound)
    assert torch.equal(f, isvd.pair_scores(Lm, Rm, torch.from_numpy(src), torch.from_numpy(dst)))


def test_pair_scores_flag_out_of_range_pairs():
    rows, cols, k = 500, 400, 16
    Lm = isvd.gaussian(1, rows, k)
    Rm = isvd.gaussian(2, cols, k)
    src = torch.tensor([0, -1, rows, 3, rows - 1], dtype=torch.int32)
    dst = torch.tensor([0, 5, 1, cols, cols - 1], dtype=torch.int32)
    info = torch.zeros(4, dtype=torch.int32, device="cuda")
    f = isvd.pair_scores(Lm, Rm, src, dst, info=info)
    bad = torch.tensor([False, True, True, True, False])
    assert torch.isnan(f.cpu()[bad]).all() and torch.isfinite(f.cpu()[~bad]).all()
    assert isvd.info_dict(info)["status"] == "INVALID_ARGUMENT"
    info.zero_()
    isvd.pair_scores(Lm, Rm, src[[0, 4]], dst[[0, 4]], info=info)
    assert isvd.info_dict(info)["status"] == "OK"
    assert isvd.pair_scores(Lm, Rm, src[:0], dst[:0]).numel() == 0


# ---- composite nodes (Sec. 4; label re-use and pseudo-dropout of Sec. 5.3) ------------

def _children(g, seed=90):
    """Leaves on both sides (GPU, oracle): two polynomials and two
    concatenations with the same sparse features."""
    x = synth.tfidf_features(g.n, 11, 0.05, seed)
    Xg = (x.d, x.rowptr, x.colidx, x.values)
    Xo = (x.d, x.rowptr, x.colidx, x.values.astype(np.float64))
    specs = [dict(coeffs=C5, ones_coeff=-LAM, norm="sym"),
             dict(norm="sym", coeffs=[0.3, -0.2], adj_coeff=0.05),
             dict(form="concat", norm="sym", L=2),
             dict(form="concat", norm="sym_noself", L=2)]
    gpu, ref = [], []
    for sp in specs:
        if sp.get("form") == "concat":
            gpu.append(isvd.graph_operator(g, X=Xg, **sp))
            ref.append(oracle.graph_operator(g, X=Xo, **sp))
        else:
            gpu.append(isvd.graph_operator(g, **sp))
            ref.append(oracle.graph_operator(g, **sp))
    return gpu, ref


def _tree(lib, kind, a, b, c, d):
    if kind == "sum":
        return lib.compose("sum", [a, b], [0.5, -2.0])
    if kind == "hcat":
        return lib.compose("hcat", [a, c, d])
    if kind == "vcat":
        return lib.compose("vcat", [c, lib.compose("product", [b, d])])
    if kind == "product":
        return lib.compose("product", [a, b, c])
    # nested: [[A | C] ; [B | C]] + weights
    return lib.compose("vcat", [lib.compose("hcat", [a, c]), lib.compose("hcat", [lib.compose("sum", [b, a], [1.0, 0.25]), c])])


@pytest.fixture(scope="module")
def children(hub_graph):
    gpu, ref = _children(hub_graph)
    yield gpu, ref
    for o in gpu:
        o.close()


@pytest.mark.parametrize("kind", ["sum", "hcat", "vcat", "product", "nested"])
@pytest.mark.parametrize("transpose", [False, True])
@pytest.mark.parametrize("b", [5, 42])
def test_composite_apply(children, kind, transpose, b):
    gpu, ref = children
    cg = _tree(isvd, kind, *gpu)
    co = _tree(oracle, kind, *ref)
    assert cg.shape == co.shape
    r, c = cg.shape
    G = isvd.gaussian(9, r if transpose else c, b)
    Y = cg.apply(G, transpose=transpose)
    Yr = co.apply(npy(G), transpose=transpose)
    assert np.abs(npy(Y) - Yr).max() <= 1e-5 * np.abs(Yr).max()
    cg.close()


def test_composite_apply_bf16(children):
    gpu, ref = children
    cg = _tree(isvd, "nested", *gpu)
    co = _tree(oracle, "nested", *ref)
    G = isvd.gaussian(10, cg.shape[1], 24, dtype=torch.bfloat16)
    Y = cg.apply(G)
    Yr = co.apply(npy(G))
    assert np.abs(npy(Y) - Yr).max() <= 3e-2 * np.abs(Yr).max()
    cg.close()


def test_label_reuse_svd(hub_graph):
    """M_LR = [X | ÂX | Â^2 X | N0 Y | N0^2 Y] as HCAT(M_NC, PRODUCT(N0, [Y | N0 Y]))."""
    g = hub_graph
    x = synth.tfidf_features(g.n, 40, 0.05, 91)
    y, mask = synth.labels(g.n, 6, 0.5, 92)
    Y = np.zeros((g.n, 6), np.float32)
    Y[mask, y[mask]] = 1.0
    ncg = isvd.graph_operator(g, form="concat", norm="sym", X=(x.d, x.rowptr, x.colidx, x.values), L=2)
    n0g = isvd.graph_operator(g, norm="sym_noself", coeffs=[1.0])
    yg = isvd.graph_operator(g, form="concat", norm="sym_noself", X=Y, L=1)
    lrg = isvd.compose("hcat", [ncg, isvd.compose("product", [n0g, yg])])
    nco = oracle.graph_operator(g, form="concat", norm="sym", X=(x.d, x.rowptr, x.colidx, x.values.astype(np.float64)), L=2)
    lro = oracle.compose("hcat", [nco, oracle.compose("product", [
        oracle.graph_operator(g, norm="sym_noself", coeffs=[1.0]),
        oracle.graph_operator(g, form="concat", norm="sym_noself", X=Y.astype(np.float64), L=1)])])
    assert lrg.shape == lro.shape == (g.n, 3 * 40 + 2 * 6)
    check_svd(lrg, lro, 16, 10, 4, 93)
    lrg.close()
    for o in (ncg, n0g, yg):
        o.close()


def test_pseudo_dropout_svd(hub_graph):
    g = hub_graph
    X = synth.dense_features(g.n, 24, 94)
    Xd = (X * (np.random.default_rng(95).random(X.shape) >= 0.3) / 0.7).astype(np.float32)
    kids = [isvd.graph_operator(g, form="concat", norm="sym", X=a, L=2) for a in (X, Xd)]
    pdg = isvd.compose("vcat", kids)
    pdo = oracle.compose("vcat", [oracle.graph_operator(g, form="concat", norm="sym", X=a.astype(np.float64), L=2)
                                  for a in (X, Xd)])
    assert pdg.shape == (2 * g.n, 72)
    check_svd(pdg, pdo, 12, 8, 4, 96)
    pdg.close()
    for o in kids:
        o.close()


def test_composite_follows_child_tuning(children):
    gpu, ref = children
    cg = _tree(isvd, "hcat", *gpu)
    _, S1, _, _ = cg.svd(8, 8, 2, 97)
    S1 = S1.clone()
    before = gpu[0].tuning()["kernel"]
    gpu[0].set_tuning(kernel="ring")
    _, S2, _, _ = cg.svd(8, 8, 2, 97)  # the cached graph holds the old launch shapes: recaptured
    gpu[0].set_tuning(kernel=before)
    assert torch.allclose(S1, S2, rtol=1e-5)
    cg.close()


def test_composite_rejections(children):
    gpu, _ = children
    a, b, c, d = gpu
    for kind, ops in (("sum", [a, c]), ("vcat", [a, c]), ("product", [c, a])):
        with pytest.raises(isvd.IsvdError, match="SHAPE"):
            isvd.compose(kind, ops)
    with pytest.raises(isvd.IsvdError, match="INVALID_ARGUMENT"):
        isvd.compose("hcat", [a, c], weights=[1.0, 2.0])
    cg = isvd.compose("sum", [a, b])
    with pytest.raises(isvd.IsvdError, match="UNSUPPORTED"):
        cg.set_tuning(kernel="ring")
    with pytest.raises(isvd.IsvdError, match="UNSUPPORTED"):
        isvd.Batch([cg], [4]).run()
    cg.close()


# ---- Gaussian-kernel edge function (Sec. 5.1, App. A.4) -------------------------------

def _factors(rows, cols, k, seed):
    rng = np.random.default_rng(seed)
    U = rng.standard_normal((rows, k)).astype(np.float32) / np.sqrt(k)
    V = rng.standard_normal((cols, k)).astype(np.float32) / np.sqrt(k)
    S = np.sort(rng.uniform(0.05, 6.0, k)).astype(np.float32)[::-1].copy()
    Ug, Vg = isvd.new_block(rows, k), isvd.new_block(cols, k)
    Ug.copy_(torch.from_numpy(U))
    Vg.copy_(torch.from_numpy(V))
    return U, S, V, Ug, torch.from_numpy(S).cuda(), Vg


@pytest.mark.parametrize("k", [1, 33, 160])
@pytest.mark.parametrize("mu,s", [(1.0, 1e-3), (1.1, 0.2), (0.7, 0.5)])
def test_edge_kernel_weights_match_oracle(k, mu, s):
    U, S, V, Ug, Sg, Vg = _factors(10, 10, k, 100 + k)
    ek = isvd.EdgeKernel(Ug, Sg, Vg, mu=mu, s=s)
    w3 = ek.weights().cpu().numpy()
    want = oracle.edge_kernel_weights(S.astype(np.float64), mu, ek.s_bar)
    # scale of the summed terms: S^x <= max(S)^2 on [0.5, 2]; the mu-derivative's
    # weights grow like sqrt(exp(s_bar)) (cancelling sums need an absolute bound)
    scale = max(1.0, float(S.max()) ** 2) * (1.0 + np.sqrt(np.exp(ek.s_bar)))
    for got, ref in zip(w3, want):
        assert np.allclose(got, ref, rtol=1e-11, atol=1e-13 * scale)


def test_edge_kernel_scores_and_loss_match_oracle():
    rows, cols, k = 3001, 2999, 72
    U, S, V, Ug, Sg, Vg = _factors(rows, cols, k, 101)
    rng = np.random.default_rng(102)
    pos = (rng.integers(0, rows, 4000), rng.integers(0, cols, 4000))
    neg = (rng.integers(0, rows, 9000), rng.integers(0, cols, 9000))
    ek = isvd.EdgeKernel(Ug, Sg, Vg, mu=1.15, s=0.25)
    w = oracle.edge_kernel_weights(S.astype(np.float64), ek.mu, ek.s_bar)[0]
    f = ek.scores(*pos)
    want = oracle.edge_scores(U, V, w, *pos)
    bound = 1e-6 * np.sum(np.abs(U[pos[0]].astype(np.float64) * w * V[pos[1]]), axis=1) + 1e-30
    assert np.all(np.abs(npy(f) - want) <= bound)
    out = ek.loss(pos, neg, 10.0)
    L, gm, gs = oracle.edge_kernel_loss(U, S, V, ek.mu, ek.s_bar, pos, neg, 10.0)
    got = out.cpu().numpy()
    assert abs(got[0] - L) <= 1e-6 * abs(L)
    assert abs(got[1] - gm) <= 1e-5 * (abs(gm) + 1e-3 * abs(L))
    assert abs(got[2] - gs) <= 1e-5 * (abs(gs) + 1e-3 * abs(L))
    assert torch.equal(out, ek.loss(pos, neg, 10.0))


def test_edge_kernel_flags_pairs_out_of_range():
    U, S, V, Ug, Sg, Vg = _factors(50, 40, 8, 103)
    ek = isvd.EdgeKernel(Ug, Sg, Vg)
    info = torch.zeros(4, dtype=torch.int32, device="cuda")
    f = ek.scores([0, 50, 3], [0, 1, 40], info=info)
    assert torch.isnan(f.cpu()[1:]).all() and torch.isfinite(f.cpu()[0])
    assert isvd.info_dict(info)["status"] == "INVALID_ARGUMENT"
    info.zero_()
    out = ek.loss(([0, 1], [2, 3]), ([-1], [0]), info=info)
    assert torch.isnan(out.cpu()).all()
    assert isvd.info_dict(info)["status"] == "INVALID_ARGUMENT"


def test_edge_kernel_fit_lowers_the_link_loss(hub_graph):
    """From the SVD of the NE operator, a few descent steps on (mu, s_bar)
    lower Eq. 9 on the graph's edges against random pairs (Sec. 5.1)."""
    g = hub_graph
    with isvd.graph_operator(g, norm="sym", coeffs=C5, ones_coeff=-LAM) as op:
        U, S, V, _ = op.svd(32, 10, 4, 104)
    rows = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    rng = np.random.default_rng(105)
    e = rng.choice(len(rows), 5000, replace=False)
    pos = (rows[e], g.colidx[e])
    neg = (rng.integers(0, g.n, 20000), rng.integers(0, g.n, 20000))
    ek = isvd.EdgeKernel(U, S, V)
    hist = ek.fit(pos, neg, 10.0, steps=30, lr=0.5)
    assert np.all(np.isfinite(hist)) and hist[-1] < hist[0]
    L, _, _ = oracle.edge_kernel_loss(npy(U), npy(S), npy(V), ek.mu, ek.s_bar, pos, neg, 10.0)
    assert abs(ek.loss(pos, neg, 10.0)[0].item() - L) <= 1e-5 * abs(L)


# ---- Split-ReLU network (Sec. 5.2, Thm. 2) ------------------------------------------------

def _splitrelu_setup(g, d=16, y=5, L=2, seed=110):
    X = synth.dense_features(g.n, d, seed)
    W_star = (np.random.default_rng(seed + 1).standard_normal((d * (L + 1), y)) / 4).astype(np.float32)
    return X, W_star


def test_splitrelu_network_at_init_is_the_linear_model(hub_graph):
    from paper_2111_06312_gb300.splitrelu import SplitReLUNet
    g = hub_graph
    L = 2
    X, W_star = _splitrelu_setup(g, L=L)
    with isvd.graph_operator(g, norm="sym", coeffs=[1.0]) as prop:
        net = SplitReLUNet(prop, torch.from_numpy(X).cuda(), torch.from_numpy(W_star).cuda(), L)
        out = net()
    ref = oracle.graph_operator(g, form="concat", norm="sym", X=X.astype(np.float64), L=L).apply(
        W_star.astype(np.float64))
    assert np.abs(npy(out) - ref).max() <= 1e-5 * np.abs(ref).max()


def test_splitrelu_gradients_match_oracle(hub_graph):
    from paper_2111_06312_gb300.splitrelu import SplitReLUNet
    g = hub_graph
    d, y, L = 16, 5, 2
    X, W_star = _splitrelu_setup(g, d, y, L)
    rng = np.random.default_rng(112)
    with isvd.graph_operator(g, norm="sym", coeffs=[1.0]) as prop:
        net = SplitReLUNet(prop, torch.from_numpy(X).cuda(), torch.from_numpy(W_star).cuda(), L)
        with torch.no_grad():  # move off the linear start: mixed ReLU signs
            for p in net.parameters():
                p.add_(torch.from_numpy((rng.standard_normal(tuple(p.shape)) * 0.3).astype(np.float32)).cuda())
        R = rng.standard_normal((g.n, y)).astype(np.float32)
        out = net()
        (out * torch.from_numpy(R).cuda()).sum().backward()
    weights = tuple([npy(p.detach()) for p in group] for group in (net.Wp, net.Wn, net.Wop, net.Won))
    Ah = oracle.graph_operator(g, norm="sym", coeffs=[1.0])
    out_ref, cache = oracle.splitrelu_forward(Ah.apply, X.astype(np.float64), *weights)
    assert np.abs(npy(out) - out_ref).max() <= 1e-5 * np.abs(out_ref).max()
    grads = oracle.splitrelu_backward(lambda G: Ah.apply(G, transpose=True), cache, weights, R.astype(np.float64))
    for group, ggroup in zip((net.Wp, net.Wn, net.Wop, net.Won), grads):
        for p, dW in zip(group, ggroup):
            assert np.linalg.norm(npy(p.grad) - dW) <= 1e-4 * np.linalg.norm(dW) + 1e-6


def test_splitrelu_finetune_starts_at_the_closed_form_fit(hub_graph):
    """W* from Thm. 1 on the rank-k SVD of [X | ÂX | Â^2 X]; the network's
    first cross-entropy equals the linear model's, and Adam lowers it."""
    from paper_2111_06312_gb300 import adjoint
    from paper_2111_06312_gb300.splitrelu import SplitReLUNet, finetune
    g = hub_graph
    d, y, L = 16, 5, 2
    X, _ = _splitrelu_setup(g, d, y, L)
    lab, mask = synth.labels(g.n, y, 0.3, 113)
    labels = torch.from_numpy(lab).cuda()
    train = torch.from_numpy(mask).cuda()
    Xg = torch.from_numpy(X).cuda()
    with isvd.graph_operator(g, form="concat", norm="sym", X=X, L=L) as m, \
            isvd.graph_operator(g, norm="sym", coeffs=[1.0]) as prop:
        W, _ = adjoint.closed_form_init(m, adjoint.one_hot_train(labels, train, y), 24, seed=114)
        lin = torch.nn.functional.cross_entropy(m.apply(W)[train], labels[train]).item()
        net = SplitReLUNet(prop, Xg, W, L)
        hist = finetune(net, labels, train, epochs=15, lr=3e-3)
    assert abs(hist[0] - lin) <= 1e-5 * lin
    assert hist[-1] < hist[0]


@pytest.mark.parametrize("p", [1, 3])
@pytest.mark.parametrize("transpose", [False, True])
def test_scalar_and_power_nodes(children, p, transpose):
    gpu, ref = children
    a = gpu[0]
    for cg, co in ((isvd.power(a, p), oracle.power(ref[0], p)), (isvd.scale(a, -2.5), oracle.scale(ref[0], -2.5))):
        G = isvd.gaussian(11, a.shape[1], 13)
        Y = cg.apply(G, transpose=transpose)
        Yr = co.apply(npy(G), transpose=transpose)
        assert np.abs(npy(Y) - Yr).max() <= 1e-5 * np.abs(Yr).max()
        cg.close()


def _spmm_launches(fn):
    """Sparse-product kernel launches made by fn() (CUDA profiler trace)."""
    from torch.profiler import ProfilerActivity, profile

    torch.cuda.synchronize()
    with profile(activities=[ProfilerActivity.CUDA]) as prof:
        fn()
        torch.cuda.synchronize()
    return sum(e.count for e in prof.key_averages() if "spmm_" in e.key)


@pytest.mark.parametrize("transpose", [False, True])
def test_lazy_product_cache(hub_graph, transpose):
    """The lazy cache of App. A.3 on composite trees with repeated products:
    S = c_1 N + c_2 N^2 + c_3 N^3 (N = Â) written as a sum of powers forms
    N G, N^2 G once each (3 products of N instead of 6), and H = [N | N^2]
    forms N^T G once in the transposed product (2 instead of 3; the forward
    product has nothing to share).  Cached and uncached results are bit for
    bit equal, and both match the oracle's composite."""
    g = hub_graph
    with isvd.graph_operator(g, norm="sym", coeffs=[1.0], check_symmetry=False) as T:
        ref_T = oracle.graph_operator(g, norm="sym", coeffs=[1.0])
        c = [0.5, -0.3, 0.2]
        p2, p3 = isvd.power(T, 2), isvd.power(T, 3)
        S = isvd.compose("sum", [T, p2, p3], c)
        H = isvd.compose("hcat", [T, p2])
        refs = {"S": oracle.compose("sum", [ref_T, oracle.power(ref_T, 2), oracle.power(ref_T, 3)], c),
                "H": oracle.compose("hcat", [ref_T, oracle.power(ref_T, 2)])}
        expect = {"S": (3, 6), "H": (2, 3) if transpose else (3, 3)}
        G1 = isvd.gaussian(1, g.n, 24)
        T.apply(G1)
        _spmm_launches(lambda: T.apply(G1))  # the first trace of a process may miss launches
        one = _spmm_launches(lambda: T.apply(G1))  # sparse-product launches of one product with N
        assert one >= 1
        for name, op in (("S", S), ("H", H)):
            rows_in = op.shape[0] if transpose else op.shape[1]
            G = isvd.gaussian(12, rows_in, 24)
            out = {}
            counts = {}
            for on in (True, False):
                isvd.set_product_cache(op, on)
                op.apply(G, transpose=transpose)  # warm the workspace
                counts[on] = _spmm_launches(lambda: out.__setitem__(on, op.apply(G, transpose=transpose)))
            assert torch.equal(out[True], out[False]), name
            assert (counts[True], counts[False]) == (expect[name][0] * one, expect[name][1] * one), (name, counts, one)
            Yr = refs[name].apply(npy(G), transpose=transpose)
            assert np.abs(npy(out[True]) - Yr).max() <= 1e-5 * np.abs(Yr).max()
        for op in (S, H, p3, p2):
            op.close()


def test_splitrelu_layers_run_in_the_library(hub_graph):
    """Every dense product and ReLU of the Split-ReLU network (Sec. 5.2),
    forward and backward, runs in the library's kernels: the split-ReLU
    entry points (tensor-core Q.B and A^T B products, elementwise ReLU and
    mask passes); no library GEMM (cuBLAS / CUTLASS) is launched."""
    from torch.profiler import ProfilerActivity, profile

    from paper_2111_06312_gb300.splitrelu import SplitReLUNet
    g = hub_graph
    d, y, L = 16, 5, 2
    X, W_star = _splitrelu_setup(g, d, y, L)
    with isvd.graph_operator(g, norm="sym", coeffs=[1.0]) as prop:
        net = SplitReLUNet(prop, torch.from_numpy(X).cuda(), torch.from_numpy(W_star).cuda(), L)
        R = torch.randn((g.n, y), device="cuda")
        (net() * R).sum().backward()  # warm
        torch.cuda.synchronize()
        with profile(activities=[ProfilerActivity.CUDA]) as prof:
            (net() * R).sum().backward()
            torch.cuda.synchronize()
    names = [e.key for e in prof.key_averages()]
    assert any("split_relu_fwd_kernel" in k for k in names), names
    assert any("split_relu_mask_kernel" in k for k in names), names
    assert any("gemm_tc_kernel" in k for k in names), names
    assert any("gram_ab_tc_kernel" in k for k in names), names
    foreign = [k for k in names if any(t in k.lower() for t in ("xmma", "nvjet", "cutlass", "sgemm", "cublas"))]
    assert not foreign, foreign
