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
KERNELS = ["ring", "chunks", "rows"]


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    build.build()
    oracle.build()


def npy(t):
    return t.double().cpu().numpy()


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
