"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, on the
same seeded inputs.  Sizes span several tiles and ragged tails; graphs
include hub rows that take the split path.  Tolerances (FP32): products
within 1e-5 of the output scale, singular values within relative 1e-5,
principal angles below 1e-3 rad (on the prefix of the spectrum that is
separated by a gap; the rest is checked for validity)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2111_06312_gb300 import build, isvd, synth
from svd_checks import check_svd, cond_block, gapped_prefix  # noqa: F401

pytestmark = pytest.mark.gpu
LAM = 0.05
C5 = oracle.ne_coefficients(5)


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
    # hubs above the split threshold (256 nonzeros) and many light rows
    return synth.chung_lu(3000, 24000, 77, max_degree=1500)


@pytest.fixture(scope="module")
def ne_small():
    return synth.workload_ne_small()


def sym_weights(g, seed):
    rows = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    key = np.minimum(rows, g.colidx).astype(np.int64) * g.n + np.maximum(rows, g.colidx)
    _, inv = np.unique(key, return_inverse=True)
    return np.random.default_rng(seed).uniform(0.5, 2.0, inv.max() + 1)[inv].astype(np.float32)


# ---- start block ----------------------------------------------------------------

@pytest.mark.parametrize("seed", [0, 1, 2**40 + 3])
def test_philox_words_bit_exact(seed):
    rows = 257
    w = isvd.philox_words(seed, rows).cpu().numpy().view(np.uint32)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for i in range(rows):
        for j in range(4):
            ref = oracle.philox4x32_10([j, i & 0xFFFFFFFF, i >> 32, 0], key)
            assert np.array_equal(w[i, 4 * j:4 * j + 4], ref)


@pytest.mark.parametrize("cols", [1, 5, 42, 144])
def test_gaussian_matches_oracle(cols):
    Z = isvd.gaussian(11, 3001, cols)
    Zr = oracle.gaussian(11, 3001, cols)
    err = np.abs(npy(Z) - Zr) / (1 + np.abs(Zr))
    assert err.max() < 2e-6
    full = Z.as_strided((Z.shape[0], Z.stride(0)), (Z.stride(0), 1))
    assert torch.all(full[:, cols:] == 0)
    Zb = isvd.gaussian(11, 3001, cols, dtype=torch.bfloat16)
    assert (np.abs(npy(Zb) - Zr) / (1 + np.abs(Zr))).max() < 1e-2


# ---- products --------------------------------------------------------------------

CASES = [
    # norm, K, ones, adj, weighted, lowrank
    ("row", 5, True, False, False, False),
    ("row", 1, True, False, False, False),
    ("row", 2, False, True, True, False),
    ("row", 5, True, True, False, True),
    ("sym", 5, True, False, False, False),
    ("sym", 1, False, False, True, False),
    ("sym", 3, True, True, False, True),
]


def make_ops(g, norm, K, ones, adj, weighted, lowrank, seed=5):
    kw = dict(norm=norm, coeffs=oracle.ne_coefficients(K), ones_coeff=-LAM if ones else 0.0,
              adj_coeff=0.02 if adj else 0.0)
    if weighted:
        kw["values"] = sym_weights(g, seed)
    if lowrank:
        rng = np.random.default_rng(seed)
        u = rng.standard_normal((g.n, 2)).astype(np.float32)
        v = rng.standard_normal((g.n, 2)).astype(np.float32)
        kw["lowrank"] = (u, v, np.array([0.01, -0.02]))
    gpu = isvd.graph_operator(g, **kw)
    if weighted:
        kw["values"] = kw["values"].astype(np.float64)
    if lowrank:
        u, v, a = kw["lowrank"]
        kw["lowrank"] = (u.astype(np.float64), v.astype(np.float64), a)
    return gpu, oracle.graph_operator(g, **kw)


KERNELS = ["ring", "chunks", "rows", "rows_wide", "rows_packed", "slab", "slab_narrow", "slab_pieces"]


def tune(op, kernel, **kw):
    """rows_wide: the row kernel with slabs wider than 32 lanes x 16 bytes
    (two 16-byte chunks per lane); rows_packed: the row kernel with packed
    Horner temporaries; slab: the packed-slab kernel at its default widths;
    slab_narrow: packed slabs of 16 columns (several rows per warp);
    slab_pieces: packed slabs with rows above 32 nonzeros cut into 32-nonzero
    pieces (many hub partials finished by the last piece)."""
    if kernel == "rows_wide":
        op.set_tuning(kernel="rows", slab_cols_f32=256, slab_cols_bf16=512, packed=False, **kw)
    elif kernel == "rows_packed":
        op.set_tuning(kernel="rows", slab_cols_f32=128, slab_cols_bf16=256, packed=True, **kw)
    elif kernel == "slab_narrow":
        op.set_tuning(kernel="slab", slab_cols_f32=16, slab_cols_bf16=16, **kw)
    elif kernel == "slab_pieces":
        op.set_tuning(kernel="slab", heavy_threshold=32, heavy_chunk=32, **kw)
    else:
        op.set_tuning(kernel=kernel, packed=False, **kw)


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("b", [1, 3, 42, 144, 200])
@pytest.mark.parametrize("transpose", [False, True])
@pytest.mark.parametrize("kernel", KERNELS)
def test_poly_apply_fp32(hub_graph, case, b, transpose, kernel):
    g = hub_graph
    gpu, ref = make_ops(g, *case)
    with gpu:
        tune(gpu, kernel, chunk_nnz=256)
        G = isvd.gaussian(3, g.n, b)
        Y = gpu.apply(G, transpose=transpose)
        Yr = ref.apply(npy(G), transpose=transpose)
    scale = np.abs(Yr).max()
    assert np.abs(npy(Y) - Yr).max() <= 1e-5 * scale


@pytest.mark.parametrize("case", CASES[:5])
@pytest.mark.parametrize("kernel", KERNELS)
def test_poly_apply_bf16(hub_graph, case, kernel):
    g = hub_graph
    gpu, ref = make_ops(g, *case)
    with gpu:
        tune(gpu, kernel)
        G = isvd.gaussian(4, g.n, 72, dtype=torch.bfloat16)
        Y = gpu.apply(G)
        Yr = ref.apply(npy(G))
    assert np.abs(npy(Y) - Yr).max() <= 3e-2 * np.abs(Yr).max()


@pytest.mark.parametrize("kernel", KERNELS)
def test_apply_empty_rows_and_hubs(kernel):
    # isolated nodes (no nonzeros) under Â, one hub spanning many chunks
    g = synth.chung_lu(2000, 9000, 91, max_degree=1200, isolated_self_loops=False)
    assert (g.degrees() == 0).any() and g.degrees().max() > 600
    gpu, ref = make_ops(g, "sym", 5, True, False, False, False)
    with gpu:
        tune(gpu, kernel, chunk_nnz=64)
        for b in (5, 40, 130):
            for tr in (False, True):
                G = isvd.gaussian(8, g.n, b)
                Y = gpu.apply(G, transpose=tr)
                Yr = ref.apply(npy(G), transpose=tr)
                assert np.abs(npy(Y) - Yr).max() <= 1e-5 * np.abs(Yr).max()


def test_apply_leaves_padding_and_is_deterministic(hub_graph):
    g = hub_graph
    gpu, ref = make_ops(g, *CASES[0])
    with gpu:
        G = isvd.gaussian(5, g.n, 42)
        out = torch.full((g.n, 48), 7.0, device="cuda")
        gpu.apply(G, out=out[:, :42])
        assert torch.all(out[:, 42:] == 7.0)
        Y1 = gpu.apply(G).clone()
        Y2 = gpu.apply(G)
        assert torch.equal(Y1, Y2)


@pytest.mark.parametrize("L", [0, 1, 2])
@pytest.mark.parametrize("norm", ["sym", "row"])
@pytest.mark.parametrize("dense", [False, True])
@pytest.mark.parametrize("transpose", [False, True])
@pytest.mark.parametrize("kernel", KERNELS)
def test_concat_apply(hub_graph, L, norm, dense, transpose, kernel):
    g = hub_graph
    d = 37
    if dense:
        X = synth.dense_features(g.n, d, 12)
        Xg, Xo = X, X.astype(np.float64)
    else:
        x = synth.tfidf_features(g.n, d, 0.05, 12)
        Xg = (d, x.rowptr, x.colidx, x.values)
        Xo = (d, x.rowptr, x.colidx, x.values.astype(np.float64))
    with isvd.graph_operator(g, form="concat", norm=norm, X=Xg, L=L) as gpu:
        tune(gpu, kernel, chunk_nnz=128)
        ref = oracle.graph_operator(g, form="concat", norm=norm, X=Xo, L=L)
        r, c = gpu.shape
        assert (r, c) == ref.shape
        G = isvd.gaussian(6, r if transpose else c, 19)
        Y = gpu.apply(G, transpose=transpose)
        Yr = ref.apply(npy(G), transpose=transpose)
    assert np.abs(npy(Y) - Yr).max() <= 1e-5 * np.abs(Yr).max()


@pytest.mark.parametrize("b,dtype", [(100, torch.float32), (19, torch.bfloat16), (60, torch.bfloat16)])
@pytest.mark.parametrize("transpose", [False, True])
def test_concat_dense_x_wide_and_bf16(hub_graph, b, dtype, transpose):
    """Dense X: the small dense products serve (L+1) * round8(b) <= 160 columns
    in FP32 (and the forward product in BF16); wider blocks and the BF16
    transposed product take the sparse form."""
    g = hub_graph
    X = synth.dense_features(g.n, 64, 14)
    with isvd.graph_operator(g, form="concat", norm="sym", X=X, L=2) as gpu:
        ref = oracle.graph_operator(g, form="concat", norm="sym", X=X.astype(np.float64), L=2)
        r, c = gpu.shape
        G = isvd.gaussian(7, r if transpose else c, b, dtype=dtype)
        Y = gpu.apply(G, transpose=transpose)
        Yr = ref.apply(npy(G), transpose=transpose)
    tol = 1e-5 if dtype == torch.float32 else 2e-2
    assert np.abs(npy(Y) - Yr).max() <= tol * np.abs(Yr).max()


# ---- orthonormalisation (Alg. 2) and the small SVD --------------------------------

@pytest.mark.parametrize("rows,l,cond", [(5000, 42, 1e2), (20011, 144, 1e3), (3001, 19, 1e5), (70000, 74, 1e6),
                                         (9000, 160, 1e5), (4000, 33, 1e4), (2500, 31, 1e2)])
def test_orthonormalize(ne_small, rows, l, cond):
    Q0 = cond_block(rows, l, cond, 8)
    with isvd.graph_operator(ne_small, coeffs=C5) as op:
        Q = torch.tensor(Q0, dtype=torch.float32, device="cuda")
        Qg, R, info = isvd.orthonormalize(op, Q)
        Qn, Rn = npy(Qg), R.cpu().numpy()
        inf = isvd.info_dict(info)
    assert inf["status"] == "OK"
    assert np.abs(Qn.T @ Qn - np.eye(l)).max() < 2e-5
    Qr, Rr, _ = oracle.cholqr2(Q0.astype(np.float32).astype(np.float64))
    assert oracle.max_principal_angle(Qr, Qn) < 50 * 6e-8 * cond * np.sqrt(l)
    assert np.abs(Qn @ Rn - Q0).max() < 1e-5 * np.abs(Q0).max() * max(1.0, cond / 1e3)
    if cond >= 1e5:
        assert inf["chol_shifts"] >= 1 and inf["cholqr_passes"] >= 3


@pytest.mark.parametrize("rows,l,width,col0", [(7001, 40, 64, 0), (3000, 144, 152, 4), (12345, 9, 24, 4)])
def test_orthonormalize_strided_view(ne_small, rows, l, width, col0):
    """A column slice of a wider buffer (row pitch above round8(l)): the Gram
    loads rows piece by piece instead of one copy per chunk; a slice starting
    at column 4 is 16- but not 32-byte aligned (16-byte stores in Q R^-1);
    the other columns stay untouched."""
    Q0 = cond_block(rows, l, 1e3, 11)
    buf = torch.full((rows, width), 7.0, dtype=torch.float32, device="cuda")
    buf[:, col0:col0 + l] = torch.tensor(Q0, dtype=torch.float32, device="cuda")
    with isvd.graph_operator(ne_small, coeffs=C5) as op:
        Qg, R, info = isvd.orthonormalize(op, buf[:, col0:col0 + l])
        assert Qg.data_ptr() == buf[:, col0:].data_ptr()  # worked in place on the view
        inf = isvd.info_dict(info)
    assert inf["status"] == "OK"
    Qn = npy(buf[:, col0:col0 + l])
    assert np.abs(Qn.T @ Qn - np.eye(l)).max() < 2e-5
    assert np.abs(Qn @ R.cpu().numpy() - Q0).max() < 1e-5 * np.abs(Q0).max()
    rest = torch.cat([buf[:, :col0], buf[:, col0 + l:]], dim=1)
    assert bool((rest == 7.0).all())


@pytest.mark.parametrize("l,cond,upper", [(8, 10.0, False), (42, 1e6, True), (144, 1e8, True), (160, 1e3, False)])
def test_small_svd(ne_small, l, cond, upper):
    A = cond_block(l, l, cond, 9)
    if upper:
        A = np.linalg.qr(A)[1]
    with isvd.graph_operator(ne_small, coeffs=C5) as op:
        U, S, V = isvd.small_svd(op, torch.tensor(A, device="cuda"))
    U, S, V = U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy()
    Sr = np.linalg.svd(A, compute_uv=False)
    assert np.allclose(S, Sr, rtol=1e-11, atol=1e-14 * Sr[0])
    assert np.abs((U * S) @ V.T - A).max() < 1e-13 * Sr[0]
    # V: the rotated columns (orthogonal to rounding); U = A V S^-1 is recovered
    # by one product, so its orthogonality error grows like eps * cond
    assert np.abs(U.T @ U - np.eye(l)).max() < max(1e-12, 1e-14 * cond)
    assert np.abs(V.T @ V - np.eye(l)).max() < 1e-12


# ---- Alg. 1 end to end ---------------------------------------------------------------

@pytest.mark.parametrize("kernel", KERNELS)
def test_svd_ne_small_parity(ne_small, kernel):
    """Cora-sized NE operator: k = 32, oversample 10, 4 power iterations."""
    g = ne_small
    with isvd.graph_operator(g, coeffs=C5, ones_coeff=-LAM) as gpu:
        tune(gpu, kernel)
        ref = oracle.graph_operator(g, coeffs=C5, ones_coeff=-LAM)
        out = check_svd(gpu, ref, 32, 10, 4, synth.BASE_SEED)
    print(out)


@pytest.mark.parametrize("k,p,q", [(1, 0, 0), (5, 3, 2), (13, 6, 3), (40, 24, 1)])
def test_svd_ragged_blocks(hub_graph, k, p, q):
    g = hub_graph
    with isvd.graph_operator(g, norm="sym", coeffs=C5, ones_coeff=-LAM) as gpu:
        ref = oracle.graph_operator(g, norm="sym", coeffs=C5, ones_coeff=-LAM)
        check_svd(gpu, ref, k, p, q, 17)


def test_svd_concat_sparse(hub_graph):
    g = hub_graph
    x = synth.tfidf_features(g.n, 60, 0.03, 13)
    with isvd.graph_operator(g, form="concat", norm="sym", X=(60, x.rowptr, x.colidx, x.values), L=2) as gpu:
        ref = oracle.graph_operator(g, form="concat", norm="sym", X=(60, x.rowptr, x.colidx,
                                                                       x.values.astype(np.float64)), L=2)
        check_svd(gpu, ref, 16, 10, 4, 23)


@pytest.mark.parametrize("kernel", KERNELS)
def test_svd_concat_pubmed_sized(kernel):
    """Feature-concatenation operator [X | ÂX | Â²X] at n = 19,717, d = 500, k = 64."""
    g, x = synth.workload_concat_graph()
    X = (x.d, x.rowptr, x.colidx, x.values)
    with isvd.graph_operator(g, form="concat", norm="sym", X=X, L=2) as gpu:
        tune(gpu, kernel)
        ref = oracle.graph_operator(g, form="concat", norm="sym",
                                    X=(x.d, x.rowptr, x.colidx, x.values.astype(np.float64)), L=2)
        out = check_svd(gpu, ref, 64, 10, 4, synth.BASE_SEED + 1)
    print(out)


@pytest.mark.parametrize("form", ["poly", "concat"])
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_row_gather_apply(hub_graph, form, dtype):
    """M[rows, :] (Thm. 1's fit on training rows): products through the
    gather and the scatter against the oracle's row-selected operator."""
    g = hub_graph
    rows = np.sort(np.random.default_rng(31).choice(g.n, g.n * 3 // 5, replace=False)).astype(np.int32)
    if form == "poly":
        kw_g = kw_o = dict(norm="sym", coeffs=C5, ones_coeff=-LAM)
    else:
        x = synth.tfidf_features(g.n, 30, 0.05, 32)
        kw_g = dict(form="concat", norm="sym", X=(30, x.rowptr, x.colidx, x.values), L=2)
        kw_o = dict(form="concat", norm="sym", X=(30, x.rowptr, x.colidx, x.values.astype(np.float64)), L=2)
    with isvd.graph_operator(g, gather_rows=rows, **kw_g) as gpu:
        ref = oracle.graph_operator(g, gather_rows=rows, **kw_o)
        assert gpu.shape == ref.shape and gpu.shape[0] == len(rows)
        tol = 1e-5 if dtype == torch.float32 else 2e-2
        for transpose in (False, True):
            G = isvd.gaussian(8, gpu.shape[0] if transpose else gpu.shape[1], 21, dtype=dtype)
            Y = gpu.apply(G, transpose=transpose)
            Yr = ref.apply(npy(G), transpose=transpose)
            assert np.abs(npy(Y) - Yr).max() <= tol * np.abs(Yr).max()


def test_row_gather_svd(hub_graph):
    g = hub_graph
    rows = np.sort(np.random.default_rng(33).choice(g.n, g.n // 2, replace=False)).astype(np.int32)
    with isvd.graph_operator(g, norm="sym", coeffs=C5, ones_coeff=-LAM, gather_rows=rows) as gpu:
        ref = oracle.graph_operator(g, norm="sym", coeffs=C5, ones_coeff=-LAM, gather_rows=rows)
        check_svd(gpu, ref, 16, 8, 4, 34)


def test_row_gather_rejects_bad_rows(hub_graph):
    g = hub_graph
    for bad in (np.array([3, 3, 5], np.int32), np.array([5, 2], np.int32), np.array([0, g.n], np.int32)):
        with pytest.raises(isvd.IsvdError, match="gather_rows"):
            isvd.graph_operator(g, coeffs=C5, gather_rows=bad)


def test_svd_is_deterministic(ne_small):
    with isvd.graph_operator(ne_small, coeffs=C5, ones_coeff=-LAM) as gpu:
        U1, S1, V1, _ = gpu.svd(16, 8, 3, 5)
        U1, S1, V1 = U1.clone(), S1.clone(), V1.clone()
        U2, S2, V2, _ = gpu.svd(16, 8, 3, 5)
        assert torch.equal(S1, S2) and torch.equal(U1, U2) and torch.equal(V1, V2)


def test_svd_mixed_precision_close(ne_small):
    g = ne_small
    with isvd.graph_operator(g, coeffs=C5, ones_coeff=-LAM) as gpu:
        ref = oracle.graph_operator(g, coeffs=C5, ones_coeff=-LAM)
        U, S, V, info = gpu.svd(32, 10, 4, synth.BASE_SEED, precision="mixed")
        _, Sr, _, _ = ref.isvd(32, 10, 4, synth.BASE_SEED)
    rel = np.abs(npy(S) - Sr) / Sr
    assert isvd.info_dict(info)["status"] == "OK"
    assert rel.max() < 5e-2
    Un = npy(U)
    assert np.abs(Un.T @ Un - np.eye(32)).max() < 1e-5


# ---- error paths (host-made failures; no GPU fault) -----------------------------------

def test_invalid_graphs_rejected():
    g = synth.cycle(10)
    bad = g.rowptr.copy()
    bad[3] = bad[4] + 1  # not monotone
    with pytest.raises(isvd.IsvdError) as e:
        isvd.Operator(g.n, bad, g.colidx, coeffs=C5)
    assert e.value.name == "INVALID_GRAPH"
    col = g.colidx.copy()
    col[0] = 99  # out of range
    with pytest.raises(isvd.IsvdError) as e:
        isvd.Operator(g.n, g.rowptr, col, coeffs=C5)
    assert e.value.name == "INVALID_GRAPH"
    # asymmetric: drop one direction of an edge
    asym = synth.from_edges(4, [(0, 1), (1, 2), (2, 3)])
    rp = asym.rowptr.copy()
    ci = asym.colidx.copy()
    ci = np.delete(ci, 0)  # drop (0, 1)
    rp[1:] -= 1
    with pytest.raises(isvd.IsvdError) as e:
        isvd.Operator(4, rp, ci, norm="sym", coeffs=C5)
    assert e.value.name == "INVALID_GRAPH" and "symmetric" in str(e.value)
    # zero degree under T = D^-1 A
    iso = synth.from_edges(4, [(0, 1), (1, 2)])  # node 3 isolated, no self-loop
    with pytest.raises(isvd.IsvdError) as e:
        isvd.Operator(4, iso.rowptr, iso.colidx, coeffs=C5)
    assert e.value.name == "INVALID_GRAPH"
    # ... but fine for Â
    isvd.Operator(4, iso.rowptr, iso.colidx, norm="sym", coeffs=C5).close()


def test_bad_svd_arguments(ne_small):
    with isvd.graph_operator(ne_small, coeffs=C5) as op:
        with pytest.raises(isvd.IsvdError) as e:
            op.svd(500, 20, 1, 0)  # block width above 512
        assert e.value.name == "UNSUPPORTED"
        with pytest.raises(isvd.IsvdError) as e:
            op.svd(150, 20, 1, 0, precision="mixed")  # above 160: FP32 only
        assert e.value.name == "UNSUPPORTED"
        with pytest.raises(isvd.IsvdError) as e:
            op.svd(0, 2, 1, 0)
        assert e.value.name == "INVALID_ARGUMENT"
    small = synth.cycle(12)
    with isvd.graph_operator(small, coeffs=C5) as op:
        with pytest.raises(isvd.IsvdError) as e:
            op.svd(10, 5, 1, 0)
        assert e.value.name == "SHAPE"


def test_nan_input_reports_breakdown(hub_graph):
    # a NaN feature (host-made) makes every Gram matrix non-finite: the
    # Cholesky kernel reports NOT_POSITIVE_DEFINITE through the device status
    g = hub_graph
    X = synth.dense_features(g.n, 16, 3)
    X[5, 2] = np.nan
    with isvd.graph_operator(g, form="concat", norm="sym", X=X, L=1) as op:
        with pytest.raises(isvd.IsvdError) as e:
            op.svd(4, 4, 1, 0)
        assert e.value.name == "NOT_POSITIVE_DEFINITE"
