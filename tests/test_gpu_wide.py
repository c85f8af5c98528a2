"""Block widths above 160 columns (FP32): the paper's own l = 2k at ranks 128
and 256 (Sec. 6), through the C ABI, against the FP64 oracle.

Wide blocks are orthonormalised in 128-column panels (block Gram-Schmidt with
two projections, then CholeskyQR2 per panel); the thin QR they give is the
one CholeskyQR2 of the whole block gives (Q with R's diagonal positive is
unique), so the oracle's full-width CholeskyQR2 is the reference.  The
Rayleigh-Ritz SVD of an l x l R above 160 columns runs over the whole grid
(column blocks in global memory, grid barriers); LAPACK's singular values pin
it.

Singular-value tolerance of Alg. 1 here: the FP32 products perturb M by
about u ||M|| (u = 2^-24) per product, and by Weyl's inequality every
singular value moves by at most that much, so the bound is
|s_i - s_ref_i| <= 1e-5 s_i + 1e-6 s_1 (relative 1e-5 where s_i is near
s_1, absolute 1e-6 s_1 in the tail)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2111_06312_gb300 import build, isvd, synth
from svd_checks import cond_block, gapped_prefix, npy

pytestmark = pytest.mark.gpu
LAM = 0.05
C5 = oracle.ne_coefficients(5)


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    build.build()
    oracle.build()


@pytest.fixture(scope="module")
def ne_small():
    return synth.workload_ne_small()


# ---- orthonormalisation ------------------------------------------------------------

# widths: two full panels; a ragged third panel (300 = 128 + 128 + 44); the
# widest block (four panels); a barely wide block (161: one column in panel 2)
@pytest.mark.parametrize("rows,l,cond", [(20011, 256, 1e3), (7001, 300, 1e2), (9000, 512, 1e2), (5003, 161, 1e4),
                                         (6000, 384, 1e5)])
def test_wide_orthonormalize(ne_small, rows, l, cond):
    Q0 = cond_block(rows, l, cond, 21 + l)
    with isvd.graph_operator(ne_small, coeffs=C5) as op:
        Q = torch.tensor(Q0, dtype=torch.float32, device="cuda")
        Qg, R, info = isvd.orthonormalize(op, Q)
        Qn, Rn = npy(Qg), R.cpu().numpy()
        inf = isvd.info_dict(info)
    assert inf["status"] == "OK"
    assert np.abs(Qn.T @ Qn - np.eye(l)).max() < 2e-5
    # R: block upper triangular with upper-triangular diagonal blocks, i.e. upper
    assert np.all(np.tril(Rn, -1) == 0.0)
    assert np.all(np.diag(Rn) > 0.0)
    assert np.abs(Qn @ Rn - Q0).max() < 1e-5 * np.abs(Q0).max() * max(1.0, cond / 1e3)
    Qr, Rr, _ = oracle.cholqr2(Q0.astype(np.float32).astype(np.float64))
    assert oracle.max_principal_angle(Qr, Qn) < 50 * 6e-8 * cond * np.sqrt(l)
    if cond <= 1e3:  # Q and R themselves (R's diagonal positive on both sides)
        assert np.abs(Qn - Qr).max() < 1e-4
        assert np.abs(Rn - Rr).max() < 1e-5 * np.abs(Rr).max()


def test_wide_orthonormalize_matches_narrow_at_160(ne_small):
    """At l = 160 the single CholeskyQR2 runs; at 161 the panel path: the
    first 160 columns of the two Q factors agree to rounding (the same thin
    QR of the same columns)."""
    Q0 = cond_block(8000, 161, 1e2, 5)
    with isvd.graph_operator(ne_small, coeffs=C5) as op:
        Qa, _, _ = isvd.orthonormalize(op, torch.tensor(Q0[:, :160], dtype=torch.float32, device="cuda"))
        Qb, _, _ = isvd.orthonormalize(op, torch.tensor(Q0, dtype=torch.float32, device="cuda"))
    assert (Qa - Qb[:, :160]).abs().max().item() < 1e-5


# ---- the small SVD ---------------------------------------------------------------

# above 160 columns the grid form (blocks of two columns in global memory, one
# CTA per block pair); 161: one column in the last block
@pytest.mark.parametrize("l,cond,upper", [(161, 1e3, False), (256, 1e6, True), (384, 1e3, False), (460, 1e4, True),
                                          (480, 1e2, False), (512, 1e8, True)])
def test_wide_small_svd(ne_small, l, cond, upper):
    A = cond_block(l, l, cond, 31 + l)
    if upper:
        A = np.linalg.qr(A)[1]
    info = torch.zeros(4, dtype=torch.int32, device="cuda")
    with isvd.graph_operator(ne_small, coeffs=C5) as op:
        U, S, V = isvd.small_svd(op, torch.tensor(A, device="cuda"), info=info)
    inf = isvd.info_dict(info)
    assert inf["status"] == "OK" and 1 <= inf["iters_done"] < 60, inf  # converged within the sweep limit
    U, S, V = U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy()
    Sr = np.linalg.svd(A, compute_uv=False)
    assert np.allclose(S, Sr, rtol=1e-11, atol=1e-14 * Sr[0])
    assert np.abs((U * S) @ V.T - A).max() < 4e-13 * Sr[0]
    assert np.abs(U.T @ U - np.eye(l)).max() < max(1e-12, 1e-14 * cond)
    assert np.abs(V.T @ V - np.eye(l)).max() < 1e-12


# ---- Alg. 1 end to end ---------------------------------------------------------------

def _oracle_all(ref, l, q, seed):
    """The oracle's Alg. 1 with k = l (no oversample): all l Ritz triplets of
    the block; those of any k <= l with oversample l - k are its first k."""
    U, S, V, _ = ref.isvd(l, 0, q, seed)
    return U, S, V


# (graph, k, oversample, iters): l = 256 on the Cora-sized NE graph; l = 512
# (rank 256, l = 2k) on an Erdos-Renyi graph; l = 200 (ragged second panel)
WIDE_SVD = [("ne_small", 128, 128, 2), ("er1200", 256, 256, 1), ("er900", 150, 50, 2)]


@pytest.mark.parametrize("graph,k,p,q", WIDE_SVD)
def test_wide_svd_parity(ne_small, graph, k, p, q):
    g = {"ne_small": ne_small, "er1200": None, "er900": None}[graph]
    if graph == "er1200":
        g = synth.erdos_renyi(1200, 16.0, 41)
    elif graph == "er900":
        g = synth.erdos_renyi(900, 12.0, 43)
    l, seed = k + p, synth.BASE_SEED
    ref = oracle.graph_operator(g, coeffs=C5, ones_coeff=-LAM)
    Ua, Sa, Va = _oracle_all(ref, l, q, seed)
    Ur, Sr, Vr = Ua[:, :k], Sa[:k], Va[:, :k]
    with isvd.graph_operator(g, coeffs=C5, ones_coeff=-LAM) as gpu:
        U, S, V, info = gpu.svd(k, p, q, seed)
        inf = isvd.info_dict(info)
    assert inf["status"] == "OK", inf
    Un, Sn, Vn = npy(U), npy(S), npy(V)
    err = np.abs(Sn - Sr)
    assert np.all(err <= 1e-5 * Sr + 1e-6 * Sr[0]), (err / Sr).max()
    j = gapped_prefix(Sa, k)
    if j:
        assert oracle.max_principal_angle(Ur[:, :j], Un[:, :j]) < 1e-3
        assert oracle.max_principal_angle(Vr[:, :j], Vn[:, :j]) < 1e-3
    assert np.abs(Un.T @ Un - np.eye(k)).max() < 2e-5
    assert np.abs(Vn.T @ Vn - np.eye(k)).max() < 2e-5
    res = oracle.residuals(ref, Un, Sn, Vn)
    res_ref = oracle.residuals(ref, Ur, Sr, Vr)
    assert res.max() <= res_ref.max() + 1e-4 * Sr[0]
    print(dict(graph=graph, l=l, rel=float((err / Sr).max()), j=j, res=float(res.max()),
               res_ref=float(res_ref.max())))


def test_wide_limits(ne_small):
    """Above 512 columns, wide blocks in mixed precision and wide batched
    problems are refused before anything is launched."""
    g = synth.erdos_renyi(1200, 8.0, 3)
    with isvd.graph_operator(g, coeffs=[1.0]) as op:
        with pytest.raises(isvd.IsvdError) as e:
            op.svd(500, 13, 1, 0)
        assert e.value.name == "UNSUPPORTED"
        with pytest.raises(isvd.IsvdError) as e:
            op.svd(150, 50, 1, 0, precision="mixed")
        assert e.value.name == "UNSUPPORTED"
        with pytest.raises(isvd.IsvdError) as e:
            isvd.Batch([op], [150], oversample=50, iters=1).run()
        assert e.value.name == "UNSUPPORTED"
        with pytest.raises(isvd.IsvdError) as e:
            isvd.orthonormalize(op, torch.zeros((1000, 513), dtype=torch.float32, device="cuda")[:, :513])
        assert e.value.name == "SHAPE"
