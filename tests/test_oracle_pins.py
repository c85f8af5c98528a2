"""Pins for the FP64 oracle: each check ties an oracle function to something
other than itself (a published value, a closed form, LAPACK, an exact
invariant), so that a dropped term, a wrong sign or index or a transposed
operand in the oracle fails at least one of them.  CPU only."""
import itertools
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.stats

import oracle
from paper_2111_06312_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")
LAM = 0.05
C5 = oracle.ne_coefficients(5)


def poly(c, x):
    return sum(c[k] * x ** (k + 1) for k in range(len(c)))


# ---- Philox / Box-Muller (start block of Alg. 1) ----------------------------

def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLD, "philox4x32_10_kat.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = oracle.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_gaussian_is_standard_normal():
    z = oracle.gaussian(7, 4096, 48).ravel()
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1) < 0.01
    assert scipy.stats.kstest(z, "norm").pvalue > 1e-3
    # columns are uncorrelated
    Z = oracle.gaussian(11, 20000, 8)
    C = np.corrcoef(Z.T)
    assert np.abs(C - np.eye(8)).max() < 0.04


def test_gaussian_prefix_and_seed():
    # element (i, j) depends only on (seed, i, j): a narrower block is a prefix
    a = oracle.gaussian(5, 50, 42)
    b = oracle.gaussian(5, 50, 40)
    assert np.array_equal(a[:, :40], b)
    assert not np.allclose(oracle.gaussian(6, 50, 40), b)


# ---- coefficients (Eq. 3 read with Fig. 1) ----------------------------------

def test_context_weights_match_fig1():
    for l in open(os.path.join(GOLD, "fig1_context_weights.txt")):
        if not l.strip() or l[0] == "#":
            continue
        parts = l.split()
        Cw = int(parts[0])
        want = [float(Fraction(x)) for x in parts[1:]]
        assert np.allclose(oracle.ne_coefficients(Cw), want, rtol=0, atol=1e-15)
    assert np.allclose(C5, (6 - np.arange(1, 6)) / 15.0)
    assert abs(C5.sum() - 1) < 1e-15


# ---- closed-form spectra -----------------------------------------------------

@pytest.mark.parametrize("n", [7, 12, 13])
def test_cycle_spectrum_row(n):
    # T on C_n has eigenvalues cos(2 pi j / n), eigenvector 1 for j = 0; M is
    # symmetric (regular graph) so singular values are |eigenvalues|.
    g = synth.cycle(n)
    op = oracle.graph_operator(g, coeffs=C5, ones_coeff=-LAM)
    mu = np.cos(2 * np.pi * np.arange(n) / n)
    ev = poly(C5, mu)
    ev[0] = poly(C5, 1.0) - LAM * n
    want = np.sort(np.abs(ev))[::-1]
    M = op.explicit()
    _, S, _ = oracle.jacobi_svd(M)
    assert np.allclose(S, want, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("n", [6, 9])
def test_cycle_spectrum_with_adjacency_term(n):
    # Eq. 3 exactly: M = p(T) - lam (J - A).  On C_n, A = 2T.
    g = synth.cycle(n)
    op = oracle.graph_operator(g, coeffs=C5, ones_coeff=-LAM, adj_coeff=LAM)
    mu = np.cos(2 * np.pi * np.arange(n) / n)
    ev = poly(C5, mu) + LAM * 2 * mu
    ev[0] -= LAM * n
    want = np.sort(np.abs(ev))[::-1]
    _, S, _ = oracle.jacobi_svd(op.explicit())
    assert np.allclose(S, want, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("n", [5, 8])
def test_complete_graph_spectrum(n):
    g = synth.complete(n)
    op = oracle.graph_operator(g, coeffs=C5, ones_coeff=-LAM)
    ev = np.array([poly(C5, 1.0) - LAM * n] + [poly(C5, -1.0 / (n - 1))] * (n - 1))
    _, S, _ = oracle.jacobi_svd(op.explicit())
    assert np.allclose(S, np.sort(np.abs(ev))[::-1], rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("n", [7, 10])
def test_cycle_spectrum_sym(n):
    # Â on C_n: (A+I)/3, eigenvalues (1 + 2 cos(2 pi j/n)) / 3
    g = synth.cycle(n)
    op = oracle.graph_operator(g, norm="sym", coeffs=C5, ones_coeff=-LAM)
    mu = (1 + 2 * np.cos(2 * np.pi * np.arange(n) / n)) / 3
    ev = poly(C5, mu)
    ev[0] -= LAM * n
    _, S, _ = oracle.jacobi_svd(op.explicit())
    assert np.allclose(S, np.sort(np.abs(ev))[::-1], rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("n", [7, 10])
def test_cycle_spectrum_noself(n):
    # label re-use's adjacency Â - (D+I)^-1 (Sec. 5.3) on C_n: A/3, with
    # eigenvalues 2 cos(2 pi j/n) / 3; Â itself does not match
    g = synth.cycle(n)
    mu = 2 * np.cos(2 * np.pi * np.arange(n) / n) / 3
    ev = poly(C5, mu)
    ev[0] -= LAM * n
    want = np.sort(np.abs(ev))[::-1]
    _, S, _ = oracle.jacobi_svd(oracle.graph_operator(g, norm="sym_noself", coeffs=C5, ones_coeff=-LAM).explicit())
    assert np.allclose(S, want, rtol=1e-12, atol=1e-13)
    _, S1, _ = oracle.jacobi_svd(oracle.graph_operator(g, norm="sym", coeffs=C5, ones_coeff=-LAM).explicit())
    assert not np.allclose(S1, want, rtol=1e-6)


@pytest.mark.parametrize("n", [5, 8])
def test_complete_graph_spectrum_noself(n):
    # K_n: d = n - 1, so Â - (D+I)^-1 = (J - I)/n, eigenvalues (n-1)/n on 1
    # and -1/n (n - 1 times)
    g = synth.complete(n)
    op = oracle.graph_operator(g, norm="sym_noself", coeffs=C5, ones_coeff=-LAM)
    ev = np.array([poly(C5, (n - 1) / n) - LAM * n] + [poly(C5, -1.0 / n)] * (n - 1))
    _, S, _ = oracle.jacobi_svd(op.explicit())
    assert np.allclose(S, np.sort(np.abs(ev))[::-1], rtol=1e-12, atol=1e-13)


def test_noself_is_sym_minus_the_identity_term():
    # Â - (Â - (D+I)^-1) = diag(1/(d_i+1)); the diagonal of Â - (D+I)^-1 is
    # zero on a graph without self-loops (no label leakage from row i of Y
    # into row i of the propagated block, Sec. 5.3)
    g = synth.chung_lu(150, 700, 41, isolated_self_loops=False)
    d = np.diff(g.rowptr).astype(np.float64)
    assert (d > 0).any() and not np.any(np.repeat(np.arange(g.n), np.diff(g.rowptr)) == g.colidx)
    Ms = oracle.graph_operator(g, norm="sym", coeffs=[1.0]).explicit()
    M0 = oracle.graph_operator(g, norm="sym_noself", coeffs=[1.0]).explicit()
    assert np.allclose(Ms - M0, np.diag(1.0 / (d + 1.0)), rtol=0, atol=1e-15)
    assert np.all(np.diag(M0) == 0.0)
    assert np.allclose(M0, M0.T, rtol=0, atol=1e-15)


def test_label_reuse_blocks_do_not_leak():
    # [Y | N0 Y | N0^2 Y] with N0 = Â - (D+I)^-1 and Y one-hot on training
    # rows: row i of N0 Y does not depend on Y_i; with Â it does
    g = synth.chung_lu(200, 1000, 42, isolated_self_loops=False)
    rng = np.random.default_rng(43)
    y = 5
    Y = np.zeros((g.n, y))
    train = rng.choice(g.n, 120, replace=False)
    Y[train, rng.integers(0, y, 120)] = 1.0
    i = int(train[np.argmax(np.diff(g.rowptr)[train])])
    Y2 = Y.copy()
    Y2[i] = np.roll(Y[i], 1)
    for norm, leaks in (("sym_noself", False), ("sym", True)):
        m1 = oracle.graph_operator(g, form="concat", norm=norm, X=Y, L=2).explicit()
        m2 = oracle.graph_operator(g, form="concat", norm=norm, X=Y2, L=2).explicit()
        assert m1.shape == (g.n, 3 * y)
        assert np.array_equal(m1[i, :y] != m2[i, :y], Y[i] != Y2[i])  # block 0 is Y itself
        changed = not np.allclose(m1[i, y:2 * y], m2[i, y:2 * y], rtol=0, atol=0)
        assert changed == leaks


@pytest.mark.parametrize("L", [1, 2, 3])
def test_concat_identity_features(L):
    # X = I: M M^T = sum_l Â^(2l), sigma_j = sqrt(sum_l mu_j^(2l))
    n = 9
    g = synth.cycle(n)
    op = oracle.graph_operator(g, form="concat", norm="sym", X=np.eye(n), L=L)
    mu = (1 + 2 * np.cos(2 * np.pi * np.arange(n) / n)) / 3
    want = np.sqrt(sum(mu ** (2 * l) for l in range(L + 1)))
    M = op.explicit()
    assert M.shape == (n, n * (L + 1))
    _, S, _ = oracle.svd_any(M)
    assert np.allclose(S[:n], np.sort(want)[::-1], rtol=1e-12)


# ---- exact invariants on irregular graphs ------------------------------------

def _irregular(n=300, m=1400, seed=3):
    return synth.chung_lu(n, m, seed)


def test_row_operator_invariants():
    g = _irregular()
    d = g.degrees().astype(np.float64)
    op = oracle.graph_operator(g, coeffs=C5, ones_coeff=-LAM)
    one = np.ones(g.n)
    # T 1 = 1  =>  M 1 = (sum c - lam n) 1
    assert np.allclose(op.apply(one), (C5.sum() - LAM * g.n) * one, rtol=1e-13)
    # T^T d = d  =>  M^T d = (sum c) d - lam (1^T d) 1,   1^T d = nnz
    assert np.allclose(op.apply(d, transpose=True), C5.sum() * d - LAM * g.nnz * one, rtol=1e-12, atol=1e-9)
    # the transpose is not the forward operator on an irregular graph
    assert not np.allclose(op.apply(d), op.apply(d, transpose=True))


def test_sym_operator_invariant():
    g = _irregular()
    v = np.sqrt(g.degrees() + 1.0)
    op = oracle.graph_operator(g, norm="sym", coeffs=C5)
    assert np.allclose(op.apply(v), v, rtol=1e-13)  # Â v = v, sum c = 1
    assert np.allclose(op.apply(v, transpose=True), v, rtol=1e-13)


def test_weighted_row_operator():
    g = _irregular()
    rng = np.random.default_rng(0)
    w = rng.uniform(0.5, 2.0, g.nnz)
    # symmetric weights: w_ij = w_ji
    rows = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    key = np.minimum(rows, g.colidx) * g.n + np.maximum(rows, g.colidx)
    _, inv = np.unique(key, return_inverse=True)
    w = rng.uniform(0.5, 2.0, inv.max() + 1)[inv]
    op = oracle.graph_operator(g, values=w, coeffs=[1.0])
    one = np.ones(g.n)
    assert np.allclose(op.apply(one), one, rtol=1e-13)
    dw = np.bincount(rows, weights=w, minlength=g.n)
    assert np.allclose(op.apply(dw, transpose=True), dw, rtol=1e-12)


@pytest.mark.parametrize("form,norm", [("poly", "row"), ("poly", "sym"), ("concat", "sym"), ("concat", "row"),
                                       ("poly", "sym_noself"), ("concat", "sym_noself")])
def test_adjoint_identity(form, norm):
    g = _irregular(120, 500, 9)
    rng = np.random.default_rng(1)
    kw = dict(form=form, norm=norm)
    if form == "poly":
        kw.update(coeffs=C5, ones_coeff=-LAM, adj_coeff=0.02)
    else:
        x = synth.tfidf_features(g.n, 17, 0.2, 4)
        kw.update(X=(x.d, x.rowptr, x.colidx, x.values), L=2)
    op = oracle.graph_operator(g, **kw)
    r, c = op.shape
    G = rng.standard_normal((c, 5))
    H = rng.standard_normal((r, 5))
    lhs = np.sum(op.apply(G) * H)
    rhs = np.sum(G * op.apply(H, transpose=True))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1)


def _all_graphs(n):
    pairs = list(itertools.combinations(range(n), 2))
    for mask in range(1 << len(pairs)):
        e = [p for b, p in enumerate(pairs) if mask >> b & 1]
        deg = np.zeros(n, int)
        for a, b in e:
            deg[a] += 1
            deg[b] += 1
        yield synth.from_edges(n, e, self_loops=np.nonzero(deg == 0)[0])


def test_implicit_matches_explicit_all_graphs_n4():
    rng = np.random.default_rng(2)
    count = 0
    for g in _all_graphs(4):
        for norm in ("row", "sym", "sym_noself"):
            op = oracle.graph_operator(g, norm=norm, coeffs=C5, ones_coeff=-LAM, adj_coeff=0.3)
            M = op.explicit()
            G = rng.standard_normal((4, 3))
            assert np.abs(op.apply(G) - M @ G).max() <= 1e-13
            assert np.abs(op.apply(G, transpose=True) - M.T @ G).max() <= 1e-13
            count += 1
    assert count == 3 * 64


def test_implicit_matches_explicit_concat():
    g = _irregular(60, 240, 5)
    x = synth.tfidf_features(g.n, 7, 0.3, 8)
    op = oracle.graph_operator(g, form="concat", norm="sym", X=(x.d, x.rowptr, x.colidx, x.values), L=2)
    M = op.explicit()
    rng = np.random.default_rng(3)
    G = rng.standard_normal((M.shape[1], 4))
    H = rng.standard_normal((M.shape[0], 4))
    assert np.abs(op.apply(G) - M @ G).max() <= 1e-13
    assert np.abs(op.apply(H, transpose=True) - M.T @ H).max() <= 1e-13
    # block 0 of M is X itself
    Xd = np.zeros((g.n, x.d))
    for i in range(g.n):
        Xd[i, x.colidx[x.rowptr[i]:x.rowptr[i + 1]]] = x.values[x.rowptr[i]:x.rowptr[i + 1]]
    assert np.allclose(M[:, :x.d], Xd, rtol=0, atol=1e-7)


# ---- dense kernels: Jacobi SVD, Cholesky, CholeskyQR, Householder -----------

@pytest.mark.parametrize("shape,cond", [((50, 20), 1e2), ((30, 30), 1e8), ((200, 12), 1e12)])
def test_jacobi_matches_lapack(shape, cond):
    rng = np.random.default_rng(4)
    r, c = shape
    Ua, _ = np.linalg.qr(rng.standard_normal((r, c)))
    Va, _ = np.linalg.qr(rng.standard_normal((c, c)))
    s = np.geomspace(1.0, 1.0 / cond, c)
    A = (Ua * s) @ Va.T
    U, S, V = oracle.jacobi_svd(A)
    S_ref = np.linalg.svd(A, compute_uv=False)
    assert np.allclose(S, S_ref, rtol=1e-10, atol=1e-15 * S_ref[0])
    assert np.abs(U.T @ U - np.eye(c)).max() < 1e-12
    assert np.abs(V.T @ V - np.eye(c)).max() < 1e-12
    assert np.abs((U * S) @ V.T - A).max() < 1e-13 * S_ref[0]
    assert np.all(np.diff(S) <= 0)


def test_eckart_young():
    g = _irregular(80, 300, 12)
    op = oracle.graph_operator(g, coeffs=C5, ones_coeff=-LAM)
    M = op.explicit()
    U, S, V = oracle.jacobi_svd(M)
    for k in (1, 5, 20):
        E = M - (U[:, :k] * S[:k]) @ V[:, :k].T
        assert abs(np.sum(E * E) - np.sum(S[k:] ** 2)) <= 1e-10 * np.sum(S ** 2)


def test_cholesky_matches_lapack():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((40, 25))
    W = A.T @ A
    Lf, info = oracle.cholesky(W)
    assert info == 0
    assert np.allclose(Lf, np.linalg.cholesky(W), rtol=1e-12, atol=1e-12)
    W[3, 3] = -1.0
    _, info = oracle.cholesky(W)
    assert info == 4


def _cond_matrix(r, c, cond, seed):
    rng = np.random.default_rng(seed)
    Ua, _ = np.linalg.qr(rng.standard_normal((r, c)))
    Va, _ = np.linalg.qr(rng.standard_normal((c, c)))
    return (Ua * np.geomspace(1, 1 / cond, c)) @ Va.T


def test_cholqr_alg2():
    Q0 = _cond_matrix(500, 30, 1e3, 6)
    Q, R, info = oracle.cholqr(Q0)
    assert info == 0
    assert np.abs(Q.T @ Q - np.eye(30)).max() < 1e-9  # one pass: O(u cond^2)
    assert np.abs(Q @ R - Q0).max() < 1e-13
    assert np.allclose(R, np.triu(R))
    Qh, Rh = oracle.householder_qr(Q0)
    assert oracle.max_principal_angle(Qh, Q) < 1e-10  # same span (Alg. 2 footnote)
    Qn, Rn = np.linalg.qr(Q0)
    sg = np.sign(np.diag(Rn)) * np.sign(np.diag(Rh))
    assert np.allclose(Qh, Qn * sg, atol=1e-12)


@pytest.mark.parametrize("cond,passes", [(1e3, 2), (1e7, 2), (1e11, 3)])
def test_cholqr2_orthonormal(cond, passes):
    Q0 = _cond_matrix(800, 24, cond, 7)
    Q, R, p = oracle.cholqr2(Q0)
    assert p == passes
    assert np.abs(Q.T @ Q - np.eye(24)).max() < 1e-14 * 800
    assert np.abs(Q @ R - Q0).max() < 1e-12 * np.abs(Q0).max()
    Qh, _ = oracle.householder_qr(Q0)
    assert oracle.max_principal_angle(Qh, Q) < 1e-12 * cond


# ---- Alg. 1 ------------------------------------------------------------------

def test_isvd_cycle_closed_form():
    n = 64
    g = synth.cycle(n)
    op = oracle.graph_operator(g, coeffs=C5, ones_coeff=-LAM)
    mu = np.cos(2 * np.pi * np.arange(n) / n)
    ev = poly(C5, mu)
    ev[0] = poly(C5, 1.0) - LAM * n
    want = np.sort(np.abs(ev))[::-1]
    # k = 5 sits at a gap (pairs of equal values follow the first)
    U, S, V, _ = op.isvd(5, 10, 8, 99)
    assert want[4] - want[5] > 1e-3
    assert np.allclose(S, want[:5], rtol=1e-10)
    assert np.abs(U.T @ U - np.eye(5)).max() < 1e-13
    assert np.abs(V.T @ V - np.eye(5)).max() < 1e-13
    # vectors converge at the square root of the values' rate: more iterations
    U, S, V, _ = op.isvd(5, 10, 40, 99)
    assert oracle.residuals(op, U, S, V).max() < 1e-9


def test_isvd_error_falls_with_iterations():
    # Thm. 4 (Halko et al. Thm 1.2): error decays with the number of
    # iterations towards the optimal rank-k error.
    g = _irregular(250, 1200, 21)
    op = oracle.graph_operator(g, coeffs=C5, ones_coeff=-LAM)
    M = op.explicit()
    S_ref = np.linalg.svd(M, compute_uv=False)
    k = 10
    errs = []
    for q in (0, 1, 2, 4, 8):
        U, S, V, _ = op.isvd(k, 5, q, 4)
        E = M - (U * S) @ V.T
        errs.append(np.linalg.norm(E, 2))
        assert np.all(S <= S_ref[:k] * (1 + 1e-12))  # Ritz values never exceed the truth
    opt = S_ref[k]
    assert errs[-1] <= 1.05 * opt
    assert errs[0] <= 4 * opt * np.sqrt(250)
    assert errs[-1] <= errs[0]


def test_isvd_matches_lapack_when_gapped():
    g = _irregular(200, 1000, 22)
    op = oracle.graph_operator(g, norm="sym", coeffs=C5, ones_coeff=-LAM)
    M = op.explicit()
    Ur, Sr, Vrt = np.linalg.svd(M)
    k = int(np.argmax(np.diff(-Sr[:12]))) + 1  # largest gap among the top 12
    U, S, V, _ = op.isvd(k, 8, 10, 5)
    assert np.allclose(S, Sr[:k], rtol=1e-8)
    assert oracle.max_principal_angle(Ur[:, :k], U) < 1e-5
    assert oracle.max_principal_angle(Vrt[:k].T, V) < 1e-5


def test_isvd_concat_matches_lapack():
    g = _irregular(150, 600, 23)
    x = synth.tfidf_features(g.n, 20, 0.2, 24)
    op = oracle.graph_operator(g, form="concat", norm="sym", X=(x.d, x.rowptr, x.colidx, x.values), L=2)
    M = op.explicit()
    Sr = np.linalg.svd(M, compute_uv=False)
    U, S, V, _ = op.isvd(8, 8, 40, 6)  # sigma_8 / sigma_9 = 1.002: slow
    assert U.shape == (150, 8) and V.shape == (60, 8)
    assert np.allclose(S, Sr[:8], rtol=1e-10)


def test_isvd_ritz_prefix_consistency():
    # The start block for width l is the same whatever split k + p = l
    # (counter-based draw), so the Ritz values agree.
    g = _irregular(200, 900, 25)
    op = oracle.graph_operator(g, coeffs=C5, ones_coeff=-LAM)
    _, S1, _, _ = op.isvd(10, 6, 3, 8)
    _, S2, _, _ = op.isvd(16, 0, 3, 8)
    assert np.allclose(S1, S2[:10], rtol=1e-12)


# ---- sensitivity: plausible mistakes fail a pin -------------------------------

def test_pins_reject_planted_mistakes():
    n = 12
    g = synth.cycle(n)
    mu = np.cos(2 * np.pi * np.arange(n) / n)
    ev = poly(C5, mu)
    ev[0] = poly(C5, 1.0) - LAM * n
    want = np.sort(np.abs(ev))[::-1]
    # dropped all-ones term
    _, S, _ = oracle.jacobi_svd(oracle.graph_operator(g, coeffs=C5).explicit())
    assert not np.allclose(S, want, rtol=1e-6)
    # wrong sign of the all-ones term
    _, S, _ = oracle.jacobi_svd(oracle.graph_operator(g, coeffs=C5, ones_coeff=+LAM).explicit())
    assert not np.allclose(S, want, rtol=1e-6)
    # reversed coefficients (index slip c_k <-> c_{K+1-k})
    _, S, _ = oracle.jacobi_svd(oracle.graph_operator(g, coeffs=C5[::-1], ones_coeff=-LAM).explicit())
    assert not np.allclose(S, want, rtol=1e-6)
    # symmetric normalisation in place of T fails the row-stochastic invariant
    gi = _irregular()
    one = np.ones(gi.n)
    wrong = oracle.graph_operator(gi, norm="sym", coeffs=C5).apply(one)
    assert not np.allclose(wrong, one)


def test_lowrank_term_closed_form():
    # u v^T with v orthogonal to the all-ones vector and u = 1: on C_n the
    # matrix p(T) + a 1 v^T has p(T)'s spectrum deformed only in the 1
    # direction; check against the definition through its action instead:
    # (a u v^T) G = a u (v^T G) -- and the transpose swaps u and v.
    g = _irregular(100, 400, 31)
    rng = np.random.default_rng(7)
    u = rng.standard_normal((g.n, 2))
    v = rng.standard_normal((g.n, 2))
    al = np.array([0.3, -1.2])
    base = oracle.graph_operator(g, coeffs=C5)
    op = oracle.graph_operator(g, coeffs=C5, lowrank=(u, v, al))
    G = rng.standard_normal((g.n, 3))
    want = base.apply(G) + (u * al) @ (v.T @ G)
    assert np.allclose(op.apply(G), want, rtol=1e-13, atol=1e-12)
    want_t = base.apply(G, transpose=True) + (v * al) @ (u.T @ G)
    assert np.allclose(op.apply(G, transpose=True), want_t, rtol=1e-13, atol=1e-12)
    M = op.explicit()
    assert np.allclose(M @ G, want, rtol=1e-12, atol=1e-11)
    # rank-one all-ones coefficient equals the low-rank form with u = v = 1
    one = np.ones((g.n, 1))
    a1 = oracle.graph_operator(g, coeffs=C5, ones_coeff=-LAM).apply(G)
    a2 = oracle.graph_operator(g, coeffs=C5, lowrank=(one, one, [-LAM])).apply(G)
    assert np.allclose(a1, a2, rtol=1e-13, atol=1e-12)


@pytest.mark.parametrize("form", ["poly", "concat"])
def test_row_gather_is_a_row_selection(form):
    # M[rows, :] (the training-row fit of Thm. 1): a row selection of the
    # explicit matrix, whose products follow from the selection S (S M G and
    # M^T S^T H) and whose SVD is LAPACK's on the selected rows
    g = _irregular(120, 500, 26)
    rows = np.sort(np.random.default_rng(27).choice(g.n, 70, replace=False))
    kw = dict(norm="sym", coeffs=C5, ones_coeff=-LAM) if form == "poly" else dict(
        form="concat", norm="sym", X=np.random.default_rng(28).standard_normal((g.n, 9)), L=2)
    full = oracle.graph_operator(g, **kw)
    sub = oracle.graph_operator(g, gather_rows=rows, **kw)
    M = full.explicit()
    assert sub.shape == (70, M.shape[1])
    assert np.array_equal(sub.explicit(), M[rows])
    rng = np.random.default_rng(29)
    G = rng.standard_normal((M.shape[1], 5))
    H = rng.standard_normal((70, 5))
    assert np.allclose(sub.apply(G), M[rows] @ G, rtol=1e-12, atol=1e-12)
    assert np.allclose(sub.apply(H, transpose=True), M[rows].T @ H, rtol=1e-12, atol=1e-12)
    Sr = np.linalg.svd(M[rows], compute_uv=False)
    k = int(np.argmax(np.diff(-Sr[:8]))) + 1  # largest gap among the top 8
    _, S, _, _ = sub.isvd(k, 8, 12, 30)
    assert np.allclose(S, Sr[:k], rtol=1e-8)


# ---- embeddings and pair scores (Sec. 3.1) -----------------------------------

def test_embeddings_reach_the_eckart_young_error():
    # L R^T = U_k S_k V_k^T: ||M - L R^T||_F^2 is the tail sum of sigma^2
    # (LAPACK's SVD of the explicit matrix)
    g = _irregular(80, 360, 44)
    M = oracle.graph_operator(g, coeffs=C5, ones_coeff=-LAM).explicit()
    U, S, Vt = np.linalg.svd(M)
    for k in (1, 5, 20):
        Lm, Rm = oracle.embeddings(U[:, :k], S[:k], Vt[:k].T)
        err = np.linalg.norm(M - Lm @ Rm.T) ** 2
        assert abs(err - np.sum(S[k:] ** 2)) <= 1e-10 * np.sum(S ** 2)
        # both sides carry S^1/2: the column norms of L and R are sqrt(S)
        assert np.allclose(np.linalg.norm(Lm, axis=0), np.sqrt(S[:k]), rtol=1e-12)
        assert np.allclose(np.linalg.norm(Rm, axis=0), np.sqrt(S[:k]), rtol=1e-12)


def test_embeddings_coincide_for_a_psd_matrix():
    # Â^2 is symmetric PSD: its SVD has U = V, hence L = R (Sec. 3.1 on the
    # symmetric variant)
    g = _irregular(60, 260, 45)
    M = oracle.graph_operator(g, norm="sym", coeffs=[0.0, 1.0]).explicit()
    U, S, Vt = np.linalg.svd(M)
    k = 6
    assert S[k - 1] > S[k] * (1 + 1e-6)
    Lm, Rm = oracle.embeddings(U[:, :k], S[:k], Vt[:k].T)
    assert np.allclose(Lm, Rm, rtol=0, atol=1e-10)


def test_pair_scores_recover_entries_at_full_rank():
    # f(i, j) = <L_i, R_j> equals M_ij when k = rank(M); M = T (row
    # normalised, not symmetric) so that f(i, j) != f(j, i)
    g = _irregular(50, 220, 46)
    M = oracle.graph_operator(g, coeffs=[1.0]).explicit()
    U, S, Vt = np.linalg.svd(M)
    Lm, Rm = oracle.embeddings(U, S, Vt.T)
    rng = np.random.default_rng(47)
    src = rng.integers(0, g.n, 200)
    dst = rng.integers(0, g.n, 200)
    f = oracle.pair_scores(Lm, Rm, src, dst)
    assert np.allclose(f, M[src, dst], rtol=0, atol=1e-12)
    assert not np.allclose(oracle.pair_scores(Lm, Rm, dst, src), M[src, dst], rtol=0, atol=1e-6)


# ---- composite nodes (Sec. 4, App. A.3; Sec. 5.3's add-ons) ------------------------

C2 = np.array([0.3, -0.2])


@pytest.mark.parametrize("kind", ["sum", "hcat", "vcat", "product"])
def test_composite_cycle_spectra(kind):
    # on C_n, T = A/2 is symmetric with eigenvalues mu_j = cos(2 pi j/n) and
    # p(T), q(T) share its eigenvectors: sum -> |w1 p + w2 q|; [P | Q] and
    # [P ; Q] -> sqrt(p^2 + q^2); P Q -> |p q|
    n = 11
    g = synth.cycle(n)
    P = oracle.graph_operator(g, coeffs=C5)
    Q = oracle.graph_operator(g, coeffs=C2)
    mu = np.cos(2 * np.pi * np.arange(n) / n)
    p, q = poly(C5, mu), poly(C2, mu)
    w = (1.5, -0.7)
    want = {"sum": np.abs(w[0] * p + w[1] * q), "hcat": np.hypot(p, q), "vcat": np.hypot(p, q),
            "product": np.abs(p * q)}[kind]
    op = oracle.compose(kind, [P, Q], w if kind == "sum" else None)
    _, S, _ = oracle.svd_any(op.explicit())
    assert np.allclose(S[:n], np.sort(want)[::-1], rtol=1e-12, atol=1e-14)


def _mixed_children(g, seed):
    x = synth.tfidf_features(g.n, 11, 0.2, seed)
    X = (x.d, x.rowptr, x.colidx, x.values)
    a = oracle.graph_operator(g, coeffs=C5, ones_coeff=-LAM)
    b = oracle.graph_operator(g, norm="sym", coeffs=C2, adj_coeff=0.1)
    c = oracle.graph_operator(g, form="concat", norm="sym", X=X, L=2)
    d = oracle.graph_operator(g, form="concat", norm="sym_noself", X=X, L=1)
    return a, b, c, d


def test_composite_explicit_is_the_block_arrangement():
    # the C recursion against numpy's own stacking and matmul of the children
    g = _irregular(70, 300, 50)
    a, b, c, d = _mixed_children(g, 51)
    A, B, Cm, Dm = (o.explicit() for o in (a, b, c, d))
    assert np.allclose(oracle.compose("sum", [a, b], [2.0, -3.0]).explicit(), 2 * A - 3 * B, rtol=0, atol=1e-15)
    assert np.array_equal(oracle.compose("hcat", [a, c, d]).explicit(), np.hstack([A, Cm, Dm]))
    assert np.array_equal(oracle.compose("vcat", [a, b]).explicit(), np.vstack([A, B]))
    assert np.allclose(oracle.compose("product", [a, b, c]).explicit(), A @ B @ Cm, rtol=1e-13, atol=1e-15)
    nested = oracle.compose("hcat", [oracle.compose("sum", [a, b]), oracle.compose("product", [b, c])])
    assert np.allclose(nested.explicit(), np.hstack([A + B, B @ Cm]), rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("kind", ["sum", "hcat", "vcat", "product", "nested"])
def test_composite_products_match_explicit(kind):
    g = _irregular(90, 400, 52)
    a, b, c, d = _mixed_children(g, 53)
    op = {"sum": lambda: oracle.compose("sum", [a, b], [0.5, 2.0]),
          "hcat": lambda: oracle.compose("hcat", [a, c, d]),
          "vcat": lambda: oracle.compose("vcat", [c, oracle.compose("product", [b, c])]),
          "product": lambda: oracle.compose("product", [a, b, d]),
          "nested": lambda: oracle.compose("vcat", [oracle.compose("hcat", [a, c]), oracle.compose("hcat", [b, c])]),
          }[kind]()
    M = op.explicit()
    assert op.shape == M.shape
    rng = np.random.default_rng(54)
    G = rng.standard_normal((M.shape[1], 4))
    H = rng.standard_normal((M.shape[0], 4))
    assert np.allclose(op.apply(G), M @ G, rtol=1e-12, atol=1e-12)
    assert np.allclose(op.apply(H, transpose=True), M.T @ H, rtol=1e-12, atol=1e-12)
    lhs, rhs = np.sum(op.apply(G) * H), np.sum(G * op.apply(H, transpose=True))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1)


def test_composite_shapes_are_checked():
    g = _irregular(40, 160, 55)
    a, _, c, _ = _mixed_children(g, 56)
    for kind in ("sum", "vcat"):
        with pytest.raises(ValueError):
            oracle.compose(kind, [a, c])
    with pytest.raises(ValueError):
        oracle.compose("product", [c, a])  # 33 columns against n rows
    assert oracle.compose("hcat", [a, c]).shape == (g.n, g.n + c.shape[1])
    assert oracle.compose("product", [a, c]).shape == c.shape


def test_label_reuse_design_matrix():
    # Sec. 5.3: M_LR = [X | ÂX | Â^2 X | N0 Y | N0^2 Y], N0 = Â - (D+I)^-1, as
    # a side-by-side node whose second child is the product N0 [Y | N0 Y]
    g = synth.chung_lu(120, 500, 57, isolated_self_loops=False)
    X = np.random.default_rng(58).standard_normal((g.n, 6))
    y, mask = synth.labels(g.n, 4, 0.4, 59)
    Y = np.zeros((g.n, 4))
    Y[mask, y[mask]] = 1.0
    nc = oracle.graph_operator(g, form="concat", norm="sym", X=X, L=2)
    n0 = oracle.graph_operator(g, norm="sym_noself", coeffs=[1.0])
    lr = oracle.compose("hcat", [nc, oracle.compose("product", [n0, oracle.graph_operator(
        g, form="concat", norm="sym_noself", X=Y, L=1)])])
    N0 = n0.explicit()
    Ah = oracle.graph_operator(g, norm="sym", coeffs=[1.0]).explicit()
    want = np.hstack([X, Ah @ X, Ah @ Ah @ X, N0 @ Y, N0 @ N0 @ Y])
    assert np.allclose(lr.explicit(), want, rtol=1e-13, atol=1e-15)
    Sr = np.linalg.svd(want, compute_uv=False)
    k = int(np.argmax(-np.diff(Sr[:8]))) + 1
    _, S, _, _ = lr.isvd(k, 6, 10, 60)
    assert np.allclose(S, Sr[:k], rtol=1e-8)


def test_pseudo_dropout_rows_keep_the_width():
    # Sec. 5.3: [M ; PD(M)] has M's column count (the model keeps its
    # parameters); here PD drops feature entries of X at random
    g = _irregular(80, 320, 61)
    X = np.random.default_rng(62).standard_normal((g.n, 5))
    Xd = X * (np.random.default_rng(63).random(X.shape) >= 0.5) / 0.5
    m = oracle.graph_operator(g, form="concat", norm="sym", X=X, L=2)
    pd = oracle.graph_operator(g, form="concat", norm="sym", X=Xd, L=2)
    op = oracle.compose("vcat", [m, pd])
    assert op.shape == (2 * g.n, m.shape[1])
    assert np.array_equal(op.explicit(), np.vstack([m.explicit(), pd.explicit()]))


# ---- Gaussian-kernel edge function (Sec. 5.1, App. A.4) --------------------------------

def test_edge_kernel_grid_has_301_points():
    x = oracle.edge_kernel_grid()
    assert len(x) == 301 and x[0] == 0.5 and x[-1] == 2.0
    assert np.allclose(np.diff(x), 0.005, rtol=0, atol=1e-15)


@pytest.mark.parametrize("mu,s", [(1.2, 0.1), (1.0, 0.07), (1.5, 0.08)])
def test_edge_kernel_weights_match_the_truncated_normal_moment(mu, s):
    # E[S^X] = E[exp(a X)], a = log S, for X ~ N(mu, s) truncated to [0.5, 2]:
    # exp(a mu + a^2 s^2 / 2) (Phi(beta - a s) - Phi(alpha - a s)) / (Phi(beta) - Phi(alpha)).
    # The 301-point sum is a rectangle rule: exact to rounding when the density
    # is negligible at both ends of the interval (the cases here), O(h) otherwise.
    from scipy.special import ndtr
    S = np.array([3.0, 1.0, 0.4, 0.05, 1e-3])
    s_bar = np.log(1.0 / (2 * s * s))
    w, _, _ = oracle.edge_kernel_weights(S, mu, s_bar)
    a = np.log(S)
    al, be = (0.5 - mu) / s, (2.0 - mu) / s
    want = np.exp(a * mu + a * a * s * s / 2) * (ndtr(be - a * s) - ndtr(al - a * s)) / (ndtr(be) - ndtr(al))
    assert np.allclose(w, want, rtol=2e-8, atol=0)


def test_edge_kernel_reduces_to_the_svd_score():
    # mu = 1, s -> 0: w -> S, so f(i, j) = <U_i, V_j>_S (the no-op start of Sec. 5.1)
    S = np.array([5.0, 2.0, 0.7, 0.01])
    w, _, _ = oracle.edge_kernel_weights(S, 1.0, np.log(1.0 / (2 * 1e-4 ** 2)))
    assert np.allclose(w, S, rtol=1e-12, atol=0)


def test_edge_kernel_gradient_is_the_derivative():
    # central differences of the loss (and of w) in mu and s_bar
    rng = np.random.default_rng(70)
    n, k = 60, 6
    U = rng.standard_normal((n, k)) / 3
    V = rng.standard_normal((n, k)) / 3
    S = np.sort(rng.uniform(0.2, 4.0, k))[::-1]
    pos = (rng.integers(0, n, 40), rng.integers(0, n, 40))
    neg = (rng.integers(0, n, 90), rng.integers(0, n, 90))
    mu, sb = 1.1, np.log(1.0 / (2 * 0.2 ** 2))
    _, gm, gs = oracle.edge_kernel_loss(U, S, V, mu, sb, pos, neg, 10.0)
    h = 1e-5
    Lp = oracle.edge_kernel_loss(U, S, V, mu + h, sb, pos, neg, 10.0)[0]
    Lm = oracle.edge_kernel_loss(U, S, V, mu - h, sb, pos, neg, 10.0)[0]
    assert abs((Lp - Lm) / (2 * h) - gm) <= 1e-7 * (abs(gm) + 1e-3)
    Lp = oracle.edge_kernel_loss(U, S, V, mu, sb + h, pos, neg, 10.0)[0]
    Lm = oracle.edge_kernel_loss(U, S, V, mu, sb - h, pos, neg, 10.0)[0]
    assert abs((Lp - Lm) / (2 * h) - gs) <= 1e-7 * (abs(gs) + 1e-3)
    w0, dwm, dws = oracle.edge_kernel_weights(S, mu, sb)
    wp = oracle.edge_kernel_weights(S, mu + h, sb)[0]
    wm = oracle.edge_kernel_weights(S, mu - h, sb)[0]
    assert np.allclose((wp - wm) / (2 * h), dwm, rtol=1e-7, atol=1e-10)


def test_edge_kernel_loss_is_the_cross_entropy_of_the_svd_scores():
    # at the no-op start and full rank, f = M_ij: Eq. 9 on the explicit entries
    g = _irregular(40, 160, 71)
    M = oracle.graph_operator(g, norm="sym", coeffs=[1.0]).explicit()
    U, S, Vt = np.linalg.svd(M)
    rng = np.random.default_rng(72)
    rows = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    pos = (rows[:50], g.colidx[:50])  # edges of A
    neg = (rng.integers(0, g.n, 70), rng.integers(0, g.n, 70))
    L, _, _ = oracle.edge_kernel_loss(U, S, Vt.T, 1.0, np.log(1.0 / (2 * 1e-4 ** 2)), pos, neg, 10.0)
    fp, fn = M[pos], M[neg]
    want = np.mean(-np.log(1 / (1 + np.exp(-fp)))) + 10.0 * np.mean(-np.log(1 - 1 / (1 + np.exp(-fn))))
    assert abs(L - want) <= 1e-12 * abs(want)


# ---- Split-ReLU network (Sec. 5.2, Thm. 2) ----------------------------------------------

def test_split_relu_is_linear_on_the_hyperplane():
    rng = np.random.default_rng(80)
    X = rng.standard_normal((30, 7))
    W = rng.standard_normal((7, 4))
    assert np.allclose(oracle.split_relu(X, W, -W), X @ W, rtol=0, atol=1e-14)
    # Wn = 0: a plain ReLU layer
    assert np.array_equal(oracle.split_relu(X, W, np.zeros_like(W)), np.maximum(X @ W, 0))


@pytest.mark.parametrize("L", [1, 2, 3])
def test_splitrelu_network_at_init_is_the_linear_model(L):
    # Thm. 2: with Wp = I, Wn = -I, Wop = W*_l, Won = -W*_l the network equals
    # [X | ÂX | ... | Â^L X] W*, the explicit design matrix of Eq. 6 times W*
    g = _irregular(80, 320, 81)
    d, y = 5, 3
    rng = np.random.default_rng(82)
    X = rng.standard_normal((g.n, d))
    W_star = rng.standard_normal((d * (L + 1), y))
    Ah = oracle.graph_operator(g, norm="sym", coeffs=[1.0])
    out, _ = oracle.splitrelu_forward(Ah.apply, X, *oracle.splitrelu_init(W_star, d, L))
    M = oracle.graph_operator(g, form="concat", norm="sym", X=X, L=L).explicit()
    assert np.allclose(out, M @ W_star, rtol=1e-12, atol=1e-12)


def test_splitrelu_gradients_are_the_derivative():
    g = _irregular(40, 160, 83)
    d, y, L = 4, 3, 2
    rng = np.random.default_rng(84)
    X = rng.standard_normal((g.n, d))
    Ah = oracle.graph_operator(g, norm="sym", coeffs=[1.0])
    prop = Ah.apply
    prop_T = lambda G: Ah.apply(G, transpose=True)  # noqa: E731
    Wp = [rng.standard_normal((d, d)) for _ in range(L)]
    Wn = [rng.standard_normal((d, d)) for _ in range(L)]
    Wop = [rng.standard_normal((d, y)) for _ in range(L + 1)]
    Won = [rng.standard_normal((d, y)) for _ in range(L + 1)]
    R = rng.standard_normal((g.n, y))
    weights = (Wp, Wn, Wop, Won)
    out, cache = oracle.splitrelu_forward(prop, X, *weights)
    grads = oracle.splitrelu_backward(prop_T, cache, weights, R)

    def loss():
        return float(np.sum(oracle.splitrelu_forward(prop, X, *weights)[0] * R))

    h = 1e-6
    for group, ggroup in zip(weights, grads):
        for W, dW in zip(group, ggroup):
            for (a, b) in [(0, 0), (W.shape[0] - 1, W.shape[1] - 1), (1, 2)]:
                old = W[a, b]
                W[a, b] = old + h
                lp = loss()
                W[a, b] = old - h
                lm = loss()
                W[a, b] = old
                assert abs((lp - lm) / (2 * h) - dW[a, b]) <= 1e-6 * (1 + abs(dW[a, b]))


@pytest.mark.parametrize("p", [1, 2, 3])
def test_scalar_and_power_nodes_on_a_cycle(p):
    # on C_n: w p(T) has singular values |w p(mu)|, p(T)^p has |p(mu)|^p
    n = 9
    g = synth.cycle(n)
    P = oracle.graph_operator(g, coeffs=C5)
    mu = np.cos(2 * np.pi * np.arange(n) / n)
    _, S, _ = oracle.svd_any(oracle.power(P, p).explicit())
    assert np.allclose(S, np.sort(np.abs(poly(C5, mu)) ** p)[::-1], rtol=1e-12, atol=1e-15)
    _, S, _ = oracle.svd_any(oracle.scale(P, -2.5).explicit())
    assert np.allclose(S, np.sort(2.5 * np.abs(poly(C5, mu)))[::-1], rtol=1e-12, atol=1e-15)
    # T^p as a power node equals the polynomial leaf with c_p = 1
    T = oracle.graph_operator(g, coeffs=[1.0])
    Tp = oracle.graph_operator(g, coeffs=[0.0] * (p - 1) + [1.0])
    assert np.allclose(oracle.power(T, p).explicit(), Tp.explicit(), rtol=0, atol=1e-15)


def test_gather_pushed_to_the_leaves_selects_composite_rows():
    # (the reading for Gather on a tree) [A | C][rows] = [A[rows] | C[rows]] and
    # (A + B)[rows] = A[rows] + B[rows]
    g = _irregular(70, 300, 85)
    x = synth.tfidf_features(g.n, 9, 0.2, 86)
    X = (x.d, x.rowptr, x.colidx, x.values)
    rows = np.sort(np.random.default_rng(87).choice(g.n, 25, replace=False))
    a, b, c = (dict(coeffs=C5, ones_coeff=-LAM), dict(norm="sym", coeffs=C2),
               dict(form="concat", norm="sym", X=X, L=2))
    full_h = oracle.compose("hcat", [oracle.graph_operator(g, **a), oracle.graph_operator(g, **c)]).explicit()
    sub_h = oracle.compose("hcat", [oracle.graph_operator(g, gather_rows=rows, **a),
                                    oracle.graph_operator(g, gather_rows=rows, **c)]).explicit()
    assert np.array_equal(sub_h, full_h[rows])
    full_s = oracle.compose("sum", [oracle.graph_operator(g, **a), oracle.graph_operator(g, **b)]).explicit()
    sub_s = oracle.compose("sum", [oracle.graph_operator(g, gather_rows=rows, **a),
                                   oracle.graph_operator(g, gather_rows=rows, **b)]).explicit()
    assert np.array_equal(sub_s, full_s[rows])


def test_edge_score_at_the_start_is_the_embedding_score():
    # w = S at mu = 1, s -> 0: U_i^T diag(w) V_j = <L_i, R_j> with L = U S^1/2, R = V S^1/2
    rng = np.random.default_rng(88)
    U = rng.standard_normal((30, 5))
    V = rng.standard_normal((25, 5))
    S = np.array([4.0, 2.5, 1.0, 0.3, 0.02])
    w, _, _ = oracle.edge_kernel_weights(S, 1.0, np.log(1.0 / (2 * 1e-4 ** 2)))
    src, dst = rng.integers(0, 30, 40), rng.integers(0, 25, 40)
    Lm, Rm = oracle.embeddings(U, S, V)
    assert np.allclose(oracle.edge_scores(U, V, w, src, dst), oracle.pair_scores(Lm, Rm, src, dst),
                       rtol=1e-12, atol=1e-12)


def test_splitrelu_head_gradients_at_init_are_the_linear_models():
    # at the start dWop_l - dWon_l = H_l^T R with H_l = Â^l X, i.e. block l of
    # M^T R for M = [X | ÂX | ... | Â^L X] (the gradient of the linear model)
    g = _irregular(60, 250, 89)
    d, y, L = 4, 3, 2
    rng = np.random.default_rng(90)
    X = rng.standard_normal((g.n, d))
    W_star = rng.standard_normal((d * (L + 1), y))
    R = rng.standard_normal((g.n, y))
    Ah = oracle.graph_operator(g, norm="sym", coeffs=[1.0])
    weights = oracle.splitrelu_init(W_star, d, L)
    _, cache = oracle.splitrelu_forward(Ah.apply, X, *weights)
    _, _, dWop, dWon = oracle.splitrelu_backward(lambda G: Ah.apply(G, transpose=True), cache, weights, R)
    MtR = oracle.graph_operator(g, form="concat", norm="sym", X=X, L=L).apply(R, transpose=True)
    for l in range(L + 1):
        assert np.allclose(dWop[l] - dWon[l], MtR[d * l:d * (l + 1)], rtol=1e-11, atol=1e-11)


def test_new_pins_reject_planted_mistakes():
    # plausible slips in the newer oracle functions, each caught by its pin
    rng = np.random.default_rng(91)
    # embeddings with S in place of S^1/2: L R^T = U S^2 V^T misses Eckart-Young
    g = _irregular(50, 220, 92)
    M = oracle.graph_operator(g, coeffs=C5, ones_coeff=-LAM).explicit()
    U, S, Vt = np.linalg.svd(M)
    k = 5
    bad = (U[:, :k] * S[:k]) @ (Vt[:k].T * S[:k]).T
    assert abs(np.linalg.norm(M - bad) ** 2 - np.sum(S[k:] ** 2)) > 1e-6 * np.sum(S ** 2)
    # softmax of +(x - mu)^2 exp(s_bar) (sign slip) misses the truncated-normal moment
    from scipy.special import ndtr
    Sv = np.array([3.0, 0.4])
    mu, s = 1.2, 0.1
    sb = np.log(1 / (2 * s * s))
    x = oracle.edge_kernel_grid()
    z = (x - mu) ** 2 * np.exp(sb)
    pi = np.exp(z - z.max())
    pi /= pi.sum()
    a = np.log(Sv)
    al, be = (0.5 - mu) / s, (2.0 - mu) / s
    want = np.exp(a * mu + a * a * s * s / 2) * (ndtr(be - a * s) - ndtr(al - a * s)) / (ndtr(be) - ndtr(al))
    assert not np.allclose(pi @ (Sv[None, :] ** x[:, None]), want, rtol=1e-3)
    # Split-ReLU started with Wn = +I is not the linear model of Thm. 2
    d, y, L = 3, 2, 2
    X = rng.standard_normal((g.n, d))
    W_star = rng.standard_normal((d * (L + 1), y))
    Ah = oracle.graph_operator(g, norm="sym", coeffs=[1.0])
    Wp, Wn, Wop, Won = oracle.splitrelu_init(W_star, d, L)
    out_bad, _ = oracle.splitrelu_forward(Ah.apply, X, Wp, [-w for w in Wn], Wop, Won)
    Mc = oracle.graph_operator(g, form="concat", norm="sym", X=X, L=L).explicit()
    assert not np.allclose(out_bad, Mc @ W_star, rtol=1e-6)
    # side-by-side children in the wrong order fail the block arrangement
    P = oracle.graph_operator(g, coeffs=C5)
    Q = oracle.graph_operator(g, norm="sym", coeffs=C2)
    assert not np.allclose(oracle.compose("hcat", [Q, P]).explicit(), np.hstack([P.explicit(), Q.explicit()]))


@pytest.mark.parametrize("n", [4, 7])
def test_complete_graph_spectrum_sym(n):
    # Â on K_n is (A + I)/n = J/n: eigenvalues 1 (on the all-ones vector) and 0
    g = synth.complete(n)
    op = oracle.graph_operator(g, norm="sym", coeffs=C5, ones_coeff=-LAM)
    ev = np.array([poly(C5, 1.0) - LAM * n] + [0.0] * (n - 1))
    _, S, _ = oracle.jacobi_svd(op.explicit())
    assert np.allclose(S, np.sort(np.abs(ev))[::-1], rtol=1e-12, atol=1e-13)


def test_implicit_matches_explicit_all_graphs_n5():
    # every undirected graph on 5 nodes (isolated nodes with self-loops), both
    # normalisations with all correction terms
    rng = np.random.default_rng(93)
    count = 0
    for g in _all_graphs(5):
        for norm in ("row", "sym"):
            op = oracle.graph_operator(g, norm=norm, coeffs=C5, ones_coeff=-LAM, adj_coeff=0.3)
            M = op.explicit()
            G = rng.standard_normal((5, 2))
            assert np.abs(op.apply(G) - M @ G).max() <= 1e-12
            assert np.abs(op.apply(G, transpose=True) - M.T @ G).max() <= 1e-12
            count += 1
    assert count == 2 * 1024


@pytest.mark.parametrize("r,c,rank", [(20, 10, 3), (12, 12, 1), (40, 8, 5), (9, 9, 0)])
def test_jacobi_on_rank_deficient_matrices(r, c, rank):
    # exact zero singular values (the case that once kept the sweep from
    # converging): LAPACK's spectrum, and orthonormal factors on the range
    rng = np.random.default_rng(94 + r + c + rank)
    A = rng.standard_normal((r, rank)) @ rng.standard_normal((rank, c)) if rank else np.zeros((r, c))
    U, S, V = oracle.jacobi_svd(A)
    want = np.linalg.svd(A, compute_uv=False)
    assert np.allclose(S, want, rtol=1e-12, atol=1e-13 * max(1.0, want[0] if len(want) else 0.0))
    assert np.allclose(V.T @ V, np.eye(c), atol=1e-12)
    if rank:
        assert np.allclose((U[:, :rank] * S[:rank]) @ V[:, :rank].T, A, atol=1e-12 * np.abs(A).max())


def test_jacobi_on_clustered_spectra():
    # a 6-fold exact cluster among distinct values (degenerate clusters rotate
    # freely; the values must not)
    rng = np.random.default_rng(95)
    Qa, _ = np.linalg.qr(rng.standard_normal((30, 10)))
    Qb, _ = np.linalg.qr(rng.standard_normal((10, 10)))
    s = np.array([5.0, 3.0, 2.0, 2.0, 2.0, 2.0, 2.0, 2.0, 0.5, 1e-3])
    A = (Qa * s) @ Qb.T
    _, S, _ = oracle.jacobi_svd(A)
    assert np.allclose(S, s, rtol=1e-12, atol=1e-14)


def test_jacobi_after_householder_is_the_same_spectrum():
    # the tall-matrix route: Householder QR first, Jacobi on the c x c R
    rng = np.random.default_rng(96)
    A = rng.standard_normal((300, 12)) * np.geomspace(1, 1e-6, 12)
    _, S1, _ = oracle.jacobi_svd(A)
    _, R = oracle.householder_qr(A)
    _, S2, _ = oracle.jacobi_svd(R)
    assert np.allclose(S1, S2, rtol=1e-10, atol=0)


def test_rayleigh_ritz_routes_agree():
    # the GPU's route for Alg. 1's svd(B): B^T = Qt R (CholeskyQR2), SVD of R^T
    # = Ur diag(s) Vr^T gives B = R^T Qt^T = Ur diag(s) (Qt Vr)^T; the oracle
    # takes the one-sided Jacobi of B^T directly.  Same values, same subspaces.
    rng = np.random.default_rng(97)
    Bt = rng.standard_normal((400, 14)) * np.geomspace(1, 1e-3, 14)
    W, s_direct, UB = oracle.jacobi_svd(Bt)  # B^T = W diag(s) UB^T
    Qt, R, _ = oracle.cholqr2(Bt)
    Ur, s_route, Vr = oracle.jacobi_svd(R.T)  # R^T = Ur diag(s) Vr^T
    assert np.allclose(s_route, s_direct, rtol=1e-10)
    # left singular vectors of B: UB (direct) and Ur (route); right: W and Qt Vr
    assert oracle.max_principal_angle(UB[:, :5], Ur[:, :5]) < 1e-10
    assert oracle.max_principal_angle(W[:, :5], (Qt @ Vr)[:, :5]) < 1e-10


def test_isvd_block_wider_than_the_rank_breaks_down():
    # Â on K_n with the all-ones term has rank one: a block of width k + p > 1
    # leaves CholeskyQR a singular Gram matrix that no shift repairs (the range
    # has fewer directions than the block), and the oracle reports it; at
    # k + p <= rank it recovers the spectrum (here T on C_8, rank 6)
    g = synth.complete(6)
    op = oracle.graph_operator(g, norm="sym", coeffs=C5, ones_coeff=-LAM)
    assert np.linalg.matrix_rank(op.explicit()) == 1
    with pytest.raises(RuntimeError, match="isvd failed"):
        op.isvd(2, 3, 2, 1)
    c8 = oracle.graph_operator(synth.cycle(8), coeffs=[1.0])
    _, S, _, _ = c8.isvd(3, 3, 3, 2)
    assert np.allclose(S, [1.0, 1.0, np.sqrt(0.5)], rtol=1e-12)


def test_weighted_sym_and_noself_invariants():
    # weighted symmetric A, d = A 1: Â (D+I)^1/2 1 = (D+I)^1/2 1 and
    # (Â - (D+I)^-1) (D+I)^1/2 1 = (D+I)^-1/2 d (both directions: symmetric)
    g = _irregular()
    rows = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    key = np.minimum(rows, g.colidx) * g.n + np.maximum(rows, g.colidx)
    _, inv = np.unique(key, return_inverse=True)
    w = np.random.default_rng(98).uniform(0.5, 2.0, inv.max() + 1)[inv]
    dw = np.bincount(rows, weights=w, minlength=g.n)
    v = np.sqrt(dw + 1.0)
    sym = oracle.graph_operator(g, norm="sym", values=w, coeffs=[1.0])
    n0 = oracle.graph_operator(g, norm="sym_noself", values=w, coeffs=[1.0])
    for tr in (False, True):
        assert np.allclose(sym.apply(v, transpose=tr), v, rtol=1e-13)
        assert np.allclose(n0.apply(v, transpose=tr), dw / v, rtol=1e-13)
