"""Pins for the oracle's gradient and closed-form pieces of the linear model
Y = M W on M = [X | Â X | Â^2 X] (Eq. 6; Sec. 3.3): the transposed product
against central finite differences of the forward product, and the closed
form of Thm. 1 against LAPACK least squares / the pseudo-inverse.  CPU only."""
import numpy as np
import pytest

import oracle
from paper_2111_06312_gb300 import synth


@pytest.fixture(scope="module")
def sub():
    g, x, y, train = synth.workload_finetune_sub(2000)
    op = oracle.graph_operator(g, form="concat", norm="sym", X=x.astype(np.float64), L=2)
    return g, x, y, train, op


def test_finite_difference_gradient(sub):
    """f(W) = 1/2 ||M W - T||_F^2 has gradient M^T (M W - T).  f is quadratic,
    so central differences are exact up to rounding."""
    _, _, _, _, op = sub
    r, c = op.shape
    assert (r, c) == (2000, 3 * 128)
    rng = np.random.default_rng(11)
    W = rng.standard_normal((c, 40)) * 0.1
    T = rng.standard_normal((r, 40))

    def f(W_):
        R = op.apply(W_) - T
        return 0.5 * float(np.sum(R * R))

    grad = op.apply(op.apply(W) - T, transpose=True)
    h = 1e-3
    scale = np.abs(grad).max()
    for _ in range(16):
        i, j = int(rng.integers(c)), int(rng.integers(40))
        E = np.zeros_like(W)
        E[i, j] = h
        fd = (f(W + E) - f(W - E)) / (2 * h)
        assert abs(fd - grad[i, j]) <= 1e-6 * scale, (i, j, fd, grad[i, j])


def test_finite_difference_catches_a_wrong_transpose(sub):
    """Planted mistake: using M^T without the Â factors (i.e. [X | X | X]^T)
    must fail the same finite-difference check."""
    _, x, _, _, op = sub
    r, c = op.shape
    rng = np.random.default_rng(12)
    W = rng.standard_normal((c, 8)) * 0.1
    T = rng.standard_normal((r, 8))
    R = op.apply(W) - T
    wrong = np.vstack([x.T.astype(np.float64) @ R] * 3)
    i, j = 200, 3  # a row of the Â X block
    E = np.zeros_like(W)
    h = 1e-3
    E[i, j] = h
    f = lambda W_: 0.5 * float(np.sum((op.apply(W_) - T) ** 2))
    fd = (f(W + E) - f(W - E)) / (2 * h)
    assert abs(fd - wrong[i, j]) > 1e-3 * np.abs(wrong).max()


def _small_concat(dup_columns=False):
    g = synth.chung_lu(60, 240, 5)
    x = synth.dense_features(60, 8, 6).astype(np.float64)
    if dup_columns:
        x[:, 7] = x[:, 6]  # rank-deficient M
    return oracle.graph_operator(g, form="concat", norm="sym", X=x, L=2)


def test_closed_form_equals_least_squares():
    op = _small_concat()
    M = op.explicit()
    U, S, V = oracle.svd_any(M)
    rng = np.random.default_rng(3)
    Y = rng.standard_normal((M.shape[0], 5))
    W = oracle.closed_form(U, S, V, Y)
    W_ls = np.linalg.lstsq(M, Y, rcond=None)[0]
    assert np.abs(W - W_ls).max() <= 1e-9 * np.abs(W_ls).max()


def test_closed_form_rank_deficient_equals_pinv():
    op = _small_concat(dup_columns=True)
    M = op.explicit()
    U, S, V = oracle.svd_any(M)
    assert S[-3] < 1e-12 * S[0] and S[-4] > 1e-3 * S[0]  # three duplicated columns
    rng = np.random.default_rng(4)
    Y = rng.standard_normal((M.shape[0], 5))
    W = oracle.closed_form(U, S, V, Y, rcond=1e-10)
    W_p = np.linalg.pinv(M, rcond=1e-10) @ Y
    assert np.abs(W - W_p).max() <= 1e-8 * np.abs(W_p).max()
    # normal equations hold and W has no component in the null space
    assert np.abs(M.T @ (M @ W - Y)).max() <= 1e-9 * np.abs(M.T @ Y).max()
    null = V[:, S < 1e-10 * S[0]]
    assert np.abs(null.T @ W).max() <= 1e-9 * np.abs(W).max()


def test_closed_form_truncated_is_projection():
    """Rank-k truncation: M W = U_k U_k^T Y (the fit is the projection of Y
    onto the top-k left singular subspace)."""
    op = _small_concat()
    M = op.explicit()
    U, S, V = oracle.svd_any(M)
    k = 6
    rng = np.random.default_rng(5)
    Y = rng.standard_normal((M.shape[0], 4))
    W = oracle.closed_form(U[:, :k], S[:k], V[:, :k], Y)
    assert np.abs(M @ W - U[:, :k] @ (U[:, :k].T @ Y)).max() <= 1e-9 * np.abs(Y).max()
