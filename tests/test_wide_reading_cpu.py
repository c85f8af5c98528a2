"""The reading behind block widths above 160 (no GPU): orthonormalising a
block in 128-column panels by block Gram-Schmidt with two projections, each
panel then by CholeskyQR2, gives the thin QR with a positive diagonal of R,
the same Q and R that the oracle's CholeskyQR2 of the whole block gives (the
thin QR of a full-rank block is unique).  Written here in FP64 numpy, panel by
panel as the GPU path takes them, and compared with oracle.cholqr2."""
import numpy as np
import pytest

import oracle


@pytest.fixture(scope="module", autouse=True)
def built():
    oracle.build()


def panel_qr(Q0, panel=128):
    Q = Q0.copy()
    n, l = Q.shape
    R = np.zeros((l, l))
    for j0 in range(0, l, panel):
        j1 = min(l, j0 + panel)
        Y = Q[:, j0:j1]
        for _ in range(2):  # two projections off the panels before it
            if j0 == 0:
                break
            C = Q[:, :j0].T @ Y
            Y = Y - Q[:, :j0] @ C
            R[:j0, j0:j1] += C
        Qj, Rj, _ = oracle.cholqr2(Y)
        Q[:, j0:j1] = Qj
        R[j0:j1, j0:j1] = Rj
    return Q, R


@pytest.mark.parametrize("n,l,cond", [(3000, 300, 1e2), (2000, 161, 1e3), (4000, 512, 1e1)])
def test_panel_qr_is_the_thin_qr(n, l, cond):
    rng = np.random.default_rng(l)
    Ua, _ = np.linalg.qr(rng.standard_normal((n, l)))
    Va, _ = np.linalg.qr(rng.standard_normal((l, l)))
    Q0 = (Ua * np.geomspace(1, 1 / cond, l)) @ Va.T
    Qp, Rp = panel_qr(Q0)
    Qr, Rr, _ = oracle.cholqr2(Q0)
    assert np.all(np.tril(Rp, -1) == 0.0) and np.all(np.diag(Rp) > 0)
    assert np.abs(Qp.T @ Qp - np.eye(l)).max() < 1e-12
    assert np.abs(Qp @ Rp - Q0).max() < 1e-12 * np.abs(Q0).max()
    assert np.abs(Qp - Qr).max() < 1e-9 * cond
    assert np.abs(Rp - Rr).max() < 1e-11 * cond * np.abs(Rr).max()
