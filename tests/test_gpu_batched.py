"""Many independent problems in one call (isvd_svd_batched): every problem's
result must equal, bit for bit, that of its own isvd_svd call with the same
arguments (the kernels and their launch shapes are the same; only the
scheduling differs), and match the FP64 oracle like a single call does."""
import numpy as np
import pytest
import torch

import oracle
from paper_2111_06312_gb300 import build, isvd, synth

pytestmark = pytest.mark.gpu
LAM = 0.05
C5 = oracle.ne_coefficients(5)
SEED = 20211106315


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    build.build()
    oracle.build()


@pytest.fixture(scope="module")
def problems():
    sizes = [700, 1500, 3100, 900, 2500, 4000, 520]
    ranks = [16, 32, 64, 16, 32, 8, 16]
    graphs = []
    for i, n in enumerate(sizes):
        if i % 2 == 0:
            graphs.append(synth.erdos_renyi(n, 8.0, 900 + i))
        else:
            graphs.append(synth.chung_lu(n, 8 * n, 900 + i))
    ops = [isvd.graph_operator(g, coeffs=C5, ones_coeff=-LAM) for g in graphs]
    yield graphs, ops, ranks
    for op in ops:
        op.close()


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_batched_equals_single_calls(problems, precision):
    graphs, ops, ranks = problems
    batch = isvd.Batch(ops, ranks, oversample=10, iters=4, seed=SEED, precision=precision)
    U, S, V = batch.run()
    U = [u.clone() for u in U]
    S = [s.clone() for s in S]
    V = [v.clone() for v in V]
    assert isvd.Batch.kernel_nodes() > 0
    for i, (op, k) in enumerate(zip(ops, ranks)):
        u, s, v, info = op.svd(k, 10, 4, seed=SEED + i, precision=precision)
        assert torch.equal(s, S[i]), i
        assert torch.equal(u, U[i]), i
        assert torch.equal(v, V[i]), i
    # the replayed graph gives the same bits again
    U2, S2, V2 = batch.run()
    for i in range(len(ops)):
        assert torch.equal(S2[i], S[i]) and torch.equal(U2[i], U[i]) and torch.equal(V2[i], V[i])


def test_batched_matches_oracle(problems):
    graphs, ops, ranks = problems
    batch = isvd.Batch(ops, ranks, oversample=10, iters=4, seed=SEED)
    U, S, V = batch.run()
    for i in (1, 2):
        oop = oracle.graph_operator(graphs[i], coeffs=C5, ones_coeff=-LAM)
        Uo, So, Vo, _ = oop.isvd(ranks[i], 10, 4, SEED + i)
        s = S[i].double().cpu().numpy()
        assert np.abs(s - So).max() <= 1e-5 * So[0]


def test_batched_rejects_repeated_operator(problems):
    _, ops, ranks = problems
    batch = isvd.Batch([ops[0], ops[0]], [8, 8])
    with pytest.raises(isvd.IsvdError) as e:
        batch.run()
    assert e.value.name == "INVALID_ARGUMENT"


def test_batched_rejects_oversized_block(problems):
    _, ops, ranks = problems
    batch = isvd.Batch([ops[0], ops[6]], [8, 515])
    with pytest.raises(isvd.IsvdError) as e:
        batch.run()
    assert e.value.name in ("SHAPE", "UNSUPPORTED")
