"""Many independent problems in one call (isvd_svd_batched): every problem's
result must equal, bit for bit, that of its own isvd_svd call with the same
arguments (the kernels and their launch shapes are the same; only the
scheduling differs), and match the FP64 oracle like a single call does."""
import numpy as np
import pytest
import torch

import oracle
from paper_2111_06312_gb300 import build, isvd, synth
from svd_checks import assert_svd, measure_svd, npy

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


# stated error of the mixed-precision path against the FP64 oracle on these
# problems (BF16 blocks in the power iterations, FP32 refinement and
# Rayleigh-Ritz): measured on a GB300 at most 2.8e-4 (sigma, relative) and
# 9.9e-2 rad (principal angle on the gapped prefix), asserted at about twice that
MIXED_TOL_S, MIXED_TOL_ANGLE, MIXED_TOL_ORTH = 6e-4, 2e-1, 1e-5


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_batched_matches_oracle(problems, precision):
    """Every problem of the batch against the oracle's Alg. 1 with its own
    seed: FP32 within the single-call tolerances (sigma within relative 1e-5
    per value, principal angles below 1e-3 rad on the gapped prefix,
    orthonormality 1e-5, residuals no worse than the oracle's); the mixed path
    within its stated error."""
    graphs, ops, ranks = problems
    batch = isvd.Batch(ops, ranks, oversample=10, iters=4, seed=SEED, precision=precision)
    U, S, V = batch.run()
    for i, g in enumerate(graphs):
        oop = oracle.graph_operator(g, coeffs=C5, ones_coeff=-LAM)
        out = measure_svd(npy(U[i]), npy(S[i]), npy(V[i]), oop, ranks[i], 10, 4, SEED + i)
        print(i, precision, out)
        if precision == "fp32":
            assert_svd(out)
        else:
            assert_svd(out, MIXED_TOL_S, MIXED_TOL_ANGLE, MIXED_TOL_ORTH)


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
