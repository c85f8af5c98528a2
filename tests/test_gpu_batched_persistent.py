"""The batch in one persistent kernel (isvd_svd_batched_persistent), through
the C ABI: every problem against the FP64 oracle's Alg. 1 with its own seed
(the single-call tolerances), against the graph form of the batch, the same
bits on a second run and across team sizes up to rounding; and the failure
path without a fault: teams that wait for a member that does not exist give
up within their spin budget, report ISVD_ERR_TIMEOUT per problem, and the
next call works."""
import numpy as np
import pytest
import torch

import oracle
from paper_2111_06312_gb300 import build, isvd, synth
from svd_checks import assert_svd, measure_svd, npy

pytestmark = pytest.mark.gpu
LAM = 0.05
C5 = oracle.ne_coefficients(5)
SEED = 20211106316


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    build.build()
    oracle.build()


# sizes span one-member teams and teams of 2 and 3 (one member per 16,384
# rows by default); norms: T = D^-1 A and A-hat (with and without its
# identity term)
SIZES = [700, 1500, 3100, 900, 2500, 4000, 520, 20000, 33000]
RANKS = [16, 32, 64, 16, 32, 8, 16, 32, 64]
NORMS = ["row", "row", "sym", "row", "sym_noself", "row", "row", "sym", "row"]


@pytest.fixture(scope="module")
def problems():
    graphs = []
    for i, n in enumerate(SIZES):
        if i % 2 == 0:
            graphs.append(synth.erdos_renyi(n, 8.0, 1900 + i))
        else:
            graphs.append(synth.chung_lu(n, 8 * n, 1900 + i))
    ops = [isvd.graph_operator(g, coeffs=C5, ones_coeff=-LAM, norm=nm) for g, nm in zip(graphs, NORMS)]
    yield graphs, ops
    for op in ops:
        op.close()


def _run(ops, **kw):
    b = isvd.Batch(ops, RANKS, oversample=10, iters=4, seed=SEED, persistent=True, **kw)
    U, S, V = b.run()
    return [u.clone() for u in U], [s.clone() for s in S], [v.clone() for v in V], b.info.clone()


def test_persistent_matches_oracle(problems):
    graphs, ops = problems
    U, S, V, info = _run(ops)
    assert int(info[:, 0].abs().sum()) == 0
    for i, g in enumerate(graphs):
        oop = oracle.graph_operator(g, coeffs=C5, ones_coeff=-LAM, norm=NORMS[i])
        out = measure_svd(npy(U[i]), npy(S[i]), npy(V[i]), oop, RANKS[i], 10, 4, SEED + i)
        print(i, SIZES[i], NORMS[i], out)
        assert_svd(out)


def test_persistent_agrees_with_graph_batch_and_itself(problems):
    _, ops = problems
    U, S, V, _ = _run(ops)
    U2, S2, V2, _ = _run(ops)
    for i in range(len(ops)):  # deterministic: fixed-order sums within a team
        assert torch.equal(S[i], S2[i]) and torch.equal(U[i], U2[i]) and torch.equal(V[i], V2[i]), i
    g = isvd.Batch(ops, RANKS, oversample=10, iters=4, seed=SEED)
    Ug, Sg, Vg = g.run()
    for i in range(len(ops)):
        rel = ((S[i].double() - Sg[i].double()).abs() / Sg[i].double()).max().item()
        assert rel < 1e-5, (i, rel)


def test_persistent_team_size_changes_rounding_only(problems):
    _, ops = problems
    _, S1, _, _ = _run(ops, max_team=1)
    _, S3, _, info = _run(ops, max_team=3)
    _, S9, _, info9 = _run(ops, rows_per_member=4096)  # teams of up to 9
    assert int(info[:, 0].abs().sum()) == 0 and int(info9[:, 0].abs().sum()) == 0
    for i in range(len(ops)):
        rel = ((S9[i].double() - S3[i].double()).abs() / S3[i].double()).max().item()
        assert rel < 1e-5, (i, rel)
        rel = ((S1[i].double() - S3[i].double()).abs() / S3[i].double()).max().item()
        assert rel < 1e-5, (i, rel)


def test_persistent_wait_runs_out_without_a_fault(problems):
    """Every team waits for one member more than it has: each problem's first
    meeting gives up after the spin budget and reports TIMEOUT; the kernel
    ends, and the next call on the same operators is correct."""
    _, ops = problems
    small = ops[:4]
    b = isvd.Batch(small, RANKS[:4], oversample=10, iters=4, seed=SEED, persistent=True, spin_limit=2000,
                   test_phantom=True)
    b.run(check=False)
    torch.cuda.synchronize()
    st = b.info[:, 0].cpu().tolist()
    assert all(isvd.STATUS_NAMES[x] == "TIMEOUT" for x in st), st
    ok = isvd.Batch(small, RANKS[:4], oversample=10, iters=4, seed=SEED, persistent=True)
    U, S, V = ok.run()
    assert int(ok.info[:, 0].abs().sum()) == 0
    for i in range(4):
        u, s, v, info = small[i].svd(RANKS[i], 10, 4, seed=SEED + i)
        rel = ((S[i].double() - s.double()).abs() / s.double()).max().item()
        assert rel < 1e-5, (i, rel)


def test_persistent_refuses_what_it_does_not_take(problems):
    graphs, ops = problems
    with pytest.raises(isvd.IsvdError) as e:  # block wider than the persistent form takes
        isvd.Batch([ops[8]], [90], oversample=10, iters=1, persistent=True).run()
    assert e.value.name == "UNSUPPORTED"
    g = graphs[0]
    w = np.full(g.nnz, 1.5, dtype=np.float32)  # a weighted graph (constant weights: symmetric)
    with isvd.Operator(g.n, g.rowptr, g.colidx, values=w, coeffs=C5) as wop:
        with pytest.raises(isvd.IsvdError) as e:
            isvd.Batch([wop], [8], oversample=4, iters=1, persistent=True).run()
        assert e.value.name == "UNSUPPORTED"
    with pytest.raises(ValueError):
        isvd.Batch([ops[0]], [8], precision="mixed", persistent=True).run()
