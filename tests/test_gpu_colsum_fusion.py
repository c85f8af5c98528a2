"""The all-ones projection 1^T Q of Eq. 3's alpha 1 1^T term, formed in the
epilogue of the Q R^-1 pass that writes Q (CholeskyQR, Alg. 2) instead of a
separate pass over Q before each product: through the C ABI, one rank-k SVD
launches the standalone projection only for the Gaussian start block and
reduces the orthonormalisation's column sums before every other product; the
SVD still matches the FP64 oracle (test_gpu_parity covers the same operators
at more sizes)."""
import pytest
import torch

import oracle
from paper_2111_06312_gb300 import build, isvd, synth
from svd_checks import check_svd

pytestmark = pytest.mark.gpu
LAM = 0.05
C5 = oracle.ne_coefficients(5)


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    build.build()
    oracle.build()


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_ones_projection_comes_from_the_orthonormalisation(precision):
    from torch.profiler import ProfilerActivity, profile

    g = synth.workload_ne_small()
    k, p, q, seed = 24, 8, 3, 11
    with isvd.graph_operator(g, coeffs=C5, ones_coeff=-LAM) as op:
        op.svd(k, p, q, seed, precision=precision)  # captures the graph
        torch.cuda.synchronize()
        with profile(activities=[ProfilerActivity.CUDA]):  # the first trace of a process can come back empty
            op.svd(k, p, q, seed, precision=precision)
            torch.cuda.synchronize()
        with profile(activities=[ProfilerActivity.CUDA]) as prof:
            op.svd(k, p, q, seed, precision=precision)
            torch.cuda.synchronize()
        counts = {}
        for e in prof.key_averages():
            counts[e.key] = counts.get(e.key, 0) + e.count
        proj = sum(v for key, v in counts.items() if "project_partial_kernel" in key)
        red = sum(v for key, v in counts.items() if "colsum_reduce_kernel" in key)
        assert proj == 1, counts  # the start block's product only
        assert red == 2 * q + 1, counts
        if precision == "fp32":
            ref = oracle.graph_operator(g, coeffs=C5, ones_coeff=-LAM)
            check_svd(op, ref, k, p, q, seed)


def test_operators_without_the_ones_term_are_unchanged():
    from torch.profiler import ProfilerActivity, profile

    g = synth.workload_ne_small()
    with isvd.graph_operator(g, coeffs=C5) as op:
        op.svd(8, 4, 2, 3)
        torch.cuda.synchronize()
        with profile(activities=[ProfilerActivity.CUDA]):
            op.svd(8, 4, 2, 3)
            torch.cuda.synchronize()
        with profile(activities=[ProfilerActivity.CUDA]) as prof:
            op.svd(8, 4, 2, 3)
            torch.cuda.synchronize()
        names = [e.key for e in prof.key_averages()]
        assert any("spmm" in n for n in names), names  # the trace saw the SVD
        assert not any("colsum_reduce_kernel" in n or "project_partial_kernel" in n for n in names), names
