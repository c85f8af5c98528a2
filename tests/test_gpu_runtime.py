"""Runtime pieces around the method: the launch-shape autotuner (results stay
correct whatever shape it picks; its cache round-trips) and the bounded-wait
failure detection (a wait on a barrier that nothing arrives on reports
ISVD_ERR_TIMEOUT and leaves the context usable)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2111_06312_gb300 import build, isvd, synth

pytestmark = pytest.mark.gpu
C5 = oracle.ne_coefficients(5)


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    build.build()
    oracle.build()


@pytest.fixture(scope="module")
def graph():
    return synth.chung_lu(5000, 60000, 91, max_degree=2000)


def _check_apply(gop, oop, b, dtype=torch.float32, tol=1e-5):
    G = isvd.gaussian(5, gop.shape[1], b, dtype=dtype)
    Y = gop.apply(G).double().cpu().numpy()
    Yr = oop.apply(G.double().cpu().numpy())
    assert np.abs(Y - Yr).max() <= tol * np.abs(Yr).max()


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_autotune_keeps_results_and_caches(graph, dtype, tmp_path):
    cache = str(tmp_path / "tune.txt")
    gop = isvd.graph_operator(graph, coeffs=C5, ones_coeff=-0.05)
    oop = oracle.graph_operator(graph, coeffs=C5, ones_coeff=-0.05)
    try:
        t1 = gop.autotune(42, dtype=dtype, cache_path=cache)
        assert t1["kernel"] in ("rows", "ring", "slab")
        _check_apply(gop, oop, 42, dtype, 1e-5 if dtype == torch.float32 else 2e-2)
        lines = open(cache).read().strip().splitlines()
        assert len(lines) == 1 and "b=42" in lines[0]
        gop.set_tuning(kernel="chunks")
        t2 = gop.autotune(42, dtype=dtype, cache_path=cache)  # cache hit: same shape back
        assert t2 == t1
        assert len(open(cache).read().strip().splitlines()) == 1
    finally:
        gop.close()


def test_selftest_wait_reports_timeout_and_context_survives(graph):
    st = isvd.selftest_wait(2000)
    assert st["status"] == "TIMEOUT"
    gop = isvd.graph_operator(graph, coeffs=C5, ones_coeff=-0.05)
    oop = oracle.graph_operator(graph, coeffs=C5, ones_coeff=-0.05)
    try:
        _check_apply(gop, oop, 16)
    finally:
        gop.close()


def test_selftest_wait_rejects_bad_limits():
    info = torch.zeros(4, dtype=torch.int32, device="cuda")
    for bad in (0, -5, (1 << 24) + 1):
        with pytest.raises(isvd.IsvdError):
            isvd._check(isvd.lib().isvd_selftest_wait(bad, isvd._ptr(info), isvd._stream()), "isvd_selftest_wait")
