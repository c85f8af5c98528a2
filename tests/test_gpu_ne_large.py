"""Parity at the 10^6-node network-embedding workload (Chung-Lu, 20,000,205
directed edges; NE operator sum_k c_k T^k - 0.05 11^T; rank 128, oversample
16, 6 power iterations: the configuration the benchmark times).

- On a 20,000-node induced subgraph of the same graph (breadth-first ball),
  the FP32 GPU SVD matches the FP64 oracle's Alg. 1 with the same seed:
  singular values within relative 1e-5, principal angles below 1e-3 rad on
  the gapped prefix, residuals no worse than the oracle's.
- At full size, against the oracle's own Alg. 1 on the whole graph (same
  seed; about two hours of CPU, stored by tests/golden/make_ne_large_golden.py
  in tests/golden/ne_large_k128_p16_q6.txt): the 128 singular values, and the
  residuals ||M v_i - s_i u_i||, ||M^T u_i - s_i v_i|| of the GPU's triplets
  (FP64 oracle products) against the oracle's.
- At full size, properties of Alg. 1's Rayleigh-Ritz step that hold at any
  size, checked with FP64 oracle products: M^T U = V diag(S) (V is M^T Q
  times the small singular vectors), U^T M V = diag(S), U and V orthonormal,
  S descending."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2111_06312_gb300 import build, isvd, synth
from svd_checks import check_svd

pytestmark = pytest.mark.gpu
LAM = 0.05
C5 = oracle.ne_coefficients(5)
K, P, Q = 128, 16, 6
SEED = synth.BASE_SEED + 2


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    build.build()
    oracle.build()


@pytest.fixture(scope="module")
def big():
    return synth.cached("ne_large")


def test_subgraph_20k_matches_oracle(big):
    g = synth.induced_subgraph(big, synth.bfs_ball(big, 20000))
    with isvd.graph_operator(g, coeffs=C5, ones_coeff=-LAM) as gpu:
        ref = oracle.graph_operator(g, coeffs=C5, ones_coeff=-LAM)
        out = check_svd(gpu, ref, K, P, Q, SEED)
    print(out)


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "ne_large_k128_p16_q6.txt")
GOLDEN_SEED = 20211106312


def _golden():
    rows = [ln.split() for ln in open(GOLDEN) if ln.strip() and not ln.startswith("#")]
    a = np.array([[float(x) for x in r[1:]] for r in rows])
    return a[:, 0], a[:, 1], a[:, 2]


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_full_size_matches_oracle_golden(big, precision):
    """sigma within relative 1e-5 (FP32; the mixed path within its stated
    error), and each triplet's residuals no larger than the oracle's plus what
    the triplet's own rounding adds: |s_i - s_ref_i| (the residual of a
    triplet is at least its value's distance to a singular value) and
    s_1 |dv| <= s_1 1e-5 (an FP32 vector carries a component of size up to its
    orthonormality error, 1e-5 here, along the top singular vector, and the
    all-ones term makes s_1 = 5e4 times the rest)."""
    S_ref, r1_ref, r2_ref = _golden()
    with isvd.graph_operator(big, coeffs=C5, ones_coeff=-LAM) as gpu:
        U, S, V, info = gpu.svd(K, P, Q, GOLDEN_SEED, precision=precision)
        assert isvd.info_dict(info)["status"] == "OK"
        Un, Sn, Vn = U.double().cpu().numpy(), S.double().cpu().numpy(), V.double().cpu().numpy()
    ref = oracle.graph_operator(big, coeffs=C5, ones_coeff=-LAM)
    r1 = np.linalg.norm(ref.apply(Vn) - Un * Sn[None, :], axis=0)
    r2 = np.linalg.norm(ref.apply(Un, transpose=True) - Vn * Sn[None, :], axis=0)
    rel = np.abs(Sn - S_ref) / S_ref
    slack = np.abs(Sn - S_ref) + 1e-5 * S_ref[0]
    out = dict(precision=precision, max_rel_sigma=rel.max(), argmax=int(rel.argmax()),
               worst_r1_excess=float((r1 - r1_ref).max()), worst_r2_excess=float((r2 - r2_ref).max()),
               max_r1=float(r1.max()), max_r1_ref=float(r1_ref.max()), min_slack=float(slack.min()))
    print(out)
    for i in np.argsort(r1 - r1_ref)[::-1][:4]:
        print(f"  i {i} s {Sn[i]:.9g} ref {S_ref[i]:.9g} gap- {S_ref[i-1]-S_ref[i] if i else 0:.3g} "
              f"gap+ {S_ref[i]-S_ref[i+1] if i < K-1 else 0:.3g} r1 {r1[i]:.4g} r1_ref {r1_ref[i]:.4g} "
              f"r2 {r2[i]:.4g} r2_ref {r2_ref[i]:.4g}")
    tol_s = 1e-5 if precision == "fp32" else MIXED_FULL_SIZE_TOL_S
    assert rel.max() <= tol_s, out
    assert np.all(r1 <= r1_ref + slack) and np.all(r2 <= r2_ref + slack), out


# stated error of the mixed path at full size against the oracle's sigma (same
# seed and iterations): measured on a GB300 2.7e-3 (the FP32 path: 4.0e-6),
# asserted at about twice that
MIXED_FULL_SIZE_TOL_S = 6e-3


@pytest.mark.parametrize("precision,tol", [("fp32", 2e-5), ("mixed", 2e-5)])
def test_full_size_rayleigh_ritz_properties(big, precision, tol):
    with isvd.graph_operator(big, coeffs=C5, ones_coeff=-LAM) as gpu:
        U, S, V, info = gpu.svd(K, P, Q, SEED, precision=precision)
        assert isvd.info_dict(info)["status"] == "OK"
        Ud, Vd = U.double(), V.double()
        eye = torch.eye(K, dtype=torch.float64, device=U.device)
        orth_u = float((Ud.T @ Ud - eye).abs().max())
        orth_v = float((Vd.T @ Vd - eye).abs().max())
        Un, Sn, Vn = Ud.cpu().numpy(), S.double().cpu().numpy(), Vd.cpu().numpy()
    ref = oracle.graph_operator(big, coeffs=C5, ones_coeff=-LAM)
    MtU = ref.apply(Un, transpose=True)
    MV = ref.apply(Vn)
    s1 = Sn[0]
    err_t = np.abs(MtU - Vn * Sn[None, :]).max()          # M^T U = V diag(S)
    err_p = np.abs(Un.T @ MV - np.diag(Sn)).max()          # U^T M V = diag(S)
    out = dict(precision=precision, orth_u=orth_u, orth_v=orth_v, err_t=err_t / s1, err_p=err_p / s1,
               s1=s1, sk=Sn[-1])
    print(out)
    assert np.all(np.diff(Sn) <= 0), out
    assert orth_u <= 1e-5 and orth_v <= 1e-5, out
    assert err_t <= tol * s1 and err_p <= tol * s1, out
