"""Shared comparison of a GPU SVD with the FP64 oracle's Alg. 1 (test helper)."""
import numpy as np

import oracle
from paper_2111_06312_gb300 import isvd


def npy(t):
    return t.double().cpu().numpy()


def gapped_prefix(S_ritz, k, rel_gap=1e-3):
    """Largest j <= k with (s_j - s_{j+1}) >= rel_gap * s_j (1-based)."""
    best = 0
    for j in range(1, k + 1):
        # j == len(S_ritz): the whole block is the subspace, no gap to check
        if j == len(S_ritz) or S_ritz[j - 1] - S_ritz[j] >= rel_gap * S_ritz[j - 1]:
            best = j
    return best


def oracle_reference(ref_op, k, p, q, seed):
    """The oracle's Alg. 1 (U, S, V) and all k + p Ritz values of the same block."""
    Ur, Sr, Vr, _ = ref_op.isvd(k, p, q, seed)
    _, S_all, _, _ = ref_op.isvd(k + p, 0, q, seed)
    return Ur, Sr, Vr, S_all


def measure_svd(Un, Sn, Vn, ref_op, k, p, q, seed, ref=None):
    """Errors of a computed rank-k SVD (numpy FP64 copies) against the oracle's
    Alg. 1 with the same k, oversample, iterations and seed: per-value
    relative sigma error, principal angles of U and V on the prefix the
    oracle's Ritz values separate by a relative gap >= 1e-3, orthonormality,
    and the residuals max(||M v - s u||, ||M^T u - s v||) of both (FP64
    oracle products)."""
    Ur, Sr, Vr, S_all = ref if ref is not None else oracle_reference(ref_op, k, p, q, seed)
    rel = np.abs(Sn - Sr) / Sr
    j = gapped_prefix(S_all, k)
    ang_u = oracle.max_principal_angle(Ur[:, :j], Un[:, :j]) if j else 0.0
    ang_v = oracle.max_principal_angle(Vr[:, :j], Vn[:, :j]) if j else 0.0
    orth_u = np.abs(Un.T @ Un - np.eye(k)).max()
    orth_v = np.abs(Vn.T @ Vn - np.eye(k)).max()
    res = oracle.residuals(ref_op, Un, Sn, Vn)
    res_ref = oracle.residuals(ref_op, Ur, Sr, Vr)
    return dict(rel=rel.max(), j=j, ang_u=ang_u, ang_v=ang_v, orth_u=orth_u, orth_v=orth_v,
                res=res.max(), res_ref=res_ref.max(), s1=Sr[0])


def assert_svd(out, tol_s=1e-5, tol_angle=1e-3, tol_orth=1e-5, res_slack=1e-4):
    assert out["rel"] <= tol_s, out
    assert out["ang_u"] <= tol_angle and out["ang_v"] <= tol_angle, out
    assert out["orth_u"] <= tol_orth and out["orth_v"] <= tol_orth, out
    # the rest is valid: residuals no worse than the oracle's own plus rounding
    assert out["res"] <= out["res_ref"] + res_slack * out["s1"], out


def check_svd(gpu_op, ref_op, k, p, q, seed, tol_s=1e-5, tol_angle=1e-3, precision="fp32"):
    U, S, V, info = gpu_op.svd(k, p, q, seed, precision=precision)
    out = measure_svd(npy(U), npy(S), npy(V), ref_op, k, p, q, seed)
    out["info"] = isvd.info_dict(info)
    assert out["info"]["status"] == "OK", out
    assert_svd(out, tol_s, tol_angle)
    return out


def cond_block(r, c, cond, seed):
    """r x c FP64 block with singular values geomspace(1, 1/cond) and random
    singular vectors (seeded)."""
    rng = np.random.default_rng(seed)
    Ua, _ = np.linalg.qr(rng.standard_normal((r, c)))
    Va, _ = np.linalg.qr(rng.standard_normal((c, c)))
    return (Ua * np.geomspace(1, 1 / cond, c)) @ Va.T
