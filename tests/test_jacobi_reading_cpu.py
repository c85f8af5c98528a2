"""The reading behind the GPU Jacobi's FP32 tangent (no GPU): a one-sided
Jacobi sweep whose Rutishauser tangent is rounded to FP32 (cos and sin formed
in FP64 from it, the orthogonality test on squares) converges to the same
singular values as one with the FP64 tangent, to FP64 rounding, in about the
same number of sweeps; LAPACK's values pin both.  Plain numpy, pair by pair."""
import numpy as np
import pytest


def one_sided_jacobi(A, fp32_tangent, max_sweeps=60):
    G = A.T.copy()  # columns of G = A^T
    l = G.shape[1]
    eps = np.finfo(np.float64).eps
    tol = max(1e-15, np.sqrt(l) * eps)
    for sweep in range(1, max_sweeps + 1):
        rotated = False
        for p in range(l - 1):
            for q in range(p + 1, l):
                gp, gq = G[:, p], G[:, q]
                ga = gp @ gq
                al, be = gp @ gp, gq @ gq
                if ga == 0.0 or ga * ga <= tol * tol * al * be:
                    continue
                if fp32_tangent:
                    # zeta in FP32 from num and den scaled by a power of two
                    # (den to [1, 2)); t ~ 1/(2 zeta) where zeta^2 would overflow
                    num, den = be - al, 2.0 * ga
                    sc = 2.0 ** -np.frexp(abs(den))[1] * 2.0
                    with np.errstate(over="ignore"):
                        z = np.float32(num * sc) / np.float32(den * sc)
                    if abs(z) < np.float32(1e18):
                        t = np.float64(np.copysign(np.float32(1), z) / (np.abs(z) + np.sqrt(np.float32(1) + z * z)))
                    else:
                        t = np.float64(np.float32(0.5) / z)
                else:
                    zeta = (be - al) / (2.0 * ga)
                    t = np.copysign(1.0, zeta) / (abs(zeta) + np.sqrt(1.0 + zeta * zeta))
                cs = 1.0 / np.sqrt(1.0 + t * t)
                sn = cs * t
                G[:, p], G[:, q] = cs * gp - sn * gq, sn * gp + cs * gq
                rotated = True
        if not rotated:
            return np.sort(np.linalg.norm(G, axis=0))[::-1], sweep
    return np.sort(np.linalg.norm(G, axis=0))[::-1], max_sweeps


@pytest.mark.parametrize("l,cond,seed", [(24, 1e3, 1), (40, 1e8, 2), (32, 10.0, 3)])
def test_fp32_tangent_reaches_the_same_singular_values(l, cond, seed):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((l, l)))
    V, _ = np.linalg.qr(rng.standard_normal((l, l)))
    A = np.linalg.qr((U * np.geomspace(1, 1 / cond, l)) @ V.T)[1]  # upper triangular, like R
    ref = np.linalg.svd(A, compute_uv=False)
    s64, n64 = one_sided_jacobi(A, False)
    s32, n32 = one_sided_jacobi(A, True)
    assert np.allclose(s64, ref, rtol=1e-11, atol=1e-14 * ref[0])
    assert np.allclose(s32, ref, rtol=1e-11, atol=1e-14 * ref[0])
    assert n32 <= n64 + 2, (n32, n64)
