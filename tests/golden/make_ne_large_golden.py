"""Write the oracle's rank-128 SVD of the 10^6-node network-embedding operator
to ``ne_large_k128_p16_q6.txt`` (test infrastructure: calls only ``oracle/``
and the seeded input generators).

Operator: M = sum_{k=1..5} c_k T^k - 0.05 11^T, c_k = (6-k)/15, T = D^-1 A
(Eq. 3 with the normalised window weights; Sec. 2 for T), on the seeded
Chung-Lu graph with n = 10^6 and 2x10^7 directed edges.  The oracle runs
Alg. 1 (App. A.2) in FP64 with k = 128, oversample 16 (block width 144),
6 power iterations and the start block of seed 20211106312, i.e. the same
Alg. 1 run as the GPU's ``isvd_svd`` with those arguments.  For each of the
128 Ritz triplets the file records sigma_i and the two residual norms
||M v_i - sigma_i u_i|| and ||M^T u_i - sigma_i v_i|| (FP64 oracle products),
the certificate that some singular value of M lies within the larger of the
two of sigma_i.

    python tests/golden/make_ne_large_golden.py      # ~1 h on 8 x86 cores
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "ne_large_k128_p16_q6.txt")
K, P, Q, SEED, LAM = 128, 16, 6, 20211106312, 0.05


def main():
    import oracle
    from paper_2111_06312_gb300 import synth

    oracle.build()
    g = synth.cached("ne_large")
    op = oracle.graph_operator(g, coeffs=oracle.ne_coefficients(5), ones_coeff=-LAM)
    t0 = time.perf_counter()
    U, S, V, passes = op.isvd(K, P, Q, SEED)
    t1 = time.perf_counter()
    MV = op.apply(V)
    MtU = op.apply(U, transpose=True)
    r_left = np.linalg.norm(MV - U * S[None, :], axis=0)
    r_right = np.linalg.norm(MtU - V * S[None, :], axis=0)
    t2 = time.perf_counter()
    with open(OUT + ".tmp", "w") as f:
        f.write("# Alg. 1 (App. A.2) in FP64 by the oracle: M = sum_{k=1..5} (6-k)/15 T^k - 0.05 11^T (Eq. 3),\n")
        f.write(f"# T = D^-1 A on synth.cached('ne_large') (n = {g.n}, nnz = {g.nnz}); k = {K}, oversample = {P},\n")
        f.write(f"# iterations = {Q}, seed = {SEED}; {passes} CholeskyQR passes.  Written by\n")
        f.write("# tests/golden/make_ne_large_golden.py.  Columns: i, sigma_i, ||M v_i - sigma_i u_i||,\n")
        f.write("# ||M^T u_i - sigma_i v_i||.\n")
        for i in range(K):
            f.write(f"{i} {S[i]:.17e} {r_left[i]:.17e} {r_right[i]:.17e}\n")
    os.replace(OUT + ".tmp", OUT)
    print(f"oracle Alg. 1: {t1 - t0:.1f} s on {oracle.num_threads()} threads; residuals {t2 - t1:.1f} s; "
          f"sigma_1 {S[0]:.6e}, sigma_128 {S[-1]:.6e}, max residual {max(r_left.max(), r_right.max()):.3e}")


if __name__ == "__main__":
    main()
