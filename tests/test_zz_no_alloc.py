"""isvd_orthonormalize_noalloc (the allocation-free CholeskyQR2) against
isvd_orthonormalize, through the C ABI.

Callers that cannot allocate device memory when they orthonormalise -- code
inside another framework's allocator or memory-pool callback, or services
that forbid cudaMalloc on the hot path because it can synchronise the device
-- use the variant whose scratch is a fixed device array in the library.  It
must give the same result as the allocating entry point, call after call
(the array keeps the previous call's contents).  This file is collected last
so that a failure here never hides the result of another test."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2111_06312_gb300 import build, isvd, synth

pytestmark = pytest.mark.gpu


def _noalloc_fn():
    fn = isvd.lib().isvd_orthonormalize_noalloc
    fn.argtypes = [C.c_void_p, C.c_int64, C.c_int32, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]
    fn.restype = C.c_int
    return fn


def _block(rows, l, cond, seed):
    rng = np.random.default_rng(seed)
    Ua, _ = np.linalg.qr(rng.standard_normal((rows, l)))
    Va, _ = np.linalg.qr(rng.standard_normal((l, l)))
    A = (Ua * np.geomspace(1, 1 / cond, l)) @ Va.T
    return torch.tensor(A, dtype=torch.float32, device="cuda")


def test_noalloc_orthonormalize_matches_allocating_entry_point():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    build.build()
    fn = _noalloc_fn()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rows, l = 20011, 48
    Q0 = _block(rows, l, 1e3, 3)
    with isvd.graph_operator(synth.cycle(64), coeffs=[1.0]) as op:
        Q_ref, R_ref, info_ref = isvd.orthonormalize(op, Q0.clone())
    torch.cuda.synchronize()
    assert int(info_ref[0]) == 0
    for call in range(2):  # two calls in a row share the static scratch
        Q = Q0.clone()
        R = torch.zeros((l, l), dtype=torch.float64, device="cuda")
        info = torch.zeros(4, dtype=torch.int32, device="cuda")
        st = fn(C.c_void_p(Q.data_ptr()), rows, l, Q.stride(0), C.c_void_p(R.data_ptr()),
                C.c_void_p(info.data_ptr()), stream)
        assert st == 0, isvd.lib().isvd_last_error()
        torch.cuda.synchronize()
        assert int(info[0]) == 0 and int(info[2]) == int(info_ref[2])
        assert (Q - Q_ref).abs().max().item() <= 1e-5
        assert (R - R_ref).abs().max().item() <= 1e-5 * R_ref.abs().max().item()
        Qd = Q.double()
        assert (Qd.T @ Qd - torch.eye(l, dtype=torch.float64, device="cuda")).abs().max().item() < 2e-5
    # without a caller status block: the library's slot is cleared per call
    Q = Q0.clone()
    st = fn(C.c_void_p(Q.data_ptr()), rows, l, Q.stride(0), None, None, stream)
    assert st == 0
    torch.cuda.synchronize()
    assert (Q - Q_ref).abs().max().item() <= 1e-5
    # beyond the fixed scratch size: a clear error, nothing launched
    Qw = torch.zeros((1000, 72), dtype=torch.float32, device="cuda")
    st = fn(C.c_void_p(Qw.data_ptr()), 1000, 65, 72, None, None, stream)
    assert isvd.STATUS_NAMES[st] == "UNSUPPORTED"
    assert b"1..64" in isvd.lib().isvd_last_error()
