"""isvd_orthonormalize_noalloc (the allocation-free CholeskyQR2) against
isvd_orthonormalize, through the C ABI.

Callers that cannot allocate device memory when they orthonormalise -- code
inside another framework's allocator or memory-pool callback, or services
that forbid cudaMalloc on the hot path because it can synchronise the device
-- use the variant whose scratch is a fixed device array in the library.  It
must give the same result as the allocating entry point, call after call
(the array keeps the previous call's contents), at every block width up to
the array's limit, on contiguous and strided blocks, and once the device is
set up its calls must leave the device's free memory unchanged.  This file is
collected last so that a failure here never hides the result of another
test."""
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


def _block(rows, l, ldq, cond, seed):
    """A rows x l FP32 block of condition number `cond`, as the first l
    columns of a rows x ldq buffer (ldq - l padding columns of zeros)."""
    rng = np.random.default_rng(seed)
    Ua, _ = np.linalg.qr(rng.standard_normal((rows, l)))
    Va, _ = np.linalg.qr(rng.standard_normal((l, l)))
    A = (Ua * np.geomspace(1, 1 / cond, l)) @ Va.T
    buf = torch.zeros((rows, ldq), dtype=torch.float32, device="cuda")
    buf[:, :l] = torch.tensor(A, dtype=torch.float32, device="cuda")
    return buf


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    build.build()


# (rows, l, ldq): one column; the array's partial-count cap (20011 rows gives
# the largest Gram partial count); the widest block the array holds, dense
# and with a row stride above the width (the strided Gram path)
CASES = [(5003, 1, 8), (20011, 48, 48), (20011, 64, 64), (20011, 64, 72)]


@pytest.mark.parametrize("rows,l,ldq", CASES)
def test_noalloc_orthonormalize_matches_allocating_entry_point(rows, l, ldq):
    fn = _noalloc_fn()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    Q0 = _block(rows, l, ldq, 1e3, 3 + l)
    with isvd.graph_operator(synth.cycle(64), coeffs=[1.0]) as op:
        Q_ref, R_ref, info_ref = isvd.orthonormalize(op, Q0.clone()[:, :l])
    torch.cuda.synchronize()
    assert int(info_ref[0]) == 0
    # every buffer of the two calls exists before the first, so that the
    # device's free memory can be compared around the second
    Qs = [Q0.clone() for _ in range(2)]
    Rs = [torch.zeros((l, l), dtype=torch.float64, device="cuda") for _ in range(2)]
    infos = [torch.zeros(4, dtype=torch.int32, device="cuda") for _ in range(2)]
    torch.cuda.synchronize()
    free_before = None
    for call in range(2):  # two calls in a row share the static scratch
        if call == 1:
            free_before = torch.cuda.mem_get_info()[0]
        Q, R, info = Qs[call], Rs[call], infos[call]
        st = fn(C.c_void_p(Q.data_ptr()), rows, l, ldq, C.c_void_p(R.data_ptr()), C.c_void_p(info.data_ptr()),
                stream)
        assert st == 0, isvd.lib().isvd_last_error()
        torch.cuda.synchronize()
        if call == 1:
            # the first call set the device up (module load, symbol address);
            # the next allocates nothing
            assert torch.cuda.mem_get_info()[0] == free_before
        assert int(info[0]) == 0 and int(info[2]) == int(info_ref[2])
        Qv = Q[:, :l]
        assert (Qv - Q_ref).abs().max().item() <= 1e-5
        assert (R - R_ref).abs().max().item() <= 1e-5 * R_ref.abs().max().item()
        if ldq > l:
            assert Q[:, l:].abs().max().item() == 0.0  # padding columns untouched
        Qd = Qv.double()
        assert (Qd.T @ Qd - torch.eye(l, dtype=torch.float64, device="cuda")).abs().max().item() < 2e-5


def test_noalloc_orthonormalize_status_slot_and_limit():
    fn = _noalloc_fn()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rows, l = 20011, 48
    Q0 = _block(rows, l, l, 1e3, 3)
    with isvd.graph_operator(synth.cycle(64), coeffs=[1.0]) as op:
        Q_ref, _, _ = isvd.orthonormalize(op, Q0.clone())
    # without a caller status block: the library's slot is cleared per call
    for _ in range(2):
        Q = Q0.clone()
        st = fn(C.c_void_p(Q.data_ptr()), rows, l, l, None, None, stream)
        assert st == 0
        torch.cuda.synchronize()
        assert (Q - Q_ref).abs().max().item() <= 1e-5
    # beyond the fixed scratch size: a clear error, nothing launched
    Qw = torch.zeros((1000, 72), dtype=torch.float32, device="cuda")
    st = fn(C.c_void_p(Qw.data_ptr()), 1000, 65, 72, None, None, stream)
    assert isvd.STATUS_NAMES[st] == "UNSUPPORTED"
    assert b"1..64" in isvd.lib().isvd_last_error()
