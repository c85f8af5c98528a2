"""The C-ABI library builds, loads without a GPU and exports every entry point
that include/isvd.h declares; host-side argument checks that need no device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "isvd.h")).read()
    return re.findall(r"ISVD_API\s+[\w\s\*]+?\b(isvd_\w+)\s*\(", src)


@pytest.fixture(scope="module")
def libisvd():
    from paper_2111_06312_gb300 import build

    path = build.build()
    return C.CDLL(path)


def test_header_declares_the_boundary():
    names = set(declared_functions())
    for want in ("isvd_create_operator", "isvd_apply", "isvd_apply_T", "isvd_svd", "isvd_destroy_operator"):
        assert want in names


def test_library_exports_every_declared_symbol(libisvd):
    names = declared_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(libisvd, name), f"{name} declared in isvd.h but not exported"


def test_status_strings_and_null_checks(libisvd):
    libisvd.isvd_status_string.restype = C.c_char_p
    libisvd.isvd_last_error.restype = C.c_char_p
    assert libisvd.isvd_status_string(0) == b"ok"
    assert libisvd.isvd_status_string(4).startswith(b"Gram")
    # null descriptor: rejected on the host before any CUDA call
    libisvd.isvd_create_operator.argtypes = [C.c_void_p] * 4
    out = C.c_void_p()
    assert libisvd.isvd_create_operator(None, None, None, C.byref(out)) == 1
    assert b"null" in libisvd.isvd_last_error()
    libisvd.isvd_svd.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_uint64, C.c_int, C.c_void_p,
                                 C.c_int64, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]
    assert libisvd.isvd_svd(None, 4, 2, 1, 0, 0, None, 4, None, None, 4, None, None) == 1
    libisvd.isvd_destroy_operator.argtypes = [C.c_void_p]
    libisvd.isvd_destroy_operator(None)  # NULL is a no-op


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_2111_06312_gb300 import build, isvd

    monkeypatch.setattr(build, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(isvd, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        isvd.lib()


def test_orthonormalize_noalloc_rejects_bad_layouts_on_the_host(libisvd):
    # the row pitch and base alignment that the kernels' 16-byte copies need are
    # checked before the device is touched (no GPU here)
    libisvd.isvd_last_error.restype = C.c_char_p
    fn = libisvd.isvd_orthonormalize_noalloc
    fn.argtypes = [C.c_void_p, C.c_int64, C.c_int32, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]
    fn.restype = C.c_int
    fake = C.c_void_p(1 << 20)  # never dereferenced: every call below fails its host checks
    assert fn(None, 100, 8, 8, None, None, None) == 1
    assert fn(fake, 100, 8, 12, None, None, None) == 1  # pitch not a multiple of 8
    assert b"multiple of 8" in libisvd.isvd_last_error()
    assert fn(C.c_void_p((1 << 20) + 4), 100, 8, 8, None, None, None) == 1  # base not 16-byte aligned
    assert fn(fake, 100, 8, 4, None, None, None) == 1  # pitch below the width
    assert fn(fake, 4, 8, 8, None, None, None) == 3  # fewer rows than columns: ISVD_ERR_SHAPE


def test_embed_and_pair_scores_reject_bad_arguments_on_the_host(libisvd):
    # argument checks of the Sec. 3.1 outputs run before any launch (no GPU here)
    P, I32, I64 = C.c_void_p, C.c_int32, C.c_int64
    emb = libisvd.isvd_embed
    emb.argtypes = [P, I64, I64, I32, P, P, I64, P]
    emb.restype = C.c_int
    ps = libisvd.isvd_pair_scores
    ps.argtypes = [P, I64, I64, P, I64, I64, I32, P, P, I64, P, P, P]
    ps.restype = C.c_int
    fake = C.c_void_p(1 << 20)  # never dereferenced
    assert emb(None, 8, 10, 8, fake, fake, 8, None) == 1
    assert emb(fake, 8, 10, 0, fake, fake, 8, None) == 3  # k < 1: ISVD_ERR_SHAPE
    assert emb(fake, 4, 10, 8, fake, fake, 8, None) == 1  # ld below k
    assert emb(fake, 8, -1, 8, fake, fake, 8, None) == 1
    assert ps(fake, 8, 10, fake, 8, 10, 8, fake, fake, -1, fake, None, None) == 1
    assert ps(None, 8, 10, None, 8, 10, 8, None, None, 0, None, None, None) == 0  # no pairs: nothing to do
    assert ps(fake, 8, 10, None, 8, 10, 8, fake, fake, 5, fake, None, None) == 1
    assert ps(fake, 8, 10, fake, 8, 10, 0, fake, fake, 5, fake, None, None) == 3
    assert ps(fake, 8, 10, fake, 4, 10, 8, fake, fake, 5, fake, None, None) == 1


def test_compose_rejects_bad_arguments_on_the_host(libisvd):
    # kind, count and weight checks come before any child is read (no GPU here)
    P, I32 = C.c_void_p, C.c_int32
    fn = libisvd.isvd_compose_operators
    fn.argtypes = [C.c_int, P, I32, P, P, P, P]
    fn.restype = C.c_int
    out = C.c_void_p()
    one = (C.c_void_p * 1)(None)
    assert fn(0, None, 1, None, None, None, C.byref(out)) == 1
    assert fn(7, one, 1, None, None, None, C.byref(out)) == 1  # unknown kind
    assert fn(0, one, 0, None, None, None, C.byref(out)) == 1  # count < 1
    assert fn(0, one, 17, None, None, None, C.byref(out)) == 1  # count > ISVD_MAX_CHILDREN
    w = (C.c_double * 1)(1.0)
    assert fn(1, one, 1, C.cast(w, P), None, None, C.byref(out)) == 1  # weights on a non-SUM node
    assert fn(0, one, 1, None, None, None, C.byref(out)) == 1  # null child
    assert out.value is None


def test_edge_kernel_rejects_bad_arguments_on_the_host(libisvd):
    P, I32, I64, D = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    wd = libisvd.isvd_edge_kernel_work_doubles
    wd.argtypes = [I32]
    wd.restype = C.c_int64
    assert wd(0) == 0 and wd(128) > 3 * 128
    fn = libisvd.isvd_edge_kernel_loss
    fn.argtypes = [P, I64, I64, P, I64, I64, I32, P, D, D, P, P, I64, P, P, I64, D, P, P, I64, P, P]
    fn.restype = C.c_int
    f = C.c_void_p(1 << 20)  # never dereferenced
    n = wd(8)
    assert fn(f, 8, 10, f, 8, 10, 8, f, 1.0, 5.0, f, f, 4, f, f, 4, 10.0, f, f, n - 1, None, None) == 1  # small work
    assert fn(f, 8, 10, f, 8, 10, 8, f, 1.0, float("nan"), f, f, 4, f, f, 4, 10.0, f, f, n, None, None) == 1
    assert fn(f, 8, 10, f, 8, 10, 8, f, 1.0, 5.0, f, f, 0, f, f, 4, 10.0, f, f, n, None, None) == 1  # no edges
    assert fn(f, 8, 10, f, 8, 10, 0, f, 1.0, 5.0, f, f, 4, f, f, 4, 10.0, f, f, n, None, None) == 3  # k < 1
    assert fn(f, 8, 10, f, 8, 10, 8, f, 1.0, 5.0, f, f, 4, f, f, 4, -1.0, f, f, n, None, None) == 1  # k_neg < 0


def test_binding_declares_every_entry_point():
    # the ctypes binding gives every function of isvd.h its argument types, and
    # every isvd_status function an int result (loaded without a GPU)
    from paper_2111_06312_gb300 import isvd

    L = isvd.lib()
    src = open(os.path.join(ROOT, "include", "isvd.h")).read()
    for name in declared_functions():
        assert getattr(L, name).argtypes is not None, f"{name} has no argtypes in isvd.lib()"
    for name in re.findall(r"ISVD_API\s+isvd_status\s+(isvd_\w+)\s*\(", src):
        assert getattr(L, name).restype is C.c_int, f"{name} should return int"
    assert L.isvd_get_tuning(None, None) == 1  # null operator: rejected on the host


def _header():
    return open(os.path.join(ROOT, "include", "isvd.h")).read()


def test_binding_constants_match_the_header():
    from paper_2111_06312_gb300 import isvd

    src = _header()
    defines = dict(re.findall(r"#define\s+(ISVD_\w+)\s+(\d+)", src))
    assert int(defines["ISVD_MAX_BLOCK"]) == isvd.MAX_BLOCK
    assert int(defines["ISVD_MAX_BLOCK_WIDE"]) == isvd.MAX_BLOCK_WIDE
    assert int(defines["ISVD_PERSISTENT_MAX_BLOCK"]) <= isvd.MAX_BLOCK


def test_persistent_options_layout_matches_the_header():
    """The ctypes mirror of isvd_persistent_options has the header's fields in
    the header's order (a reordering would pass garbage without an error)."""
    from paper_2111_06312_gb300 import isvd

    src = _header()
    end = src.index("} isvd_persistent_options;")
    body = src[src.rindex("typedef struct {", 0, end):end]
    fields = re.findall(r"int32_t\s+(\w+);", body)
    assert fields == [f[0] for f in isvd._PersistentOptions._fields_]


def test_persistent_batch_rejects_bad_arguments_on_the_host(libisvd):
    libisvd.isvd_svd_batched_persistent.restype = C.c_int
    libisvd.isvd_svd_batched_persistent.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_int32,
                                                    C.c_uint64] + [C.c_void_p] * 6
    assert libisvd.isvd_svd_batched_persistent(None, None, 1, 4, 1, 0, None, None, None, None, None, None) == 1
    k = (C.c_int32 * 1)(4)
    ops = (C.c_void_p * 1)(None)
    assert libisvd.isvd_svd_batched_persistent(ops, k, 0, 4, 1, 0, ops, ops, ops, None, None, None) == 1
