"""Python binding of libisvd.so (C ABI in ``include/isvd.h``).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of the library.  PyTorch provides device memory (tensors and the
library's workspace, through the caching allocator) and the current stream.
If the library has not been built, every entry point raises -- there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np
import torch

from . import build as _build

ISVD_OK = 0
STATUS_NAMES = {
    0: "OK", 1: "INVALID_ARGUMENT", 2: "INVALID_GRAPH", 3: "SHAPE", 4: "NOT_POSITIVE_DEFINITE",
    5: "TIMEOUT", 6: "WORKSPACE", 7: "CUDA", 8: "UNSUPPORTED",
}
F32, BF16 = 0, 1
PREC = {"fp32": 0, "mixed": 1}
NORM = {"row": 0, "sym": 1, "sym_noself": 2}
FORM = {"poly": 0, "concat": 1}
FLAG_SKIP_SYMMETRY_CHECK = 1
MAX_BLOCK = 160
MAX_BLOCK_WIDE = 512  # FP32 block widths of svd and orthonormalize


class IsvdError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        self.status = status
        self.name = STATUS_NAMES.get(status, str(status))
        super().__init__(f"{where}: {self.name}: {detail}")


class _Csr(C.Structure):
    _fields_ = [("rows", C.c_int64), ("cols", C.c_int64), ("nnz", C.c_int64),
                ("rowptr", C.c_void_p), ("colidx", C.c_void_p), ("values", C.c_void_p)]


class _Desc(C.Structure):
    _fields_ = [("form", C.c_int), ("norm", C.c_int), ("A", _Csr),
                ("degree", C.c_int32), ("coeffs", C.c_void_p), ("ones_coeff", C.c_double),
                ("adj_coeff", C.c_double), ("lr_rank", C.c_int32), ("lr_u", C.c_void_p),
                ("lr_v", C.c_void_p), ("lr_alpha", C.c_void_p), ("d", C.c_int64), ("L", C.c_int32),
                ("X", _Csr), ("X_dense", C.c_void_p), ("flags", C.c_int32),
                ("gather_rows", C.c_void_p), ("n_gather", C.c_int64)]


_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class _Allocator(C.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("ctx", C.c_void_p)]


def _torch_alloc(nbytes, stream, ctx):
    try:
        return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
    except Exception:  # the library reports ISVD_ERR_WORKSPACE
        return None


def _torch_free(ptr, stream, ctx):
    try:
        torch.cuda.caching_allocator_delete(int(ptr))
    except Exception:
        pass


_alloc_cb = _ALLOC_FN(_torch_alloc)
_free_cb = _FREE_FN(_torch_free)
_TORCH_ALLOCATOR = _Allocator(_alloc_cb, _free_cb, None)

_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libisvd.so; raise if it is missing (no fallback path exists)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"libisvd.so is not built ({path}); run paper_2111_06312_gb300.build.build()")
            L = C.CDLL(path)
            P, I32, I64, U64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64
            L.isvd_create_operator.argtypes = [P, P, P, P]
            L.isvd_destroy_operator.argtypes = [P]
            L.isvd_destroy_operator.restype = None
            L.isvd_operator_shape.argtypes = [P, P, P]
            L.isvd_apply.argtypes = [P, P, I64, I32, P, I64, C.c_int, P]
            L.isvd_apply_T.argtypes = [P, P, I64, I32, P, I64, C.c_int, P]
            L.isvd_svd.argtypes = [P, I32, I32, I32, U64, C.c_int, P, I64, P, P, I64, P, P]
            L.isvd_gaussian.argtypes = [U64, I64, I32, P, I64, C.c_int, P]
            L.isvd_philox_words.argtypes = [U64, I64, P, P]
            L.isvd_orthonormalize.argtypes = [P, P, I64, I32, I64, P, P, P]
            L.isvd_small_svd.argtypes = [P, P, I32, P, P, P, P, P]
            L.isvd_closed_form.argtypes = [P, P, I64, P, P, I64, I32, P, I64, I32, C.c_double, P, I64, P]
            L.isvd_compose_operators.argtypes = [C.c_int, P, I32, P, P, P, P]
            L.isvd_embed.argtypes = [P, I64, I64, I32, P, P, I64, P]
            L.isvd_edge_kernel_work_doubles.argtypes = [I32]
            L.isvd_edge_kernel_work_doubles.restype = C.c_int64
            L.isvd_edge_kernel_weights.argtypes = [P, I32, C.c_double, C.c_double, P, P]
            L.isvd_edge_kernel_scores.argtypes = [P, I64, I64, P, I64, I64, I32, P, C.c_double, C.c_double, P, P,
                                                  I64, P, P, I64, P, P]
            L.isvd_edge_kernel_loss.argtypes = [P, I64, I64, P, I64, I64, I32, P, C.c_double, C.c_double, P, P,
                                                I64, P, P, I64, C.c_double, P, P, I64, P, P]
            L.isvd_pair_scores.argtypes = [P, I64, I64, P, I64, I64, I32, P, P, I64, P, P, P]
            L.isvd_get_tuning.argtypes = [P, P]
            L.isvd_set_tuning.argtypes = [P, P, P]
            L.isvd_orthonormalize_noalloc.argtypes = [P, I64, I32, I64, P, P, P]
            L.isvd_composite_cache.argtypes = [P, I32]
            L.isvd_split_relu_work_bytes.argtypes = [I64, I32, I32]
            L.isvd_split_relu_work_bytes.restype = C.c_size_t
            L.isvd_split_relu_forward.argtypes = [P, I64, I64, I32, P, P, I32, P, I64, P, P, I64, P]
            L.isvd_split_relu_backward.argtypes = [P, I64, I64, I32, P, P, I32, P, P, I64, P, I64, P, I64, P, P, P,
                                                   C.c_size_t, P]
            L.isvd_svd_batched.argtypes = [P, P, I32, I32, I32, U64, C.c_int, P, P, P, P, P]
            L.isvd_svd_batched_persistent.argtypes = [P, P, I32, I32, I32, U64, P, P, P, P, P, P]
            L.isvd_autotune.argtypes = [P, I32, C.c_int, C.c_char_p, P, P]
            L.isvd_selftest_wait.argtypes = [I32, P, P]
            L.isvd_batched_kernel_nodes.argtypes = []
            L.isvd_batched_kernel_nodes.restype = C.c_int64
            L.isvd_graph_kernel_nodes.argtypes = [P]
            L.isvd_graph_kernel_nodes.restype = C.c_int64
            L.isvd_status_string.argtypes = [C.c_int]
            L.isvd_status_string.restype = C.c_char_p
            L.isvd_last_error.argtypes = []
            L.isvd_last_error.restype = C.c_char_p
            for name in ("isvd_create_operator", "isvd_operator_shape", "isvd_apply", "isvd_apply_T", "isvd_svd",
                         "isvd_gaussian", "isvd_philox_words", "isvd_orthonormalize", "isvd_small_svd",
                         "isvd_closed_form", "isvd_compose_operators", "isvd_embed", "isvd_pair_scores",
                         "isvd_edge_kernel_weights", "isvd_edge_kernel_scores", "isvd_edge_kernel_loss",
                         "isvd_get_tuning", "isvd_set_tuning", "isvd_orthonormalize_noalloc", "isvd_svd_batched", "isvd_autotune",
                         "isvd_svd_batched_persistent",
                         "isvd_composite_cache", "isvd_split_relu_forward", "isvd_split_relu_backward",
                         "isvd_selftest_wait"):
                getattr(L, name).restype = C.c_int
            _lib = L
    return _lib


def _check(status: int, where: str):
    if status != ISVD_OK:
        raise IsvdError(status, where, lib().isvd_last_error().decode(errors="replace"))


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return F32
    if t.dtype == torch.bfloat16:
        return BF16
    raise TypeError(f"blocks must be float32 or bfloat16, got {t.dtype}")


def _as_block(G: torch.Tensor) -> torch.Tensor:
    """A 2-D CUDA block whose row stride is a multiple of 8 and whose base is
    16-byte aligned (copying into a padded buffer when needed)."""
    if G.dim() == 1:
        G = G[:, None]
    if G.dim() != 2 or not G.is_cuda:
        raise ValueError("blocks must be 2-D CUDA tensors")
    ok = G.stride(1) == 1 and G.stride(0) % 8 == 0 and G.stride(0) >= G.shape[1] and G.data_ptr() % 16 == 0
    if ok:
        return G
    ld = (G.shape[1] + 7) // 8 * 8
    buf = torch.zeros((G.shape[0], ld), dtype=G.dtype, device=G.device)
    buf[:, : G.shape[1]] = G
    return buf[:, : G.shape[1]]


def new_block(rows: int, b: int, dtype=torch.float32, device="cuda") -> torch.Tensor:
    ld = (b + 7) // 8 * 8
    return torch.zeros((rows, ld), dtype=dtype, device=device)[:, :b]


class Operator:
    """Implicit design matrix on the GPU (App. A.3: shape, dot, T).

    form='poly':   M = sum_k c_k N^k + ones_coeff 11^T + adj_coeff A + sum_t a_t u_t v_t^T  (Eq. 3)
    form='concat': M = [X | N X | ... | N^L X]                                              (Eq. 6)
    norm='row': N = D^-1 A;  norm='sym': N = (D+I)^-1/2 (A+I) (D+I)^-1/2  (Sec. 2);
    norm='sym_noself': N = (D+I)^-1/2 A (D+I)^-1/2, label re-use's adjacency (Sec. 5.3).
    gather_rows: the operator is M[gather_rows, :] (Thm. 1's fit on training rows).
    Arrays may be numpy or torch; they are copied to the device and kept
    alive for the operator's lifetime."""

    def __init__(self, n, rowptr, colidx, *, values=None, form="poly", norm="row", coeffs=(1.0,),
                 ones_coeff=0.0, adj_coeff=0.0, lowrank=None, X=None, L=0, check_symmetry=True,
                 gather_rows=None, device="cuda", use_torch_allocator=True):
        L_ = lib()
        dev = torch.device(device)
        self._keep = []

        def dev_t(a, dtype):
            t = torch.as_tensor(np.asarray(a) if not torch.is_tensor(a) else a)
            t = t.to(device=dev, dtype=dtype).contiguous()
            self._keep.append(t)
            return t

        self.n = int(n)
        rp = dev_t(rowptr, torch.int32)
        ci = dev_t(colidx, torch.int32)
        vals = dev_t(values, torch.float32) if values is not None else None
        d = _Desc()
        d.form = FORM[form]
        d.norm = NORM[norm]
        d.A = _Csr(self.n, self.n, int(ci.numel()), rp.data_ptr(), ci.data_ptr(),
                   vals.data_ptr() if vals is not None else None)
        coeffs_np = np.ascontiguousarray(np.asarray(coeffs, dtype=np.float64).reshape(-1))
        self._coeffs = coeffs_np
        d.degree = len(coeffs_np) if form == "poly" else 0
        d.coeffs = coeffs_np.ctypes.data if form == "poly" else None
        d.ones_coeff = float(ones_coeff)
        d.adj_coeff = float(adj_coeff)
        if lowrank is not None:
            u, v, alpha = lowrank
            ut = dev_t(u, torch.float32)
            vt = dev_t(v, torch.float32)
            al = np.ascontiguousarray(np.asarray(alpha, dtype=np.float64).reshape(-1))
            self._alpha = al
            d.lr_rank = len(al)
            d.lr_u, d.lr_v, d.lr_alpha = ut.data_ptr(), vt.data_ptr(), al.ctypes.data
        d.L = int(L)
        if X is not None:
            if isinstance(X, (tuple, list)):  # (d, rowptr, colidx, values)
                dd, xr, xc, xv = X
                xr_t = dev_t(xr, torch.int32)
                xc_t = dev_t(xc, torch.int32)
                xv_t = dev_t(xv, torch.float32)
                d.d = int(dd)
                d.X = _Csr(self.n, int(dd), int(xc_t.numel()), xr_t.data_ptr(), xc_t.data_ptr(), xv_t.data_ptr())
            else:
                xt = dev_t(X, torch.float32)
                d.d = int(xt.shape[1])
                d.X_dense = xt.data_ptr()
        d.flags = 0 if check_symmetry else FLAG_SKIP_SYMMETRY_CHECK
        if gather_rows is not None:  # M[gather_rows, :] (strictly increasing rows)
            gr = dev_t(gather_rows, torch.int32)
            d.gather_rows = gr.data_ptr()
            d.n_gather = int(gr.numel())
        self._desc = d
        self._handle = C.c_void_p()
        alloc = C.byref(_TORCH_ALLOCATOR) if use_torch_allocator else None
        _check(L_.isvd_create_operator(C.byref(d), alloc, _stream(), C.byref(self._handle)), "isvd_create_operator")
        r, c = C.c_int64(), C.c_int64()
        _check(L_.isvd_operator_shape(self._handle, C.byref(r), C.byref(c)), "isvd_operator_shape")
        self.shape = (r.value, c.value)
        self.device = dev

    # ---- products (App. A.3: dot and T().dot) ----
    def apply(self, G: torch.Tensor, out: torch.Tensor | None = None, transpose: bool = False) -> torch.Tensor:
        squeeze = G.dim() == 1
        G = _as_block(G)
        rows_in = self.shape[0] if transpose else self.shape[1]
        rows_out = self.shape[1] if transpose else self.shape[0]
        if G.shape[0] != rows_in:
            raise ValueError(f"G has {G.shape[0]} rows, operator needs {rows_in}")
        b = G.shape[1]
        if out is None:
            out = new_block(rows_out, b, G.dtype, G.device)
        elif out.shape != (rows_out, b) or out.dtype != G.dtype:
            raise ValueError("out has the wrong shape or dtype")
        fn = lib().isvd_apply_T if transpose else lib().isvd_apply
        _check(fn(self._handle, _ptr(G), G.stride(0), b, _ptr(out), out.stride(0), _dtype_code(G), _stream()),
               "isvd_apply_T" if transpose else "isvd_apply")
        return out[:, 0] if squeeze else out

    def dot(self, G):
        return self.apply(G)

    def dot_T(self, G):
        return self.apply(G, transpose=True)

    # ---- Alg. 1 ----
    def svd(self, k: int, oversample: int = 10, iters: int = 4, seed: int = 0, precision: str = "fp32",
            U=None, S=None, V=None, info=None, check: bool = True):
        r, c = self.shape
        U = new_block(r, k) if U is None else U
        V = new_block(c, k) if V is None else V
        S = torch.empty(k, dtype=torch.float32, device=self.device) if S is None else S
        info = torch.zeros(4, dtype=torch.int32, device=self.device) if info is None else info
        _check(lib().isvd_svd(self._handle, k, oversample, iters, C.c_uint64(seed), PREC[precision], _ptr(U),
                              U.stride(0), _ptr(S), _ptr(V), V.stride(0), _ptr(info), _stream()), "isvd_svd")
        if check:
            torch.cuda.current_stream().synchronize()
            st = int(info[0].item())
            if st != ISVD_OK:
                raise IsvdError(st, "isvd_svd (device)", "reported by the GPU")
        return U, S, V, info

    # ---- launch shapes of the sparse products ----
    _TUNING_FIELDS = ("slab_cols_f32", "slab_cols_bf16", "heavy_threshold", "heavy_chunk", "flags", "chunk_nnz",
                      "l2_budget_mb")

    def tuning(self) -> dict:
        t = (C.c_int32 * 7)()
        _check(lib().isvd_get_tuning(self._handle, t), "isvd_get_tuning")
        d = dict(zip(self._TUNING_FIELDS, list(t)))
        d["cache_hints"] = bool(d["flags"] & 1)
        d["hot_tags"] = bool(d["flags"] & 8)
        d["rows_occupancy"] = 3 if d["flags"] & 16 else 2
        d["prefetch"] = bool(d["flags"] & 32)
        d["packed"] = bool(d["flags"] & 64)
        d["kernel"] = ("slab" if d["flags"] & 128 else "ring" if d["flags"] & 4 else "rows" if d["flags"] & 2
                       else "chunks")
        return d

    def set_tuning(self, kernel=None, cache_hints=None, hot_tags=None, rows_occupancy=None, prefetch=None,
                   packed=None, **fields):
        """kernel: 'ring' (nonzero chunks, full-width gathers through shared
        memory), 'rows' (row groups with hub splitting) or 'chunks' (nonzero
        chunks over narrow column slabs); other keys as in isvd_tuning."""
        cur = self.tuning()
        vals = [int(fields.get(k, cur[k])) for k in self._TUNING_FIELDS]
        if cache_hints is not None:
            vals[4] = (vals[4] & ~1) | (1 if cache_hints else 0)
        if hot_tags is not None:
            vals[4] = (vals[4] & ~8) | (8 if hot_tags else 0)
        if rows_occupancy is not None:
            vals[4] = (vals[4] & ~16) | (16 if rows_occupancy >= 3 else 0)
        if prefetch is not None:
            vals[4] = (vals[4] & ~32) | (32 if prefetch else 0)
        if packed is not None:
            vals[4] = (vals[4] & ~64) | (64 if packed else 0)
        if kernel is not None:
            if kernel not in ("slab", "ring", "rows", "chunks"):
                raise ValueError(f"unknown kernel {kernel!r}")
            vals[4] = (vals[4] & ~134) | {"slab": 128, "ring": 4, "rows": 2, "chunks": 0}[kernel]
        t = (C.c_int32 * 7)(*vals)
        _check(lib().isvd_set_tuning(self._handle, t, _stream()), "isvd_set_tuning")
        return self.tuning()

    def autotune(self, b: int, dtype=torch.float32, cache_path: str | None = None) -> dict:
        """Time isvd_apply over the candidate launch shapes at block width b
        and keep the fastest (isvd_autotune); returns the chosen tuning."""
        code = F32 if dtype == torch.float32 else BF16
        t = (C.c_int32 * 7)()
        path = cache_path.encode() if cache_path else None
        _check(lib().isvd_autotune(self._handle, int(b), code, path, t, _stream()), "isvd_autotune")
        return self.tuning()

    def graph_kernel_nodes(self) -> int:
        """Kernel launches in the graph replayed by the last svd() call."""
        return int(lib().isvd_graph_kernel_nodes(self._handle))

    def close(self):
        if getattr(self, "_handle", None) and self._handle.value:
            lib().isvd_destroy_operator(self._handle)
            self._handle = C.c_void_p()
        self._keep = []

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def graph_operator(g, **kw) -> Operator:
    """Operator on a ``synth.Graph`` (undirected CSR)."""
    return Operator(g.n, g.rowptr, g.colidx, **kw)


COMPOSE = {"sum": 0, "hcat": 1, "vcat": 2, "product": 3}


def compose(kind: str, ops, weights=None, use_torch_allocator=True) -> Operator:
    """Composite operator (Sec. 4): ``'sum'`` sum_i w_i M_i, ``'hcat'``
    [M_1 | M_2 | ...], ``'vcat'`` [M_1 ; M_2 ; ...], ``'product'`` M_1 M_2 ...
    The children stay referenced by the result and must not be closed before
    it; tune them, not the composite."""
    ops = list(ops)
    if not ops:
        raise ValueError("compose needs at least one operator")
    op = Operator.__new__(Operator)
    op._keep = list(ops)
    arr = (C.c_void_p * len(ops))(*[o._handle.value for o in ops])
    w = None
    if weights is not None:
        w = np.ascontiguousarray(np.asarray(weights, dtype=np.float64).reshape(-1))
        if len(w) != len(ops):
            raise ValueError("one weight per operator")
    op._handle = C.c_void_p()
    alloc = C.byref(_TORCH_ALLOCATOR) if use_torch_allocator else None
    _check(lib().isvd_compose_operators(COMPOSE[kind], arr, len(ops), w.ctypes.data if w is not None else None,
                                        alloc, _stream(), C.byref(op._handle)), "isvd_compose_operators")
    r, c = C.c_int64(), C.c_int64()
    _check(lib().isvd_operator_shape(op._handle, C.byref(r), C.byref(c)), "isvd_operator_shape")
    op.shape = (r.value, c.value)
    op.device = ops[0].device
    op.n = ops[0].n
    return op


def set_product_cache(op: Operator, enable: bool) -> None:
    """Turn a composite's lazy product cache (App. A.3) on or off."""
    _check(lib().isvd_composite_cache(op._handle, 1 if enable else 0), "isvd_composite_cache")


def scale(op: Operator, w: float) -> Operator:
    """Scalar node w M (Sec. 4): a one-child weighted sum."""
    return compose("sum", [op], [w])


def power(op: Operator, p: int) -> Operator:
    """Power node M^p of a square operator (Sec. 4): the product of p copies
    (1 <= p <= 16), applied one factor after another."""
    if not 1 <= int(p) <= 16:
        raise ValueError("power needs 1 <= p <= 16")
    return compose("product", [op] * int(p))


def info_dict(info: torch.Tensor) -> dict:
    v = info.cpu().tolist()
    return {"status": STATUS_NAMES.get(v[0], v[0]), "chol_shifts": v[1], "cholqr_passes": v[2], "iters_done": v[3]}


def gaussian(seed: int, rows: int, cols: int, dtype=torch.float32, device="cuda") -> torch.Tensor:
    """Alg. 1's N(0,1) start block from Philox4x32-10 (counter-based)."""
    out = new_block(rows, cols, dtype, device)
    code = F32 if dtype == torch.float32 else BF16
    _check(lib().isvd_gaussian(C.c_uint64(seed), rows, cols, _ptr(out), out.stride(0), code, _stream()),
           "isvd_gaussian")
    return out


def philox_words(seed: int, rows: int, device="cuda") -> torch.Tensor:
    out = torch.zeros((rows, 16), dtype=torch.int32, device=device)
    _check(lib().isvd_philox_words(C.c_uint64(seed), rows, _ptr(out), _stream()), "isvd_philox_words")
    return out


def orthonormalize(op: Operator, Q: torch.Tensor, want_r: bool = True):
    """CholeskyQR2 (Alg. 2) in place on an FP32 block; returns (Q, R, info)."""
    if Q.dtype != torch.float32:
        raise TypeError("orthonormalize takes an FP32 block")
    Q = _as_block(Q)
    rows, l = Q.shape
    R = torch.zeros((l, l), dtype=torch.float64, device=Q.device) if want_r else None
    info = torch.zeros(4, dtype=torch.int32, device=Q.device)
    _check(lib().isvd_orthonormalize(op._handle, _ptr(Q), rows, l, Q.stride(0), _ptr(R), _ptr(info), _stream()),
           "isvd_orthonormalize")
    return Q, R, info


def small_svd(op: Operator, A: torch.Tensor, info: torch.Tensor | None = None):
    """SVD of a small square FP64 matrix (one-sided Jacobi): A = U diag(S) V^T.
    `info` (int32[4] on the device, optional) receives the status and, in
    iters_done, the number of sweeps."""
    A = A.to(torch.float64).contiguous()
    l = A.shape[0]
    U = torch.zeros((l, l), dtype=torch.float64, device=A.device)
    V = torch.zeros((l, l), dtype=torch.float64, device=A.device)
    S = torch.zeros(l, dtype=torch.float64, device=A.device)
    _check(lib().isvd_small_svd(op._handle, _ptr(A), l, _ptr(U), _ptr(S), _ptr(V), _ptr(info), _stream()),
           "isvd_small_svd")
    return U, S, V


def closed_form(op: Operator, U: torch.Tensor, S: torch.Tensor, V: torch.Tensor, Y: torch.Tensor,
                rcond: float = 1e-6, out: torch.Tensor | None = None) -> torch.Tensor:
    """Least-norm weights W = V diag(S)^+ U^T Y from a rank-k SVD of M
    (Thm. 1)."""
    for t in (U, S, V, Y):
        if t.dtype != torch.float32 or not t.is_cuda:
            raise TypeError("closed_form takes FP32 CUDA tensors")
    r, c = op.shape
    k = S.numel()
    m = Y.shape[1]
    if U.shape != (r, k) or V.shape != (c, k) or Y.shape[0] != r:
        raise ValueError("U, S, V, Y do not match the operator's shape")
    U, V, Y = _as_block(U), _as_block(V), _as_block(Y)
    S = S.contiguous()
    W = new_block(c, m, device=U.device) if out is None else out
    _check(lib().isvd_closed_form(op._handle, _ptr(U), U.stride(0), _ptr(S), _ptr(V), V.stride(0), k, _ptr(Y),
                                  Y.stride(0), m, float(rcond), _ptr(W), W.stride(0), _stream()), "isvd_closed_form")
    return W


def embeddings(U: torch.Tensor, S: torch.Tensor, V: torch.Tensor):
    """Network-embedding outputs of a rank-k SVD (Sec. 3.1): L = U S^1/2 and
    R = V S^1/2 (new FP32 blocks)."""
    for t in (U, S, V):
        if t.dtype != torch.float32 or not t.is_cuda:
            raise TypeError("embeddings takes FP32 CUDA tensors")
    k = S.numel()
    if U.dim() != 2 or V.dim() != 2 or U.shape[1] != k or V.shape[1] != k:
        raise ValueError("U and V need k = len(S) columns")
    S = S.contiguous()
    outs = []
    for X in (U, V):
        X = _as_block(X)
        out = new_block(X.shape[0], k, device=X.device)
        _check(lib().isvd_embed(_ptr(X), X.stride(0), X.shape[0], k, _ptr(S), _ptr(out), out.stride(0), _stream()),
               "isvd_embed")
        outs.append(out)
    return outs[0], outs[1]


def pair_scores(Lm: torch.Tensor, Rm: torch.Tensor, src: torch.Tensor, dst: torch.Tensor,
                info: torch.Tensor | None = None) -> torch.Tensor:
    """f(i, j) = <L_i, R_j> for each pair (src[p], dst[p]) (Sec. 3.1).  Pairs
    out of range score NaN and set info[0] (if given) to INVALID_ARGUMENT."""
    for t in (Lm, Rm):
        if t.dtype != torch.float32 or not t.is_cuda or t.dim() != 2:
            raise TypeError("pair_scores takes FP32 CUDA blocks")
    if Lm.shape[1] != Rm.shape[1]:
        raise ValueError("L and R need the same width")
    Lm, Rm = _as_block(Lm), _as_block(Rm)
    src = src.to(device=Lm.device, dtype=torch.int32).contiguous()
    dst = dst.to(device=Lm.device, dtype=torch.int32).contiguous()
    if src.shape != dst.shape or src.dim() != 1:
        raise ValueError("src and dst must be 1-D of equal length")
    out = torch.empty(src.numel(), dtype=torch.float32, device=Lm.device)
    _check(lib().isvd_pair_scores(_ptr(Lm), Lm.stride(0), Lm.shape[0], _ptr(Rm), Rm.stride(0), Rm.shape[0],
                                  Lm.shape[1], _ptr(src), _ptr(dst), src.numel(), _ptr(out),
                                  _ptr(info) if info is not None else None, _stream()), "isvd_pair_scores")
    return out


class EdgeKernel:
    """Gaussian-kernel edge function of Sec. 5.1 (App. A.4) on a rank-k SVD:
    f(i, j) = U_i^T E_x[S^x] V_j with x ~ N(mu, s) truncated to [0.5, 2],
    parameterised by (mu, s_bar = log(1/(2 s^2))).  Starts at the plain SVD
    score (mu = 1, s -> 0) as the paper does."""

    def __init__(self, U: torch.Tensor, S: torch.Tensor, V: torch.Tensor, mu: float = 1.0, s: float = 1e-3):
        for t in (U, S, V):
            if t.dtype != torch.float32 or not t.is_cuda:
                raise TypeError("EdgeKernel takes FP32 CUDA tensors")
        self.k = S.numel()
        if U.shape[1] != self.k or V.shape[1] != self.k:
            raise ValueError("U and V need k = len(S) columns")
        self.U, self.V, self.S = _as_block(U), _as_block(V), S.contiguous()
        self.mu = float(mu)
        self.s_bar = float(np.log(1.0 / (2.0 * s * s)))
        self.work = torch.empty(int(lib().isvd_edge_kernel_work_doubles(self.k)), dtype=torch.float64,
                                device=U.device)

    def _pairs(self, a):
        return torch.as_tensor(a).to(device=self.U.device, dtype=torch.int32).contiguous()

    def weights(self) -> torch.Tensor:
        """(3, k) FP64: w = E_x[S^x], dw/dmu, dw/ds_bar."""
        w3 = torch.empty((3, self.k), dtype=torch.float64, device=self.U.device)
        _check(lib().isvd_edge_kernel_weights(_ptr(self.S), self.k, self.mu, self.s_bar, _ptr(w3), _stream()),
               "isvd_edge_kernel_weights")
        return w3

    def scores(self, src, dst, info: torch.Tensor | None = None) -> torch.Tensor:
        src, dst = self._pairs(src), self._pairs(dst)
        out = torch.empty(src.numel(), dtype=torch.float32, device=self.U.device)
        _check(lib().isvd_edge_kernel_scores(_ptr(self.U), self.U.stride(0), self.U.shape[0], _ptr(self.V),
                                             self.V.stride(0), self.V.shape[0], self.k, _ptr(self.S), self.mu,
                                             self.s_bar, _ptr(src), _ptr(dst), src.numel(), _ptr(out),
                                             _ptr(self.work), self.work.numel(), _ptr(info), _stream()),
               "isvd_edge_kernel_scores")
        return out

    def loss(self, pos, neg, k_neg: float = 10.0, info: torch.Tensor | None = None) -> torch.Tensor:
        """Eq. 9 over edges pos = (src, dst) and non-edges neg: a (3,) FP64
        device tensor [loss, dL/dmu, dL/ds_bar]."""
        ps, pd = self._pairs(pos[0]), self._pairs(pos[1])
        ns, nd = self._pairs(neg[0]), self._pairs(neg[1])
        out = torch.empty(3, dtype=torch.float64, device=self.U.device)
        _check(lib().isvd_edge_kernel_loss(_ptr(self.U), self.U.stride(0), self.U.shape[0], _ptr(self.V),
                                           self.V.stride(0), self.V.shape[0], self.k, _ptr(self.S), self.mu,
                                           self.s_bar, _ptr(ps), _ptr(pd), ps.numel(), _ptr(ns), _ptr(nd),
                                           ns.numel(), float(k_neg), _ptr(out), _ptr(self.work), self.work.numel(),
                                           _ptr(info), _stream()), "isvd_edge_kernel_loss")
        return out

    def fit(self, pos, neg, k_neg: float = 10.0, steps: int = 50, lr: float = 0.05) -> list:
        """Gradient descent on (mu, s_bar) (Eq. 9); returns the loss per step."""
        hist = []
        for _ in range(steps):
            L, gm, gs = self.loss(pos, neg, k_neg).tolist()
            hist.append(L)
            self.mu -= lr * gm
            self.s_bar -= lr * gs
        return hist


class _PersistentOptions(C.Structure):
    _fields_ = [("max_team", C.c_int32), ("rows_per_member", C.c_int32), ("spin_limit", C.c_int32),
                ("test_phantom", C.c_int32)]


class Batch:
    """Many independent rank-k SVDs in one call: isvd_svd_batched (one
    captured graph of parallel branches), or with ``persistent=True``
    isvd_svd_batched_persistent (one persistent kernel; FP32; ``max_team``,
    ``rows_per_member``, ``spin_limit`` and ``test_phantom`` as its options).
    Output buffers are allocated once and reused."""

    def __init__(self, ops, ks, oversample: int = 10, iters: int = 4, seed: int = 0, precision: str = "fp32",
                 persistent: bool = False, max_team: int = 0, rows_per_member: int = 0, spin_limit: int = 0,
                 test_phantom: bool = False):
        self.persistent = bool(persistent)
        self._opt = _PersistentOptions(int(max_team), int(rows_per_member), int(spin_limit),
                                       1 if test_phantom else 0)
        if len(ops) != len(ks) or not ops:
            raise ValueError("need one rank per operator")
        self.ops = list(ops)
        self.ks = [int(k) for k in ks]
        self.oversample, self.iters, self.seed, self.precision = int(oversample), int(iters), int(seed), precision
        dev = self.ops[0].device
        self.U = [torch.zeros((op.shape[0], k), dtype=torch.float32, device=dev) for op, k in zip(self.ops, self.ks)]
        self.V = [torch.zeros((op.shape[1], k), dtype=torch.float32, device=dev) for op, k in zip(self.ops, self.ks)]
        self.S = [torch.zeros(k, dtype=torch.float32, device=dev) for k in self.ks]
        self.info = torch.zeros((len(self.ops), 4), dtype=torch.int32, device=dev)
        n = len(self.ops)
        self._h_ops = (C.c_void_p * n)(*[op._handle.value for op in self.ops])
        self._h_k = (C.c_int32 * n)(*self.ks)
        self._h_U = (C.c_void_p * n)(*[t.data_ptr() for t in self.U])
        self._h_S = (C.c_void_p * n)(*[t.data_ptr() for t in self.S])
        self._h_V = (C.c_void_p * n)(*[t.data_ptr() for t in self.V])

    def run(self, check: bool = True):
        if self.persistent:
            if self.precision != "fp32":
                raise ValueError("the persistent batch runs in FP32")
            _check(lib().isvd_svd_batched_persistent(self._h_ops, self._h_k, len(self.ops), self.oversample,
                                                     self.iters, C.c_uint64(self.seed), self._h_U, self._h_S,
                                                     self._h_V, _ptr(self.info), C.byref(self._opt), _stream()),
                   "isvd_svd_batched_persistent")
        else:
            _check(lib().isvd_svd_batched(self._h_ops, self._h_k, len(self.ops), self.oversample, self.iters,
                                          C.c_uint64(self.seed), PREC[self.precision], self._h_U, self._h_S,
                                          self._h_V, _ptr(self.info), _stream()), "isvd_svd_batched")
        if check:
            torch.cuda.current_stream().synchronize()
            bad = torch.nonzero(self.info[:, 0]).reshape(-1).tolist()
            if bad:
                st = int(self.info[bad[0], 0])
                raise IsvdError(st, f"isvd_svd_batched (device, problem {bad[0]})", "reported by the GPU")
        return self.U, self.S, self.V

    @staticmethod
    def kernel_nodes() -> int:
        return int(lib().isvd_batched_kernel_nodes())


def selftest_wait(spin_limit: int = 1000, device="cuda") -> dict:
    """Run the bounded-wait self-test; the returned status should be TIMEOUT."""
    info = torch.zeros(4, dtype=torch.int32, device=device)
    _check(lib().isvd_selftest_wait(int(spin_limit), _ptr(info), _stream()), "isvd_selftest_wait")
    return info_dict(info)
