"""FP64 CPU oracle for the implicit randomized SVD (arXiv 2111.06312).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg use this package; the product path never does.
It shares no code with the CUDA path (``paper_2111_06312_gb300/csrc``).

The operator products, Alg. 1 and its steps live in ``isvd_oracle.c`` (plain
FP64 loops, one function per definition in the paper); this module compiles it
with gcc and marshals numpy arrays through ctypes.  The consumers of the SVD
are written here in numpy, FP64, step by step as the paper states them: the
closed form of Thm. 1, the embeddings and pair scores of Sec. 3.1, the
Gaussian-kernel edge function of Sec. 5.1 / App. A.4 and the Split-ReLU
network of Sec. 5.2.  The metric helpers at the bottom (principal angles,
residuals) use numpy as a library primitive.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "isvd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()

# N in Sec. 2: "row" T = D^-1 A; "sym" Â = (D+I)^-1/2 (A+I) (D+I)^-1/2;
# "sym_noself" Â - (D+I)^-1, label re-use's adjacency (Sec. 5.3)
NORMS = {"row": 0, "sym": 1, "sym_noself": 2}


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, -O2, OpenMP, strict IEEE) and return the path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               "-fno-fast-math", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Op(C.Structure):
    _fields_ = [
        ("form", C.c_int32), ("norm", C.c_int32), ("n", C.c_int64),
        ("rowptr", C.c_void_p), ("colidx", C.c_void_p), ("aval", C.c_void_p),
        ("degree", C.c_int32), ("coeff", C.c_void_p),
        ("ones_coeff", C.c_double), ("adj_coeff", C.c_double),
        ("d", C.c_int64), ("L", C.c_int32),
        ("xrowptr", C.c_void_p), ("xcolidx", C.c_void_p), ("xval", C.c_void_p),
        ("xdense", C.c_void_p),
        ("lr_rank", C.c_int32), ("lr_u", C.c_void_p), ("lr_v", C.c_void_p), ("lr_alpha", C.c_void_p),
        ("grows", C.c_void_p), ("ngather", C.c_int64),
        ("kind", C.c_int32), ("nchild", C.c_int32), ("child", C.c_void_p), ("weight", C.c_void_p),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P = C.c_void_p
            L.orc_apply.argtypes = [P, P, C.c_int64, P, C.c_int]
            L.orc_explicit.argtypes = [P, P]
            L.orc_rows.argtypes = [P]
            L.orc_rows.restype = C.c_int64
            L.orc_cols.argtypes = [P]
            L.orc_cols.restype = C.c_int64
            L.orc_philox4x32_10.argtypes = [P, P, P]
            L.orc_gaussian.argtypes = [C.c_uint64, C.c_int64, C.c_int64, P, C.c_int64]
            L.orc_cholesky.argtypes = [P, C.c_int64, P]
            L.orc_cholqr.argtypes = [P, C.c_int64, C.c_int64, C.c_double, P]
            L.orc_cholqr2.argtypes = [P, C.c_int64, C.c_int64, P]
            L.orc_householder_qr.argtypes = [P, C.c_int64, C.c_int64, P]
            L.orc_jacobi_svd.argtypes = [P, C.c_int64, C.c_int64, P, P, P, C.c_double, C.c_int]
            L.orc_isvd.argtypes = [P, C.c_int32, C.c_int32, C.c_int32, C.c_uint64, P, P, P, P]
            _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Operator:
    """Implicit design matrix.  ``form='poly'``: sum_k c_k N^k + alpha 11^T +
    beta A + sum_t a_t u_t v_t^T (Eq. 3 with alpha = -lambda, beta = +lambda;
    ``lowrank=(u, v, a)``).  ``form='concat'``:
    [X | NX | ... | N^L X] (Eq. 6).  ``norm='row'``: N = T = D^-1 A;
    ``norm='sym'``: N = Â = (D+I)^-1/2 (A+I) (D+I)^-1/2 (Sec. 2).
    ``gather_rows``: the operator is M[gather_rows, :] (the training rows of
    Thm. 1's fit)."""

    def __init__(self, n, rowptr, colidx, *, form="poly", norm="row", values=None,
                 coeffs=(), ones_coeff=0.0, adj_coeff=0.0, lowrank=None,
                 X=None, L=0, gather_rows=None):
        self._keep = []

        def keep(a):
            self._keep.append(a)
            return a

        s = _Op()
        s.form = 0 if form == "poly" else 1
        s.norm = NORMS[norm]
        s.n = int(n)
        s.rowptr = _p(keep(np.ascontiguousarray(rowptr, dtype=np.int32)))
        s.colidx = _p(keep(np.ascontiguousarray(colidx, dtype=np.int32)))
        s.aval = _p(keep(_f64(values))) if values is not None else None
        c = keep(_f64(np.asarray(coeffs, dtype=np.float64).reshape(-1)))
        s.degree = len(c)
        s.coeff = _p(c) if len(c) else None
        s.ones_coeff = float(ones_coeff)
        s.adj_coeff = float(adj_coeff)
        s.L = int(L)
        if lowrank is not None:  # (u, v, alpha): n x r, n x r, r
            u, v, alpha = lowrank
            al = keep(_f64(np.asarray(alpha).reshape(-1)))
            s.lr_rank = len(al)
            s.lr_u = _p(keep(_f64(np.asarray(u).reshape(n, -1))))
            s.lr_v = _p(keep(_f64(np.asarray(v).reshape(n, -1))))
            s.lr_alpha = _p(al)
        if X is not None:
            if isinstance(X, np.ndarray):
                s.d = X.shape[1]
                s.xdense = _p(keep(_f64(X)))
            else:  # (d, rowptr, colidx, values)
                d, xr, xc, xv = X
                s.d = int(d)
                s.xrowptr = _p(keep(np.ascontiguousarray(xr, dtype=np.int32)))
                s.xcolidx = _p(keep(np.ascontiguousarray(xc, dtype=np.int32)))
                s.xval = _p(keep(_f64(xv)))
        if gather_rows is not None:  # M[gather_rows, :] (training rows of Thm. 1's fit)
            gr = keep(np.ascontiguousarray(gather_rows, dtype=np.int32))
            s.grows = _p(gr)
            s.ngather = len(gr)
        self.s = s
        self.form = form
        self.norm = norm

    @property
    def _ptr(self):
        return C.addressof(self.s)

    @property
    def shape(self):
        return int(lib().orc_rows(self._ptr)), int(lib().orc_cols(self._ptr))

    def apply(self, G, transpose=False):
        r, c = self.shape
        G = _f64(G)
        squeeze = G.ndim == 1
        if squeeze:
            G = G[:, None]
        assert G.shape[0] == (r if transpose else c)
        out = np.empty(((c if transpose else r), G.shape[1]), dtype=np.float64)
        lib().orc_apply(self._ptr, _p(G), G.shape[1], _p(out), 1 if transpose else 0)
        return out[:, 0] if squeeze else out

    def explicit(self):
        r, c = self.shape
        M = np.empty((r, c), dtype=np.float64)
        lib().orc_explicit(self._ptr, _p(M))
        return M

    def isvd(self, k, p, iters, seed):
        """Alg. 1 in FP64: returns U (r x k), S (k), V (c x k), passes."""
        r, c = self.shape
        U = np.empty((r, k))
        S = np.empty(k)
        V = np.empty((c, k))
        info = np.zeros(4, dtype=np.int32)
        rc = lib().orc_isvd(self._ptr, k, p, iters, C.c_uint64(seed), _p(U), _p(S), _p(V), _p(info))
        if rc != 0:
            raise RuntimeError(f"oracle isvd failed ({rc})")
        return U, S, V, int(info[0])


# composite nodes (Sec. 4, App. A.3)
COMPOSE = {"sum": 1, "hcat": 2, "vcat": 3, "product": 4}


def compose(kind: str, ops, weights=None) -> Operator:
    """Composite operator: ``'sum'`` sum_i w_i M_i (``weights``, default all
    ones), ``'hcat'`` [M_1 | M_2 | ...], ``'vcat'`` [M_1 ; M_2 ; ...],
    ``'product'`` M_1 M_2 ... (Sec. 4).  The children stay referenced."""
    ops = list(ops)
    if not ops:
        raise ValueError("compose needs at least one operator")
    op = Operator.__new__(Operator)
    op._keep = list(ops)
    s = _Op()
    s.kind = COMPOSE[kind]
    s.nchild = len(ops)
    arr = (C.c_void_p * len(ops))(*[o._ptr for o in ops])
    op._keep.append(arr)
    s.child = C.cast(arr, C.c_void_p)
    if weights is not None:
        w = _f64(np.asarray(weights, dtype=np.float64).reshape(-1))
        if len(w) != len(ops):
            raise ValueError("one weight per operator")
        op._keep.append(w)
        s.weight = _p(w)
    op.s = s
    op.form = "composite"
    op.norm = None
    rows = [o.shape for o in ops]
    ok = {"sum": all(r == rows[0] for r in rows), "hcat": all(r[0] == rows[0][0] for r in rows),
          "vcat": all(r[1] == rows[0][1] for r in rows),
          "product": all(rows[i][1] == rows[i + 1][0] for i in range(len(rows) - 1))}[kind]
    if not ok:
        raise ValueError(f"shapes {rows} do not fit a {kind} node")
    return op


def scale(op: Operator, w: float) -> Operator:
    """Scalar node w M: a one-child weighted sum (Sec. 4)."""
    return compose("sum", [op], [w])


def power(op: Operator, p: int) -> Operator:
    """Power node M^p: the product of p copies of a square M (Sec. 4)."""
    return compose("product", [op] * int(p))


def graph_operator(g, **kw) -> Operator:
    return Operator(g.n, g.rowptr, g.colidx, **kw)


def ne_coefficients(C_window: int) -> np.ndarray:
    """c_q = 2 (C - q + 1) / (C (C + 1)), q = 1..C: the context distribution of
    Sec. 2.1 normalised to sum 1 (Fig. 1 uses [3, 2, 1]/6 for C = 3)."""
    q = np.arange(1, C_window + 1, dtype=np.float64)
    return 2.0 * (C_window - q + 1) / (C_window * (C_window + 1))


def philox4x32_10(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def gaussian(seed, rows, cols):
    out = np.empty((rows, cols))
    lib().orc_gaussian(C.c_uint64(seed), rows, cols, _p(out), cols)
    return out


def cholesky(W):
    W = _f64(W)
    Lf = np.empty_like(W)
    info = lib().orc_cholesky(_p(W), W.shape[0], _p(Lf))
    return Lf, info


def cholqr(Q, shift=0.0):
    Q = _f64(Q).copy()
    R = np.empty((Q.shape[1], Q.shape[1]))
    info = lib().orc_cholqr(_p(Q), Q.shape[0], Q.shape[1], shift, _p(R))
    return Q, R, info


def cholqr2(Q):
    Q = _f64(Q).copy()
    R = np.empty((Q.shape[1], Q.shape[1]))
    passes = lib().orc_cholqr2(_p(Q), Q.shape[0], Q.shape[1], _p(R))
    return Q, R, passes


def householder_qr(Q):
    Q = _f64(Q).copy()
    R = np.empty((Q.shape[1], Q.shape[1]))
    lib().orc_householder_qr(_p(Q), Q.shape[0], Q.shape[1], _p(R))
    return Q, R


def jacobi_svd(A, tol=1e-15, max_sweeps=100):
    """A (r x c, r >= c) = U diag(S) V^T, S descending."""
    A = _f64(A)
    r, c = A.shape
    assert r >= c
    U = np.empty((r, c))
    S = np.empty(c)
    V = np.empty((c, c))
    sweeps = lib().orc_jacobi_svd(_p(A), r, c, _p(U), _p(S), _p(V), tol, max_sweeps)
    if sweeps < 0:
        raise RuntimeError("Jacobi did not converge")
    return U, S, V


def svd_any(A):
    """Jacobi SVD for either orientation (wide matrices via the transpose)."""
    A = _f64(A)
    if A.shape[0] >= A.shape[1]:
        return jacobi_svd(A)
    U, S, V = jacobi_svd(A.T)
    return V, S, U


def num_threads() -> int:
    lib()
    return int(C.CDLL(_LIB_PATH).orc_num_threads())


# ---- closed-form training outputs ------------------------------------------

def closed_form(U, S, V, Y, rcond=1e-6):
    """Thm. 1 (Sec. 3): the least-norm minimiser of ||M W - Y||_F is M^+ Y;
    with M = U diag(S) V^T (rank k) it is W = V diag(S)^+ U^T Y, where
    diag(S)^+ inverts S_i > rcond * max(S) and zeroes the rest.  FP64; the
    two products are numpy matmuls used as library primitives."""
    U, S, V, Y = (np.asarray(a, dtype=np.float64) for a in (U, S, V, Y))
    smax = S.max() if S.size else 0.0
    inv = np.where((S > 0) & (S > rcond * smax), 1.0 / np.where(S > 0, S, 1.0), 0.0)
    return V @ (inv[:, None] * (U.T @ Y))


def embeddings(U, S, V):
    """Network-embedding outputs of a rank-k SVD (Sec. 3.1): L = U S^1/2 and
    R = V S^1/2, so that L R^T = U diag(S) V^T.  FP64."""
    U, S, V = (np.asarray(a, dtype=np.float64) for a in (U, S, V))
    h = np.sqrt(S)
    return U * h[None, :], V * h[None, :]


def pair_scores(Lm, Rm, src, dst):
    """Similarity of the node at row i and the node at column j (Sec. 3.1):
    f(i, j) = <L_i, R_j>, for each pair (src[p], dst[p]).  FP64 loop."""
    Lm = np.asarray(Lm, dtype=np.float64)
    Rm = np.asarray(Rm, dtype=np.float64)
    out = np.empty(len(src))
    for p, (i, j) in enumerate(zip(src, dst)):
        out[p] = float(np.dot(Lm[i], Rm[j]))
    return out


# ---- Gaussian-kernel edge function (Sec. 5.1, App. A.4) ----------------------

def edge_kernel_grid(lo=0.5, hi=2.0, count=301):
    """The discretised truncation interval of App. A.4: 301 points from 0.5
    to 2.0, step 0.005."""
    return lo + (hi - lo) * np.arange(count, dtype=np.float64) / (count - 1)


def edge_kernel_weights(S, mu, s_bar, grid=None):
    """E_x[S^x] for x on the grid, weighted by softmax_x(-(x - mu)^2 exp(s_bar))
    (App. A.4, with s_bar = log(1 / (2 s^2))), and its derivatives in mu and
    s_bar.  Returns w, dw/dmu, dw/ds_bar (each of length k).  FP64, plain."""
    S = np.asarray(S, dtype=np.float64)
    x = edge_kernel_grid() if grid is None else np.asarray(grid, dtype=np.float64)
    e = np.exp(s_bar)
    z = -((x - mu) ** 2) * e
    ez = np.exp(z - z.max())
    pi = ez / ez.sum()  # softmax over the grid
    Sx = S[None, :] ** x[:, None]  # the constant tensor {S^x}, grid x k
    dz_mu = 2.0 * (x - mu) * e
    dz_s = z
    dpi_mu = pi * (dz_mu - np.dot(pi, dz_mu))  # softmax Jacobian applied to dz
    dpi_s = pi * (dz_s - np.dot(pi, dz_s))
    return pi @ Sx, dpi_mu @ Sx, dpi_s @ Sx


def edge_scores(U, V, w, src, dst):
    """f(i, j) = U_i^T diag(w) V_j for each pair (Eq. 8 with w = E_x[S^x])."""
    U = np.asarray(U, dtype=np.float64)
    V = np.asarray(V, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    out = np.empty(len(src))
    for p, (i, j) in enumerate(zip(src, dst)):
        out[p] = float(np.sum(U[i] * w * V[j]))
    return out


def edge_kernel_loss(U, S, V, mu, s_bar, pos, neg, k_neg=10.0):
    """Eq. 9: -mean_pos log sigma(f) - k_n mean_neg log(1 - sigma(f)), and its
    gradient in (mu, s_bar) through f = U_i^T diag(w(mu, s_bar)) V_j.
    pos, neg: (src, dst) index arrays.  Returns (loss, dL/dmu, dL/ds_bar)."""
    w, dw_mu, dw_s = edge_kernel_weights(S, mu, s_bar)
    total = np.zeros(3)
    for (src, dst), sign, scale in ((pos, 1.0, 1.0 / len(pos[0])), (neg, -1.0, k_neg / len(neg[0]))):
        f = edge_scores(U, V, w, src, dst)
        a = edge_scores(U, V, dw_mu, src, dst)
        b = edge_scores(U, V, dw_s, src, dst)
        # -log sigma(sign f) = softplus(-sign f); d/df = -sign sigma(-sign f)
        total[0] += scale * np.sum(np.logaddexp(0.0, -sign * f))
        g = -sign / (1.0 + np.exp(sign * f)) * scale
        total[1] += np.sum(g * a)
        total[2] += np.sum(g * b)
    return total[0], total[1], total[2]


# ---- Split-ReLU graph network (Sec. 5.2) --------------------------------------

def _relu(t):
    return np.maximum(t, 0.0)


def split_relu(X, Wp, Wn):
    """SplitReLU(X; Wp, Wn) = [X Wp]_+ - [X Wn]_+ (Sec. 5.2)."""
    return _relu(X @ Wp) - _relu(X @ Wn)


def splitrelu_init(W_star, d, L):
    """The initialisation of Sec. 5.2: Wp = I, Wn = -I for every message-
    passing layer, Wop_l = W*[dl : d(l+1)], Won_l = -W*[dl : d(l+1)]."""
    W_star = np.asarray(W_star, dtype=np.float64)
    Wp = [np.eye(d) for _ in range(L)]
    Wn = [-np.eye(d) for _ in range(L)]
    Wop = [W_star[d * l:d * (l + 1)].copy() for l in range(L + 1)]
    Won = [-W_star[d * l:d * (l + 1)] for l in range(L + 1)]
    return Wp, Wn, Wop, Won


def splitrelu_forward(prop, X, Wp, Wn, Wop, Won):
    """H_0 = X; H_{l+1} = [Â H_l Wp_l]_+ - [Â H_l Wn_l]_+ (message passing);
    output sum_{l=0..L} [H_l Wop_l]_+ - [H_l Won_l]_+ (Sec. 5.2).  prop(H) =
    Â H.  Returns the output and the layer inputs (H_l, and P_l = Â H_l)."""
    L = len(Wp)
    H = [np.asarray(X, dtype=np.float64)]
    P = []
    for l in range(L):
        P.append(prop(H[l]))
        H.append(split_relu(P[l], Wp[l], Wn[l]))
    out = sum(split_relu(H[l], Wop[l], Won[l]) for l in range(L + 1))
    return out, (H, P)


def splitrelu_backward(prop_T, cache, weights, dOut):
    """Gradients of sum(out * dOut) in every weight, by the chain rule
    through the forward pass above ([t]_+ has derivative 1 for t > 0, else 0).
    prop_T(G) = Â^T G.  Returns dWp, dWn, dWop, dWon (lists)."""
    H, P = cache
    Wp, Wn, Wop, Won = weights
    L = len(Wp)
    dWp, dWn = [None] * L, [None] * L
    dWop, dWon = [None] * (L + 1), [None] * (L + 1)
    dOut = np.asarray(dOut, dtype=np.float64)
    dH_up = None  # gradient reaching H_l from layer l + 1
    for l in range(L, -1, -1):
        gp = dOut * (H[l] @ Wop[l] > 0)
        gn = dOut * (H[l] @ Won[l] > 0)
        dWop[l] = H[l].T @ gp
        dWon[l] = -(H[l].T @ gn)
        dH = gp @ Wop[l].T - gn @ Won[l].T
        if dH_up is not None:
            dH = dH + dH_up
        if l >= 1:
            hp = dH * (P[l - 1] @ Wp[l - 1] > 0)
            hn = dH * (P[l - 1] @ Wn[l - 1] > 0)
            dWp[l - 1] = P[l - 1].T @ hp
            dWn[l - 1] = -(P[l - 1].T @ hn)
            dH_up = prop_T(hp @ Wp[l - 1].T - hn @ Wn[l - 1].T)
    return dWp, dWn, dWop, dWon


# ---- metrics ----------------------------------------------------------------

def sin_principal_angles(U_ref, U):
    """sin of the principal angles between span(U_ref) and span(U) (both with
    orthonormal columns): singular values of (I - U_ref U_ref^T) U."""
    U_ref = np.asarray(U_ref, dtype=np.float64)
    U = np.asarray(U, dtype=np.float64)
    Qr, _ = np.linalg.qr(U_ref)
    Qu, _ = np.linalg.qr(U)
    P = Qu - Qr @ (Qr.T @ Qu)
    return np.linalg.svd(P, compute_uv=False)


def max_principal_angle(U_ref, U) -> float:
    s = sin_principal_angles(U_ref, U)
    return float(np.arcsin(min(1.0, float(s.max())))) if len(s) else 0.0


def residuals(op: Operator, U, S, V):
    """r_i = max(||M v_i - s_i u_i||, ||M^T u_i - s_i v_i||), FP64 products."""
    MV = op.apply(V, transpose=False)
    MtU = op.apply(U, transpose=True)
    r1 = np.linalg.norm(MV - U * S[None, :], axis=0)
    r2 = np.linalg.norm(MtU - V * S[None, :], axis=0)
    return np.maximum(r1, r2)
