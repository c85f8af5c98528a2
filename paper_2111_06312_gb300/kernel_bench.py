"""Micro-benchmarks of the individual steps, for profiling and launch-shape sweeps.

  python -m paper_2111_06312_gb300.kernel_bench spmm  [--workload ne_large] [--width 144] [--dtype f32]
                                                      [--reps 5] [--slab 32] [--heavy 256] [--chunk 256]
  python -m paper_2111_06312_gb300.kernel_bench sweep [--workload ne_large] [--width 144] [--dtype f32]
  python -m paper_2111_06312_gb300.kernel_bench orth  [--rows 1000000] [--width 144] [--reps 5]
  python -m paper_2111_06312_gb300.kernel_bench svd   [--workload ne_large] [--k 128 --p 16 --q 6]
                                                      [--kernel rows|chunks] [--precision fp32|mixed] [--gather-frac 0.1]
  python -m paper_2111_06312_gb300.kernel_bench equal_error [--workload ne_large] [--k 128 --p 16 --q 6]
  python -m paper_2111_06312_gb300.kernel_bench batched [--count 256]
  python -m paper_2111_06312_gb300.kernel_bench finetune [--epochs 20]
  python -m paper_2111_06312_gb300.kernel_bench edge [--workload ne_large] [--k 128] [--pairs 1000000]
  python -m paper_2111_06312_gb300.kernel_bench compose [--epochs 20]
  python -m paper_2111_06312_gb300.kernel_bench splitrelu [--epochs 20]

Each prints one JSON line per measured configuration (CUDA events on the
launching stream, L2 written over between repetitions).
"""
from __future__ import annotations

import argparse
import ctypes as C
import json

import numpy as np
import torch

from . import adjoint, build, isvd, synth


def _flush(buf):
    buf.zero_()


def _time(fn, reps, flush):
    s = torch.cuda.current_stream()
    out = []
    for _ in range(reps):
        _flush(flush)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        fn()
        b.record(s)
        out.append((a, b))
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in out]


def set_tuning(op, slab32=None, slab16=None, heavy=None, chunk=None, hints=None, row_kernel=None, chunk_nnz=None):
    """Read-modify-write of isvd_tuning: [slab_f32, slab_bf16, heavy_threshold,
    heavy_chunk, flags (1 = L2 hints, 2 = row-group kernel), chunk_nnz]."""
    t = (C.c_int32 * 7)()
    isvd.lib().isvd_get_tuning.argtypes = [C.c_void_p, C.c_void_p]
    isvd.lib().isvd_set_tuning.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
    isvd.lib().isvd_get_tuning(op._handle, t)
    if slab32:
        t[0] = slab32
    if slab16:
        t[1] = slab16
    if heavy:
        t[2] = heavy
    if chunk:
        t[3] = chunk
    if hints is not None:
        t[4] = (t[4] & ~1) | (1 if hints else 0)
    if row_kernel is not None:
        t[4] = (t[4] & ~2) | (2 if row_kernel else 0)
    if chunk_nnz:
        t[5] = chunk_nnz
    isvd._check(isvd.lib().isvd_set_tuning(op._handle, t, isvd._stream()), "isvd_set_tuning")
    return list(t)


def spmm_case(g, op, width, dtype, reps, flush):
    dt = torch.float32 if dtype == "f32" else torch.bfloat16
    Q = isvd.gaussian(1, g.n, width, dtype=dt)
    Y = isvd.new_block(g.n, width, dtype=dt)
    for _ in range(2):
        op.apply(Q, out=Y)
    ts = _time(lambda: op.apply(Q, out=Y), reps, flush)
    es = 4 if dtype == "f32" else 2
    alg = 4 * (g.n + 1) + 4 * g.nnz + 2 * es * g.n * width
    ms = float(np.median(ts))
    return {"ms": ms, "gbs": alg / (ms * 1e-3) / 1e9, "alg_bytes": alg, "all_ms": ts}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["spmm", "sweep", "orth", "svd", "equal_error", "batched", "finetune", "edge",
                                     "compose", "splitrelu"])
    ap.add_argument("--pairs", type=int, default=1_000_000)  # edge: edges per loss (10x as many non-edges)
    ap.add_argument("--workload", default="ne_large")
    ap.add_argument("--width", type=int, default=144)
    ap.add_argument("--dtype", default="f32", choices=["f32", "bf16"])
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--slab", type=int, default=0)
    ap.add_argument("--heavy", type=int, default=0)
    ap.add_argument("--chunk", type=int, default=0)
    ap.add_argument("--chunk-nnz", type=int, default=0)
    ap.add_argument("--row-kernel", action="store_true")
    ap.add_argument("--rows", type=int, default=1_000_000)
    ap.add_argument("--rows-list", default="")
    ap.add_argument("--k", type=int, default=128)
    ap.add_argument("--p", type=int, default=16)
    ap.add_argument("--q", type=int, default=6)
    ap.add_argument("--precision", default="fp32")
    ap.add_argument("--kernel", default=None, choices=["rows", "chunks", "ring"])
    ap.add_argument("--count", type=int, default=256)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--q-ref", type=int, default=0)
    ap.add_argument("--q-extra", type=int, default=4)
    ap.add_argument("--gather-frac", type=float, default=0.0)  # svd of M[rows, :] on this fraction of rows
    a = ap.parse_args()
    build.build()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    if a.what in ("spmm", "sweep"):
        g = synth.cached(a.workload)
        op = isvd.graph_operator(g, coeffs=[1.0], check_symmetry=False)
        if a.what == "spmm":
            tun = set_tuning(op, slab32=min(a.slab, 256) or None, slab16=a.slab or None, heavy=a.heavy or None,
                             chunk=a.chunk or None, row_kernel=True if a.row_kernel else None,
                             chunk_nnz=a.chunk_nnz or None)
            if a.kernel:
                tun = op.set_tuning(kernel=a.kernel)
            r = spmm_case(g, op, a.width, a.dtype, a.reps, flush)
            print(json.dumps({"what": "spmm", "workload": a.workload, "width": a.width, "dtype": a.dtype,
                              "tuning": tun, **r}), flush=True)
        else:
            cases = [dict(kernel="rows", slab_cols_f32=128, slab_cols_bf16=256, cache_hints=1, hot_tags=1,
                          rows_occupancy=o, l2_budget_mb=64, prefetch=pf) for o in (2, 3) for pf in (0, 1)]
            cases += [dict(kernel="rows", slab_cols_f32=128, slab_cols_bf16=256, cache_hints=h, hot_tags=t,
                           rows_occupancy=3, l2_budget_mb=96, prefetch=0) for h, t in ((0, 0), (1, 0))]
            cases += [dict(kernel="rows", slab_cols_f32=256, slab_cols_bf16=512, cache_hints=1, hot_tags=1,
                           rows_occupancy=o, l2_budget_mb=mb) for o in (2, 3) for mb in (64, 96)]
            cases += [dict(kernel="rows", slab_cols_f32=128, slab_cols_bf16=256, cache_hints=1, hot_tags=1,
                           rows_occupancy=3, l2_budget_mb=mb) for mb in (24, 48, 64, 80, 96, 112, 128)]
            cases += [dict(kernel="rows", slab_cols_f32=128, slab_cols_bf16=256, cache_hints=1, hot_tags=1,
                           rows_occupancy=3, l2_budget_mb=64, heavy_threshold=ht, heavy_chunk=ht) for ht in (64, 256)]
            for kw in cases:
                if a.dtype == "bf16" and kw.get("slab_cols_f32") == 256:
                    kw = dict(kw, slab_cols_bf16=512)
                tun = op.set_tuning(**kw)
                r = spmm_case(g, op, a.width, a.dtype, a.reps, flush)
                r.pop("all_ms")
                print(json.dumps({"what": "spmm", "width": a.width, "dtype": a.dtype, "tuning": tun, **r}),
                      flush=True)
        op.close()
    elif a.what == "orth":
        g = synth.cycle(64)
        op = isvd.graph_operator(g, coeffs=[1.0])
        for rows in ([a.rows] if not a.rows_list else [int(x) for x in a.rows_list.split(",")]):
            Q0 = isvd.gaussian(3, rows, a.width)
            Q = Q0.clone()
            _, _, info = isvd.orthonormalize(op, Q, want_r=False)
            Qd = Q.double()
            orth = float((Qd.T @ Qd - torch.eye(a.width, dtype=torch.float64, device=Q.device)).abs().max())
            passes = isvd.info_dict(info)["cholqr_passes"]
            ts = _time(lambda: (Q.copy_(Q0), isvd.orthonormalize(op, Q, want_r=False)), a.reps, flush)
            print(json.dumps({"what": "orth", "rows": rows, "width": a.width, "ms_incl_copy": float(np.median(ts)),
                              "orthogonality": orth, "passes": passes}), flush=True)
        op.close()
    elif a.what == "svd":
        g = synth.cached(a.workload)
        rows = None
        if a.gather_frac > 0:  # seeded row subset (a training mask)
            rng = np.random.default_rng(synth.BASE_SEED + 7)
            rows = np.sort(rng.choice(g.n, int(a.gather_frac * g.n), replace=False)).astype(np.int32)
        with isvd.graph_operator(g, coeffs=C5, ones_coeff=-LAM, gather_rows=rows) as op:
            if a.kernel:
                op.set_tuning(kernel=a.kernel, chunk_nnz=a.chunk_nnz or 512)
            op.svd(a.k, a.p, a.q, 1, precision=a.precision)
            ts = _time(lambda: op.svd(a.k, a.p, a.q, 1, precision=a.precision, check=False), a.reps, flush)
            print(json.dumps({"what": "svd", "workload": a.workload, "k": a.k, "p": a.p, "q": a.q,
                              "precision": a.precision, "gather_rows": 0 if rows is None else len(rows),
                              "ms": float(np.median(ts)), "tuning": op.tuning(),
                              "kernels": op.graph_kernel_nodes()}))
    elif a.what == "equal_error":
        equal_error(a, flush)
    elif a.what == "batched":
        batched(a, flush)
    elif a.what == "edge":
        edge(a, flush)
    elif a.what == "compose":
        compose(a, flush)
    elif a.what == "splitrelu":
        splitrelu_epochs(a, flush)
    else:
        finetune(a, flush)


C5 = (6 - np.arange(1, 6)) / 15.0
LAM = 0.05
# "equal error": within 1% of the FP32 run's error (the resolution of the error estimates)
EQUAL_ERROR_TOL = 1.01


def _gapped_prefix(S_ref, k, rel_gap=1e-2):
    """Largest k' < k with sigma_k' - sigma_k'+1 > rel_gap * sigma_k' (0 if none)."""
    s = S_ref.double().cpu().numpy()
    best = 0
    for j in range(1, min(k, len(s) - 1) + 1):
        if s[j - 1] - s[j] > rel_gap * s[j - 1]:
            best = j
    return best


def _max_angle(U_ref, U, kp):
    """Largest principal angle between the spans of the first kp columns."""
    if kp == 0:
        return 0.0
    A = U_ref[:, :kp].double()
    B = U[:, :kp].double()
    P = B - A @ (A.T @ B)
    ev = torch.linalg.eigvalsh(P.T @ P).clamp_min(0)
    return float(torch.asin(torch.sqrt(ev.max()).clamp(max=1.0)))


def equal_error(a, flush):
    """Mixed vs FP32 at equal error: the FP32 run at q sets the target error
    (max principal angle of the gapped top-k left subspace and max relative
    singular-value error, both against an FP32 run with many more power
    iterations); the mixed run takes the smallest q' >= q that meets it."""
    g = synth.cached(a.workload)
    q_ref = a.q_ref or 4 * a.q
    with isvd.graph_operator(g, coeffs=C5, ones_coeff=-LAM) as op:
        U_ref, S_ref, _, _ = op.svd(a.k, a.p, q_ref, 7)
        U_ref, S_ref = U_ref.clone(), S_ref.clone()
        kp = _gapped_prefix(S_ref, a.k)

        def run(prec, q):
            U, S, V, info = op.svd(a.k, a.p, q, 1, precision=prec)
            ang = _max_angle(U_ref, U, kp)
            serr = float(((S.double() - S_ref.double()).abs() / S_ref.double())[:max(kp, 1)].max())
            ts = _time(lambda: op.svd(a.k, a.p, q, 1, precision=prec, check=False), a.reps, flush)
            rel = ((S.double() - S_ref.double()).abs() / S_ref.double()).cpu().numpy()
            return {"precision": prec, "q": q, "angle": ang, "sigma_err": serr, "sigma_err_top": float(rel[0]),
                    "sigma_err_median": float(np.median(rel)), "ms": float(np.median(ts))}

        base = run("fp32", a.q)
        rows = [base]
        chosen = None
        for q in range(a.q, a.q + a.q_extra + 1):
            r = run("mixed", q)
            rows.append(r)
            if chosen is None and r["angle"] <= base["angle"] * EQUAL_ERROR_TOL and \
                    r["sigma_err"] <= base["sigma_err"] * EQUAL_ERROR_TOL:
                chosen = r
                break
        out = {"what": "equal_error", "workload": a.workload, "k": a.k, "p": a.p, "q": a.q, "q_ref": q_ref,
               "gapped_prefix": kp, "equal_error_tolerance": EQUAL_ERROR_TOL, "runs": rows, "fp32": base,
               "mixed_at_equal_error": chosen,
               "speedup": (base["ms"] / chosen["ms"]) if chosen else None}
        print(json.dumps(out), flush=True)


def batched(a, flush):
    """Many small problems: one isvd_svd_batched call vs one isvd_svd call each,
    and mixed vs FP32 batched at equal error (max over problems of the largest
    principal angle of the gapped top-k subspace and of the relative singular
    value error there, against FP32 batched runs with 4x the power iterations)."""
    graphs, ranks = synth.workload_batched(count=a.count)
    ops = [isvd.graph_operator(gr, coeffs=C5, ones_coeff=-LAM) for gr in graphs]
    seed = 20211106315
    try:
        def run_batch(prec, q):
            b = isvd.Batch(ops, ranks, oversample=10, iters=q, seed=seed, precision=prec)
            b.run()
            ts = _time(lambda: b.run(check=False), a.reps, flush)
            U = [u.clone() for u in b.U]
            S = [x.clone() for x in b.S]
            return b, U, S, float(np.median(ts))

        _, U_ref, S_ref, _ = run_batch("fp32", 16)
        # per problem: the prefix of the reference spectrum separated by a 5% gap
        kps = [_gapped_prefix(S_ref[i], ranks[i], rel_gap=5e-2) for i in range(len(ops))]

        def errors(U, S):
            """(median over problems of the largest principal angle on the gapped
            prefix, median of the largest relative singular-value error there)."""
            angs, sigs = [], []
            for i in range(len(ops)):
                kp = kps[i]
                if not kp:
                    continue
                angs.append(_max_angle(U_ref[i], U[i], kp))
                rel = ((S[i].double() - S_ref[i].double()).abs() / S_ref[i].double())[:kp]
                sigs.append(float(rel.max()))
            return float(np.median(angs)), float(np.median(sigs))

        b32, U32, S32, t32 = run_batch("fp32", 4)
        e32 = errors(U32, S32)
        rows = []
        chosen = None
        for q in range(4, 8):
            bm, Um, Sm, tm = run_batch("mixed", q)
            em = errors(Um, Sm)
            rows.append({"q": q, "ms": tm, "angle": em[0], "sigma_err": em[1]})
            if em[0] <= e32[0] * EQUAL_ERROR_TOL and em[1] <= e32[1] * EQUAL_ERROR_TOL:
                chosen = rows[-1]
                break
        kernels = isvd.Batch.kernel_nodes()
        outs = [(isvd.new_block(op.shape[0], k), isvd.new_block(op.shape[1], k), torch.empty(k, device="cuda"))
                for op, k in zip(ops, ranks)]
        info = torch.zeros(4, dtype=torch.int32, device="cuda")

        def singles():
            for i, (op, k) in enumerate(zip(ops, ranks)):
                U, V, S = outs[i]
                op.svd(k, 10, 4, seed=seed + i, U=U, S=S, V=V, info=info, check=False)

        singles()
        torch.cuda.synchronize()
        t_single = _time(singles, a.reps, flush)
        print(json.dumps({"what": "batched", "count": len(ops), "sum_n": int(sum(gr.n for gr in graphs)),
                          "sum_nnz": int(sum(gr.nnz for gr in graphs)), "ranks": {int(k): int(v) for k, v in
                          zip(*np.unique(ranks, return_counts=True))}, "q": 4, "q_ref": 16,
                          "problems_with_gapped_prefix": int(sum(1 for kp in kps if kp)),
                          "error_metric": "median over problems of (max principal angle, max relative sigma error) "
                                          "on the 5%-gapped prefix vs FP32 with q = 16",
                          "batched_fp32_ms": t32, "fp32_angle": e32[0], "fp32_sigma_err": e32[1],
                          "equal_error_tolerance": EQUAL_ERROR_TOL, "mixed_runs": rows, "mixed_at_equal_error": chosen,
                          "speedup_mixed_vs_fp32": (t32 / chosen["ms"]) if chosen else None,
                          "single_calls_fp32_ms": float(np.median(t_single)), "kernels": kernels}), flush=True)
    finally:
        for op in ops:
            op.close()


def finetune(a, flush):
    """Linear model Y = M W on M = [X | ÂX | Â^2 X] (ogbn-arxiv-sized shapes):
    closed-form start from a rank-40 iSVD, then epochs of forward, cross-entropy
    on the training rows, backward (M^T dY) and an Adam step."""
    g, x, y, train = synth.workload_finetune()
    with isvd.Operator(g.n, g.rowptr, g.colidx, form="concat", norm="sym", X=x, L=2) as op:
        labels = torch.as_tensor(y).cuda()
        mask = torch.as_tensor(train).cuda()
        idx = torch.nonzero(mask).reshape(-1)
        Ylab = adjoint.one_hot_train(labels, mask, 40)
        adjoint.closed_form_init(op, Ylab, k=40, oversample=10, iters=4, seed=4)
        t_init = _time(lambda: adjoint.closed_form_init(op, Ylab, k=40, oversample=10, iters=4, seed=4), a.reps,
                       flush)
        W0, _ = adjoint.closed_form_init(op, Ylab, k=40, oversample=10, iters=4, seed=4)
        model = adjoint.ImplicitLinear(op, W0)
        opt = torch.optim.Adam(model.parameters(), lr=1e-3)
        f = torch.nn.functional.cross_entropy

        def epoch():
            opt.zero_grad()
            loss = f(model()[idx], labels[idx])
            loss.backward()
            opt.step()
            return loss

        acc0 = float((model().argmax(1)[idx] == labels[idx]).float().mean())
        for _ in range(3):
            epoch()
        t_epoch = _time(epoch, a.epochs, flush)
        r, c = op.shape
        W = W0.clone()
        dY = torch.randn((r, 40), device="cuda")
        Yb = isvd.new_block(r, 40)
        dWb = isvd.new_block(c, 40)
        t_fwd = _time(lambda: op.apply(W, out=Yb), a.reps, flush)
        t_bwd = _time(lambda: op.apply(dY, out=dWb, transpose=True), a.reps, flush)
        print(json.dumps({"what": "finetune", "n": g.n, "nnz": g.nnz, "d": x.shape[1], "outputs": 40,
                          "init_ms": float(np.median(t_init)), "epoch_ms": float(np.median(t_epoch)),
                          "forward_ms": float(np.median(t_fwd)), "backward_ms": float(np.median(t_bwd)),
                          "train_acc_at_init": acc0}), flush=True)


def edge(a, flush):
    """Gaussian-kernel edge function (Sec. 5.1): the Eq. 9 loss and gradient
    over `pairs` edges and 10x as many random non-edges, from the rank-k SVD of
    the NE operator.  Algorithmic bytes: two k-rows (FP32) and two indices per
    pair."""
    g = synth.cached(a.workload)
    with isvd.graph_operator(g, coeffs=C5, ones_coeff=-LAM, check_symmetry=False) as op:
        U, S, V, _ = op.svd(a.k, a.p, a.q, 1)
    rng = np.random.default_rng(synth.BASE_SEED + 11)
    e = rng.integers(0, g.nnz, a.pairs)
    src = np.searchsorted(g.rowptr, e, side="right") - 1  # row of nonzero e
    pos = (torch.as_tensor(src, dtype=torch.int32).cuda(), torch.as_tensor(g.colidx[e]).cuda())
    nneg = 10 * a.pairs
    neg = (torch.as_tensor(rng.integers(0, g.n, nneg), dtype=torch.int32).cuda(),
           torch.as_tensor(rng.integers(0, g.n, nneg), dtype=torch.int32).cuda())
    ek = isvd.EdgeKernel(U, S, V, mu=1.1, s=0.2)
    ek.loss(pos, neg)
    ts = _time(lambda: ek.loss(pos, neg), a.reps, flush)
    ms = float(np.median(ts))
    pairs = a.pairs + nneg
    bytes_ = pairs * (8 * a.k + 8)
    print(json.dumps({"what": "edge", "workload": a.workload, "k": a.k, "pairs": pairs, "ms": ms,
                      "pairs_per_s": pairs / (ms * 1e-3), "algorithmic_GBps": bytes_ / (ms * 1e-3) / 1e9}),
          flush=True)


def compose(a, flush):
    """Label re-use (Sec. 5.3) on ogbn-arxiv-sized inputs: [X | ÂX | Â^2 X] beside
    N0 [Y | N0 Y] (N0 = Â - (D+I)^-1), products and a rank-40 SVD, against the
    plain [X | ÂX | Â^2 X]."""
    g, x, y, train = synth.workload_finetune()
    classes = int(y.max()) + 1
    Y = np.zeros((g.n, classes), np.float32)
    Y[train, y[train]] = 1.0
    out = {"what": "compose", "n": g.n, "d": x.shape[1], "classes": classes}
    with isvd.graph_operator(g, form="concat", norm="sym", X=x, L=2) as nc, \
            isvd.graph_operator(g, norm="sym_noself", coeffs=[1.0]) as n0, \
            isvd.graph_operator(g, form="concat", norm="sym_noself", X=Y, L=1) as yb:
        lr = isvd.compose("hcat", [nc, isvd.compose("product", [n0, yb])])
        for name, op in (("nc", nc), ("label_reuse", lr)):
            G = isvd.gaussian(5, op.shape[1], 50)
            H = isvd.gaussian(6, op.shape[0], 50)
            out[name + "_apply_ms"] = float(np.median(_time(lambda: op.apply(G), a.reps, flush)))
            out[name + "_apply_T_ms"] = float(np.median(_time(lambda: op.apply(H, transpose=True), a.reps, flush)))
            op.svd(40, 10, 4, 1)
            out[name + "_svd_ms"] = float(np.median(_time(lambda: op.svd(40, 10, 4, 1, check=False), a.reps, flush)))
        lr.close()
    print(json.dumps(out), flush=True)


def splitrelu_epochs(a, flush):
    """Split-ReLU network (Sec. 5.2) with L = 2 on ogbn-arxiv-sized inputs,
    started from the closed-form W* of a rank-40 SVD: ms per fine-tuning epoch."""
    from .splitrelu import SplitReLUNet

    g, x, y, train = synth.workload_finetune()
    labels = torch.as_tensor(y).cuda()
    mask = torch.as_tensor(train).cuda()
    idx = torch.nonzero(mask).reshape(-1)
    with isvd.graph_operator(g, form="concat", norm="sym", X=x, L=2) as m, \
            isvd.graph_operator(g, norm="sym", coeffs=[1.0]) as prop:
        W0, _ = adjoint.closed_form_init(m, adjoint.one_hot_train(labels, mask, 40), k=40, seed=4)
        net = SplitReLUNet(prop, torch.as_tensor(x).cuda(), W0, 2)
        opt = torch.optim.Adam(net.parameters(), lr=1e-3)

        def epoch():
            opt.zero_grad(set_to_none=True)
            loss = torch.nn.functional.cross_entropy(net()[idx], labels[idx])
            loss.backward()
            opt.step()

        for _ in range(3):
            epoch()
        ts = _time(epoch, a.epochs, flush)
    print(json.dumps({"what": "splitrelu", "n": g.n, "d": x.shape[1], "L": 2, "epoch_ms": float(np.median(ts))}),
          flush=True)


if __name__ == "__main__":
    main()
