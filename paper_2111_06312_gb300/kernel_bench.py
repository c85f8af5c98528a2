"""Micro-benchmarks of the individual steps, for profiling and launch-shape sweeps.

  python -m paper_2111_06312_gb300.kernel_bench spmm  [--workload ne_large] [--width 144] [--dtype f32]
                                                      [--reps 5] [--slab 32] [--heavy 256] [--chunk 256]
  python -m paper_2111_06312_gb300.kernel_bench sweep [--workload ne_large] [--width 144] [--dtype f32]
  python -m paper_2111_06312_gb300.kernel_bench orth  [--rows 1000000] [--width 144] [--reps 5]
  python -m paper_2111_06312_gb300.kernel_bench svd   [--workload ne_large] [--k 128 --p 16 --q 6]

Each prints one JSON line per measured configuration (CUDA events on the
launching stream, L2 written over between repetitions).
"""
from __future__ import annotations

import argparse
import ctypes as C
import json

import numpy as np
import torch

from . import build, isvd, synth


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
    t = (C.c_int32 * 6)()
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
    ap.add_argument("what", choices=["spmm", "sweep", "orth", "svd"])
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
    ap.add_argument("--k", type=int, default=128)
    ap.add_argument("--p", type=int, default=16)
    ap.add_argument("--q", type=int, default=6)
    ap.add_argument("--precision", default="fp32")
    a = ap.parse_args()
    build.build()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    if a.what in ("spmm", "sweep"):
        g = synth.cached(a.workload)
        op = isvd.graph_operator(g, coeffs=[1.0], check_symmetry=False)
        if a.what == "spmm":
            tun = set_tuning(op, slab32=a.slab or None, slab16=a.slab or None, heavy=a.heavy or None,
                             chunk=a.chunk or None, row_kernel=True if a.row_kernel else None,
                             chunk_nnz=a.chunk_nnz or None)
            r = spmm_case(g, op, a.width, a.dtype, a.reps, flush)
            print(json.dumps({"what": "spmm", "workload": a.workload, "width": a.width, "dtype": a.dtype,
                              "tuning": tun, **r}), flush=True)
        else:
            cases = [dict(row_kernel=True, slab32=128, slab16=256, heavy=64, chunk=64, hints=h) for h in (0, 1)]
            cases += [dict(row_kernel=False, chunk_nnz=cn, hints=h) for cn in (256, 512, 1024, 2048) for h in (0, 1)]
            for kw in cases:
                tun = set_tuning(op, **kw)
                r = spmm_case(g, op, a.width, a.dtype, a.reps, flush)
                r.pop("all_ms")
                print(json.dumps({"what": "spmm", "width": a.width, "dtype": a.dtype, "tuning": tun, **r}),
                      flush=True)
        op.close()
    elif a.what == "orth":
        g = synth.cycle(64)
        op = isvd.graph_operator(g, coeffs=[1.0])
        Q0 = isvd.gaussian(3, a.rows, a.width)
        Q = Q0.clone()
        isvd.orthonormalize(op, Q, want_r=False)
        ts = _time(lambda: (Q.copy_(Q0), isvd.orthonormalize(op, Q, want_r=False)), a.reps, flush)
        print(json.dumps({"what": "orth", "rows": a.rows, "width": a.width, "ms_incl_copy": float(np.median(ts))}))
        op.close()
    else:
        g = synth.cached(a.workload)
        c5 = (6 - np.arange(1, 6)) / 15.0
        with isvd.graph_operator(g, coeffs=c5, ones_coeff=-0.05) as op:
            op.set_tuning(kernel="rows" if a.row_kernel else "chunks", chunk_nnz=a.chunk_nnz or 512)
            op.svd(a.k, a.p, a.q, 1, precision=a.precision)
            ts = _time(lambda: op.svd(a.k, a.p, a.q, 1, precision=a.precision, check=False), a.reps, flush)
            print(json.dumps({"what": "svd", "workload": a.workload, "k": a.k, "p": a.p, "q": a.q,
                              "precision": a.precision, "ms": float(np.median(ts)), "tuning": op.tuning(),
                              "kernels": op.graph_kernel_nodes()}))


if __name__ == "__main__":
    main()
