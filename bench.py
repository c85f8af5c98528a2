"""Benchmark: time to a rank-k implicit SVD on one GB300, FP32 and mixed
precision at equal error, plus the SpMM roofline.

Workload (default): the large network-embedding operator
M = sum_{k=1..5} c_k T^k - 0.05 11^T, c_k = (6-k)/15, T = D^-1 A on a seeded
Chung-Lu power-law graph (n = 10^6, 2x10^7 directed edges, max degree ~4x10^4),
rank 128, oversample 16, 6 power iterations (Alg. 1).  A step is one whole
isvd_svd (CUDA-graph replay) with the operator and inputs resident in HBM;
`value` is the FP32 arm's time per SVD.  The mixed arm (BF16 blocks in the
power iterations, FP32 refinement and Rayleigh-Ritz) is timed the same way,
at the configured iterations and at the smallest iteration count whose error
is no larger than the FP32 arm's (`equal_error`).

  python bench.py [--gpus N] [--steps K] [--warmup W]
  python bench.py --impl reference      # the FP64 CPU oracle, a bounded sample per step

Multi-GPU: the path does not shard across GPUs here (one GPU per problem);
N ranks run N independent replicas (weak scaling, no collective on the data
path) and the slowest rank's time is reported.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time to rank-k implicit SVD & SpMM HBM GB/s, mixed vs FP32 at equal error"
LAM = 0.05
SEED = 20211106312
GOLDEN = os.path.join(ROOT, "tests", "golden", "ne_large_k128_p16_q6.txt")
ORACLE_FULL_RUN = os.path.join(ROOT, "profiles", "oracle_alg1_ne_large.md")


def coeffs5():
    k = np.arange(1, 6, dtype=np.float64)
    return (6 - k) / 15.0


WORKLOADS = {
    # name: (description, k, p, q)
    "ne_large": ("NE operator sum_k c_k T^k - 0.05 11^T, Chung-Lu n=1e6 m=2e7 (gamma 2.5, max deg ~4.3e4), "
                 "rank 128, oversample 16, 6 power iters", 128, 16, 6),
    "ne_small": ("NE operator sum_k c_k T^k - 0.05 11^T, Chung-Lu n=2708 m~10.6k, rank 32, oversample 10, "
                 "4 power iters", 32, 10, 4),
}


def load_graph(name):
    from paper_2111_06312_gb300 import synth

    return synth.cached(name)


def config_of(desc, g, k, p, q, n_gpus):
    """The workload description shared by both arms' lines."""
    return {"workload": desc, "n": g.n, "nnz": g.nnz, "k": k, "oversample": p, "iters": q,
            "precision": "fp32 (value); mixed in equal_error", "parallelism": f"replicas x{n_gpus}",
            "l2": "256 MB buffer written between steps (untimed); per-step working set > 3 GB"}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d.get("bf16_tflops", 1900.0)), "measured"
    return 6800.0, 1900.0, "fallback"


KERNEL_SOURCES = {
    "slab": ("spmm.cu", "dense.cu"),
    "rows": ("spmm.cu", "dense.cu"),
    "ring": ("spmm_ring.cu", "dense.cu"),
    "chunks": ("spmm_chunk.cu", "dense.cu"),
}


def kernel_sources_sha1(kernel):
    h = hashlib.sha1()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_2111_06312_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def recorded_traffic(storage, kernel):
    """dram read+write bytes of one M.Q apply (all its kernels) with the given
    SpMM kernel, from the committed ncu summary; valid only while the sources
    of those kernels are unchanged."""
    path = os.path.join(ROOT, "profiles", "spmm_ne_large.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"traffic_bytes_per_apply_%s_%s:\s*([0-9.eE+]+)" % (storage, kernel), text)
    h = re.search(r"source_sha1_%s:\s*([0-9a-f]{40})" % kernel, text)
    if not m or not h:
        return None
    return float(m.group(1)) if kernel_sources_sha1(kernel) == h.group(1) else None


def golden_sigma():
    """The oracle's 128 singular values of the default workload (FP64 Alg. 1,
    same seed), written by tests/golden/make_ne_large_golden.py."""
    if not os.path.exists(GOLDEN):
        return None
    rows = [ln.split() for ln in open(GOLDEN) if ln.strip() and not ln.startswith("#")]
    return np.array([float(r[1]) for r in rows])


def oracle_full_run():
    """Wall time of one whole oracle Alg. 1 on the default workload, measured
    once (the run that wrote the golden file), from its committed summary."""
    if not os.path.exists(ORACLE_FULL_RUN):
        return None
    text = open(ORACLE_FULL_RUN).read()
    m = re.search(r"oracle_alg1_seconds:\s*([0-9.]+)", text)
    c = re.search(r"oracle_alg1_threads:\s*([0-9]+)", text)
    h = re.search(r"oracle_alg1_host:\s*(.+)", text)
    if not m:
        return None
    return {"seconds": float(m.group(1)), "threads": int(c.group(1)) if c else None,
            "host": h.group(1).strip() if h else None}


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------------------------
# CPU oracle sample (the reference arm and the cpu_baseline of our arm)
# ---------------------------------------------------------------------------------------------

SAMPLE_WIDTH = 16


def oracle_stage(op, n, width):
    """One power-iteration stage of Alg. 1 done by the FP64 oracle on the full
    graph at block width `width`: Y = M G, Z = M^T Y, CholeskyQR2 of Z.
    Returns the wall seconds of the two products and of the CholeskyQR2."""
    import oracle

    G = np.random.default_rng(0).standard_normal((n, width))
    t0 = time.perf_counter()
    Y = op.apply(G)
    Z = op.apply(Y, transpose=True)
    t1 = time.perf_counter()
    oracle.cholqr2(Z)
    return t1 - t0, time.perf_counter() - t1


def stage_estimate_ms(stages, k, p, q, width):
    """An ESTIMATE of one whole oracle SVD from stages at a narrower width:
    Alg. 1 takes 2(q+1) products (cost proportional to the width) and 2q+1
    CholeskyQR2 calls (Gram and Q R^-1: proportional to the width squared);
    the Rayleigh-Ritz Jacobi is not included."""
    l = k + p
    t_prod = float(np.mean([s[0] for s in stages]))
    t_chol = float(np.mean([s[1] for s in stages]))
    return 1e3 * ((q + 1) * t_prod * (l / width) + (2 * q + 1) * t_chol * (l / width) ** 2)


def stage_description(width, steps):
    return (f"each step: one Alg. 1 power-iteration stage by the FP64 oracle on the full graph at block width "
            f"{width} (M.G and M^T.G with the K=5 Horner products, then CholeskyQR2 of the n x {width} block); "
            f"{steps} steps")


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle

    oracle.build()
    desc, k, p, q = WORKLOADS[args.workload]
    g = load_graph(args.workload)
    op = oracle.graph_operator(g, coeffs=coeffs5(), ones_coeff=-LAM)
    for _ in range(args.warmup):
        oracle_stage(op, g.n, SAMPLE_WIDTH)
    t0 = time.perf_counter()
    steps = [oracle_stage(op, g.n, SAMPLE_WIDTH) for _ in range(args.steps)]
    wall = time.perf_counter() - t0
    ms = 1e3 * float(np.mean([sum(s) for s in steps]))
    cpu = {"value": ms, "unit": "ms", "cores": oracle.num_threads(), "kind": "oracle",
           "sample": stage_description(SAMPLE_WIDTH, args.steps),
           "estimate_full_svd_ms": stage_estimate_ms(steps, k, p, q, SAMPLE_WIDTH),
           "estimate_note": "not measured: scaled from the stage (products x width, CholeskyQR2 x width^2), "
                            "Rayleigh-Ritz excluded"}
    full = oracle_full_run()
    if full:
        cpu["full_svd_measured_once"] = full
    line = {"impl": "reference", "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(desc, g, k, p, q, args.gpus), "timed_wall_s": wall, "cpu_baseline": cpu,
            "e2e": {"value": ms, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------------------------

def slowest_rank_ms(ms, world, device):
    """The step time reported for N replicas: the slowest rank's (all-reduce MAX;
    the replicas share no data, so this is the only collective)."""
    if world <= 1:
        return float(ms)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def timed_steps(fn, steps, flush, stream):
    """CUDA-event time of each of `steps` calls on `stream`, with the L2 written
    over (untimed) before each."""
    import torch

    evs = []
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def relative_residuals(op, U, S, V):
    """r_i / s_i with r_i = max(||M v_i - s_i u_i||, ||M^T u_i - s_i v_i||), the
    products taken by the library in FP32: by the residual bound for the
    symmetric embedding [[0, M], [M^T, 0]], some singular value of M lies
    within r_i of s_i."""
    import torch

    MV = op.apply(V)
    MtU = op.apply(U, transpose=True)
    r = torch.maximum((MV - U * S[None, :]).norm(dim=0), (MtU - V * S[None, :]).norm(dim=0))
    return (r / S).double().cpu().numpy()


def batched_section(args, flush, stream):
    """Many uneven problems (256 seeded graphs, n ~ U[500, 50,000], mean degree
    8, rank drawn from {16, 32, 64}, oversample 10, 4 power iterations): one
    isvd_svd_batched call (graph of parallel branches) and one
    isvd_svd_batched_persistent call (one persistent kernel) against one
    isvd_svd call per problem, FP32 and mixed; equal error as for the single
    SVD, with the error the largest over all problems."""
    import torch

    from paper_2111_06312_gb300 import isvd, synth

    graphs, ranks = synth.workload_batched()
    seed, p, q = 20211106315, 10, 4
    ops = [isvd.graph_operator(gr, coeffs=coeffs5(), ones_coeff=-LAM) for gr in graphs]
    try:
        def batch_ms(prec, iters):
            b = isvd.Batch(ops, ranks, oversample=p, iters=iters, seed=seed, precision=prec)
            b.run()
            ms = float(np.mean(timed_steps(lambda: b.run(check=False), args.steps, flush, stream)))
            b.run()
            torch.cuda.synchronize()
            err = max(float(relative_residuals(op, b.U[i], b.S[i], b.V[i]).max()) for i, op in enumerate(ops))
            return ms, err

        ms32, err32 = batch_ms("fp32", q)
        msm, errm = batch_ms("mixed", q)
        # the same batch in one persistent kernel (FP32)
        bp = isvd.Batch(ops, ranks, oversample=p, iters=q, seed=seed, persistent=True)
        bp.run()
        ms_p = float(np.mean(timed_steps(lambda: bp.run(check=False), args.steps, flush, stream)))
        bp.run()
        torch.cuda.synchronize()
        err_p = max(float(relative_residuals(op, bp.U[i], bp.S[i], bp.V[i]).max()) for i, op in enumerate(ops))
        eq = None
        for qm in range(q, q + 5):
            t, e = (msm, errm) if qm == q else batch_ms("mixed", qm)
            if e <= err32:
                eq = {"iters": qm, "ms": t, "max_rel_residual": e, "speedup_mixed_over_fp32": ms32 / t}
                break
        outs = [(isvd.new_block(op.shape[0], k), isvd.new_block(op.shape[1], k), torch.empty(k, device="cuda"))
                for op, k in zip(ops, ranks)]
        info = torch.zeros(4, dtype=torch.int32, device="cuda")

        def singles():
            for i, (op, k) in enumerate(zip(ops, ranks)):
                U, V, S = outs[i]
                op.svd(k, p, q, seed=seed + i, U=U, S=S, V=V, info=info, check=False)

        singles()
        single_ms = float(np.mean(timed_steps(singles, max(1, args.steps // 2), flush, stream)))
        return {"count": len(ops), "sum_n": int(sum(gr.n for gr in graphs)),
                "sum_nnz": int(sum(gr.nnz for gr in graphs)), "oversample": p, "iters": q,
                "batched_fp32_ms": ms32, "single_calls_fp32_ms": single_ms, "speedup_batched_over_single": single_ms / ms32,
                "persistent_fp32_ms": ms_p, "persistent_max_rel_residual": err_p,
                "speedup_persistent_over_graph": ms32 / ms_p, "persistent_teams": int(sum(
                    min(32, max(1, -(-gr.n // 16384))) for gr in graphs)),
                "batched_mixed_ms": msm, "fp32_max_rel_residual": err32, "mixed_max_rel_residual": errm,
                "mixed_at_equal_error": eq,
                "error": "largest over all problems of max_i r_i / s_i (library FP32 products)"}
    finally:
        for op in ops:
            op.close()


def finetune_section(args, flush, stream):
    """Fine-tuning step of the linear model Y = M W, M = [X | ÂX | Â^2 X]
    (ogbn-arxiv-sized: n = 169,343, 1.17M directed edges, dense X n x 128,
    40 outputs, W 384 x 40 from the closed form of a rank-40 iSVD): forward
    M W, backward M^T dY, and one whole epoch (forward, cross-entropy on the
    training rows, backward, Adam step)."""
    import torch

    from paper_2111_06312_gb300 import adjoint, isvd, synth

    g, x, y, train = synth.workload_finetune()
    with isvd.Operator(g.n, g.rowptr, g.colidx, form="concat", norm="sym", X=x, L=2) as op:
        labels = torch.as_tensor(y).cuda()
        mask = torch.as_tensor(train).cuda()
        idx = torch.nonzero(mask).reshape(-1)
        Ylab = adjoint.one_hot_train(labels, mask, 40)
        W0, _ = adjoint.closed_form_init(op, Ylab, k=40, oversample=10, iters=4, seed=4)
        init_ms = float(np.mean(timed_steps(
            lambda: adjoint.closed_form_init(op, Ylab, k=40, oversample=10, iters=4, seed=4), 3, flush, stream)))
        model = adjoint.ImplicitLinear(op, W0)
        opt = torch.optim.Adam(model.parameters(), lr=1e-3)

        def epoch():
            opt.zero_grad()
            loss = torch.nn.functional.cross_entropy(model()[idx], labels[idx])
            loss.backward()
            opt.step()

        for _ in range(3):
            epoch()
        epoch_ms = float(np.mean(timed_steps(epoch, args.steps, flush, stream)))
        r, c = op.shape
        dY = torch.randn((r, 40), device="cuda")
        Yb = isvd.new_block(r, 40)
        dWb = isvd.new_block(c, 40)
        fwd = float(np.mean(timed_steps(lambda: op.apply(W0, out=Yb), args.steps, flush, stream)))
        bwd = float(np.mean(timed_steps(lambda: op.apply(dY, out=dWb, transpose=True), args.steps, flush, stream)))
        return {"n": g.n, "nnz": g.nnz, "d": int(x.shape[1]), "outputs": 40, "forward_ms": fwd, "backward_ms": bwd,
                "forward_plus_backward_ms": fwd + bwd, "epoch_ms": epoch_ms, "closed_form_init_ms": init_ms}


def wide_section(args, op, g, q, flush, stream):
    """The paper's own block width l = 2k at rank 256 (l = 512, FP32) on the
    same operator and iterations as the main line: the whole SVD, its error
    (max_i r_i / s_i over the top 256), and two of its steps alone: the
    orthonormalisation of an n x 512 block (128-column panels) and the small
    SVD of a 512 x 512 upper-triangular factor (global-memory Jacobi)."""
    import torch

    from paper_2111_06312_gb300 import isvd

    k, p = 256, 256
    l = k + p
    U = isvd.new_block(g.n, k)
    V = isvd.new_block(g.n, k)
    S = torch.empty(k, device="cuda")
    info = torch.zeros(4, dtype=torch.int32, device="cuda")
    fn = lambda: op.svd(k, p, q, seed=SEED, U=U, S=S, V=V, info=info, check=False)  # noqa: E731
    fn()
    torch.cuda.synchronize()
    st = isvd.info_dict(info)
    if st["status"] != "OK":
        raise RuntimeError(f"device status {st}")
    steps = max(2, args.steps // 3)
    ms = float(np.mean(timed_steps(fn, steps, flush, stream)))
    err = relative_residuals(op, U, S, V)
    del U, V
    Q0 = isvd.gaussian(5, g.n, l)
    Q = Q0.clone()
    isvd.orthonormalize(op, Q, want_r=False)
    orth_ms = float(np.mean(timed_steps(lambda: (Q.copy_(Q0), isvd.orthonormalize(op, Q, want_r=False)),
                                        steps, flush, stream)))
    copy_ms = float(np.mean(timed_steps(lambda: Q.copy_(Q0), steps, flush, stream)))
    del Q, Q0
    R = torch.linalg.qr(torch.randn((l, l), dtype=torch.float64, device="cuda"))[1]
    isvd.small_svd(op, R)
    jac_ms = float(np.mean(timed_steps(lambda: isvd.small_svd(op, R), steps, flush, stream)))
    return {"k": k, "oversample": p, "iters": q, "width": l, "ms": ms, "cholqr_passes": st["cholqr_passes"],
            "max_rel_residual": float(err.max()), "median_rel_residual": float(np.median(err)),
            "orthonormalize_ms": orth_ms - copy_ms, "orthonormalize_rows": g.n,
            "small_svd_ms": jac_ms}


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2111_06312_gb300 import build as libbuild
    from paper_2111_06312_gb300 import isvd

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    libbuild.build()
    dev = torch.device("cuda", local)

    desc, k, p, q = WORKLOADS[args.workload]
    g = load_graph(args.workload)
    l = k + p
    c5 = coeffs5()

    # operator construction (timed separately from the SVD)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    op = isvd.graph_operator(g, coeffs=c5, ones_coeff=-LAM, device=dev)
    torch.cuda.synchronize()
    construct_ms = (time.perf_counter() - t0) * 1e3

    U = isvd.new_block(g.n, k, device=dev)
    V = isvd.new_block(g.n, k, device=dev)
    S = torch.empty(k, device=dev)
    info = torch.zeros(4, dtype=torch.int32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)
    stream = torch.cuda.current_stream()

    def svd_fn(precision, iters):
        return lambda: op.svd(k, p, iters, seed=SEED, precision=precision, U=U, S=S, V=V, info=info, check=False)

    def checked_status():
        torch.cuda.synchronize()
        st = isvd.info_dict(info)
        if st["status"] != "OK":
            raise RuntimeError(f"device status {st}")
        return st

    # ---- the two arms at the configured iterations ----
    fp32 = svd_fn("fp32", q)
    mixed = svd_fn("mixed", q)
    for _ in range(args.warmup):
        fp32()
    st = checked_status()
    for _ in range(args.warmup):
        mixed()
    checked_status()

    clocks = ClockSampler(torch.cuda.current_device())
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    torch.cuda.nvtx.range_push("timed_steps")
    step_ms = timed_steps(fp32, args.steps, flush, stream)
    torch.cuda.nvtx.range_pop()
    kernels_per_step = op.graph_kernel_nodes()
    mixed_ms_list = timed_steps(mixed, args.steps, flush, stream)
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = slowest_rank_ms(float(np.mean(step_ms)), world, dev)
    mixed_ms = slowest_rank_ms(float(np.mean(mixed_ms_list)), world, dev)

    # ---- equal error: the smallest mixed iteration count whose error is no
    # larger than the FP32 arm's at q (error = max_i r_i / s_i over the top k) ----
    fp32()
    checked_status()
    S_fp32 = S.double().cpu().numpy()
    err_fp32 = relative_residuals(op, U, S, V)
    eq = {"error": "max over the top k of r_i / s_i, r_i = max(||M v_i - s_i u_i||, ||M^T u_i - s_i v_i||) "
                   "(library FP32 products)",
          "fp32": {"iters": q, "ms": ms, "max_rel_residual": float(err_fp32.max()),
                   "median_rel_residual": float(np.median(err_fp32))}}
    q_eq, err_m = None, None
    tried = []
    for qm in range(q, q + 6):
        svd_fn("mixed", qm)()
        checked_status()
        e = relative_residuals(op, U, S, V)
        tried.append({"iters": qm, "max_rel_residual": float(e.max())})
        if e.max() <= err_fp32.max():
            q_eq, err_m = qm, e
            break
    eq["mixed_tried"] = tried
    if q_eq is not None:
        fn = svd_fn("mixed", q_eq)
        for _ in range(max(1, args.warmup)):
            fn()
        checked_status()
        eq_ms = slowest_rank_ms(float(np.mean(timed_steps(fn, args.steps, flush, stream))), world, dev)
        eq["mixed"] = {"iters": q_eq, "ms": eq_ms, "max_rel_residual": float(err_m.max()),
                       "median_rel_residual": float(np.median(err_m))}
        eq["speedup_mixed_over_fp32"] = ms / eq_ms
    else:
        eq["mixed"] = {"iters": None, "note": f"no iteration count up to {q + 5} reached the FP32 error"}
    sig = golden_sigma()
    if sig is not None and args.workload == "ne_large":
        eq["fp32"]["max_sigma_rel_err_vs_oracle"] = float(np.max(np.abs(S_fp32 - sig) / sig))

    # ---- SpMM step roofline: one M.Q apply of this operator at the SVD's block width
    # (K Horner SpMMs with fused epilogues plus the V^T G projection of the all-ones term) ----
    hbm, _, peak_src = measured_peaks()
    K = len(c5)
    csr_bytes = 4 * (g.n + 1) + 4 * g.nnz
    spmm = {}
    for name, dt, es in (("f32", torch.float32, 4), ("bf16", torch.bfloat16, 2)):
        Q = isvd.gaussian(1, g.n, l, device=dev).to(dt)
        Y = torch.empty_like(Q)
        for _ in range(3):
            op.apply(Q, out=Y)
        torch.cuda.nvtx.range_push("roofline_apply")
        apply_ms = float(np.mean(timed_steps(lambda: op.apply(Q, out=Y), 10, flush, stream)))
        torch.cuda.nvtx.range_pop()
        blk = es * g.n * l
        # per SpMM: CSR once, input block once, output block once; axpy operand in K-1 of K
        # steps; plus one read of Q for the projection c = 1^T Q
        alg_bytes = K * (csr_bytes + 2 * blk) + (K - 1) * blk + blk
        spmm[name] = {"ms_per_apply": apply_ms, "algorithmic_bytes": alg_bytes,
                      "gbs": alg_bytes / (apply_ms * 1e-3) / 1e9, "width": l, "spmm_per_apply": K}
        del Q, Y
    kernel = op.tuning()["kernel"]
    traffic = recorded_traffic("f32", kernel)
    f32 = spmm["f32"]
    roofline = {"bound": "hbm", "achieved": f32["gbs"], "peak": hbm, "unit": "GB/s", "frac": f32["gbs"] / hbm,
                "traffic": traffic, "peak_source": peak_src + " (copy, burst)",
                "traffic_gbs": (traffic / (f32["ms_per_apply"] * 1e-3) / 1e9) if traffic else None,
                "traffic_frac": (traffic / (f32["ms_per_apply"] * 1e-3) / 1e9 / hbm) if traffic else None,
                "kernel": "SpMM: one M.Q apply = %d Horner SpMMs (%s kernel) + projection, width %d, FP32"
                          % (K, kernel, l),
                "bf16_frac": spmm["bf16"]["gbs"] / hbm}

    # ---- end to end through the public API, host buffers ----
    e2e = None
    if not args.no_e2e:
        rp_h = torch.from_numpy(g.rowptr).pin_memory()
        ci_h = torch.from_numpy(g.colidx).pin_memory()
        U_h = torch.empty((g.n, k), dtype=torch.float32).pin_memory()
        V_h = torch.empty((g.n, k), dtype=torch.float32).pin_memory()
        S_h = torch.empty(k, dtype=torch.float32).pin_memory()
        e2e_ms = []
        for it in range(1 + min(args.steps, 3)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rp_d = rp_h.to(dev, non_blocking=True)
            ci_d = ci_h.to(dev, non_blocking=True)
            with isvd.Operator(g.n, rp_d, ci_d, coeffs=c5, ones_coeff=-LAM, device=dev) as op2:
                Ud, Sd, Vd, _ = op2.svd(k, p, q, seed=SEED, precision="fp32")
                U_h.copy_(Ud, non_blocking=True)
                V_h.copy_(Vd, non_blocking=True)
                S_h.copy_(Sd, non_blocking=True)
                torch.cuda.synchronize()
            if it > 0:  # the first call warms the allocator pools
                e2e_ms.append((time.perf_counter() - t0) * 1e3)
        e2e = {"value": float(np.mean(e2e_ms)), "unit": "ms",
               "h2d_bytes_per_step": int(rp_h.numel() * 4 + ci_h.numel() * 4),
               "d2h_bytes_per_step": int((U_h.numel() + V_h.numel() + S_h.numel()) * 4),
               "includes": "H2D of the CSR, operator construction (validation, symmetry check, work lists), "
                           "FP32 SVD, D2H of U, S, V"}

    extras = {}
    if not args.no_extras:
        extras["wide"] = wide_section(args, op, g, q, flush, stream)
        extras["batched"] = batched_section(args, flush, stream)
        extras["finetune"] = finetune_section(args, flush, stream)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle

        oracle.build()
        oop = oracle.graph_operator(g, coeffs=c5, ones_coeff=-LAM)
        reps = [oracle_stage(oop, g.n, SAMPLE_WIDTH) for _ in range(2)]
        cpu = {"value": 1e3 * float(np.mean([sum(r) for r in reps])), "unit": "ms", "cores": oracle.num_threads(),
               "kind": "oracle", "sample": stage_description(SAMPLE_WIDTH, 2),
               "estimate_full_svd_ms": stage_estimate_ms(reps, k, p, q, SAMPLE_WIDTH),
               "estimate_note": "not measured: scaled from the stage (products x width, CholeskyQR2 x width^2), "
                                "Rayleigh-Ritz excluded"}
        full = oracle_full_run()
        if full:
            cpu["full_svd_measured_once"] = full

    op.close()
    if rank == 0:
        cfg = config_of(desc, g, k, p, q, world)
        line = {
            "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg,
            "step_ms": step_ms, "construct_ms": construct_ms,
            "mixed": {"iters": q, "ms": mixed_ms, "dtype": "bf16+f32", "speedup_at_same_iters": ms / mixed_ms},
            "equal_error": eq,
            "spmm": spmm, "roofline": roofline, **extras,
            "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
            "gpu_launches": int(kernels_per_step * args.steps) if kernels_per_step > 0 else None,
            "device_status": st,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_case_orth(args):
    """CholeskyQR2 (isvd_orthonormalize) of a seeded N(0,1) block of
    `--rows` x `--width` FP32, one JSON line per repetition set: a fixed case
    for profiling the orthonormalisation kernels (Gram, FP64 Cholesky, Q R^-1)."""
    import torch

    from paper_2111_06312_gb300 import build as libbuild
    from paper_2111_06312_gb300 import isvd, synth

    libbuild.build()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    with isvd.graph_operator(synth.cycle(64), coeffs=[1.0]) as op:
        Q0 = isvd.gaussian(3, args.rows, args.width)
        Q = Q0.clone()
        _, _, info = isvd.orthonormalize(op, Q, want_r=False)
        Qd = Q.double()
        orth = float((Qd.T @ Qd - torch.eye(args.width, dtype=torch.float64, device=Q.device)).abs().max())
        passes = isvd.info_dict(info)["cholqr_passes"]
        stream = torch.cuda.current_stream()
        ms = timed_steps(lambda: (Q.copy_(Q0), isvd.orthonormalize(op, Q, want_r=False)), args.steps, flush, stream)
    print(json.dumps({"case": "orth", "rows": args.rows, "width": args.width, "ms_incl_copy": float(np.median(ms)),
                      "orthogonality": orth, "passes": passes}), flush=True)


def run_case_wide(args):
    """The rank-256 SVD with the paper's l = 2k = 512 (FP32) on the default
    workload, alone (a profiling case): one JSON line with its time per SVD
    and its error; the timed SVDs run inside the NVTX range "wide_svd"."""
    import torch

    from paper_2111_06312_gb300 import build as libbuild
    from paper_2111_06312_gb300 import isvd

    libbuild.build()
    desc, _, _, q = WORKLOADS[args.workload]
    g = load_graph(args.workload)
    k, p = 256, 256
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    with isvd.graph_operator(g, coeffs=coeffs5(), ones_coeff=-LAM) as op:
        U = isvd.new_block(g.n, k)
        V = isvd.new_block(g.n, k)
        S = torch.empty(k, device="cuda")
        info = torch.zeros(4, dtype=torch.int32, device="cuda")
        fn = lambda: op.svd(k, p, q, seed=SEED, U=U, S=S, V=V, info=info, check=False)  # noqa: E731
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("wide_svd")
        ms = timed_steps(fn, args.steps, flush, stream)
        torch.cuda.nvtx.range_pop()
        err = relative_residuals(op, U, S, V)
        st = isvd.info_dict(info)
    print(json.dumps({"case": "wide", "k": k, "oversample": p, "iters": q, "width": k + p, "ms": float(np.mean(ms)),
                      "step_ms": ms, "max_rel_residual": float(err.max()), "device_status": st}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="ne_large")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched and fine-tuning sections")
    ap.add_argument("--case", choices=["svd", "orth", "wide"], default="svd",
                    help="orth: only the CholeskyQR2 of a --rows x --width block; wide: only the rank-256, "
                         "l = 512 SVD (profiling cases)")
    ap.add_argument("--rows", type=int, default=1_000_000)
    ap.add_argument("--width", type=int, default=144)
    args = ap.parse_args()
    if args.case == "orth":
        run_case_orth(args)
    elif args.case == "wide":
        run_case_wide(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
