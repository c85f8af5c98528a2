"""Benchmark: time to a rank-k implicit SVD on one GB300, plus the SpMM
roofline.

Workload (default): the large network-embedding operator
M = sum_{k=1..5} c_k T^k - 0.05 11^T, c_k = (6-k)/15, T = D^-1 A on a seeded
Chung-Lu power-law graph (n = 10^6, 2x10^7 directed edges, max degree ~4x10^4),
rank 128, oversample 16, 6 power iterations (Alg. 1).  A step is one whole
isvd_svd (CUDA-graph replay) with the operator and inputs resident in HBM.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32|mixed]
  python bench.py --impl reference      # the FP64 CPU oracle, bounded sample

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
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time to rank-k implicit SVD & SpMM HBM GB/s, mixed vs FP32 at equal error"
LAM = 0.05


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


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d.get("bf16_tflops", 1900.0)), "measured"
    return 6800.0, 1900.0, "fallback"


KERNEL_SOURCES = {
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

def oracle_sample(g, k, p, q, b_sample=32):
    """Time the FP64 oracle on a bounded sample of the same workload and scale
    to one whole SVD: one forward and one transposed product M G, M^T G at
    block width b_sample (cost proportional to the width) and one CholeskyQR2
    of an n x b_sample block (cost proportional to the width squared)."""
    import oracle

    oracle.build()
    op = oracle.graph_operator(g, coeffs=coeffs5(), ones_coeff=-LAM)
    rng = np.random.default_rng(0)
    G = rng.standard_normal((g.n, b_sample))
    t0 = time.perf_counter()
    Y = op.apply(G)
    t1 = time.perf_counter()
    op.apply(Y, transpose=True)
    t2 = time.perf_counter()
    oracle.cholqr2(Y)
    t3 = time.perf_counter()
    l = k + p
    applies_fwd = q + 1
    applies_t = q + 1
    orths = 2 * q + 2
    scale_w = l / b_sample
    est = (applies_fwd * (t1 - t0) + applies_t * (t2 - t1)) * scale_w + orths * (t3 - t2) * scale_w ** 2
    sample = (f"one M.G and one M^T.G (K=5 sparse products each) at width {b_sample} and one CholeskyQR2 of an "
              f"n x {b_sample} block on the full graph ({t3 - t0:.1f} s); scaled to {applies_fwd}+{applies_t} "
              f"products at width {l} (x{scale_w:.1f}) and {orths} CholeskyQR2 (x{scale_w ** 2:.0f}); "
              f"Rayleigh-Ritz not included")
    return est * 1e3, sample, oracle.num_threads(), t3 - t0


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    desc, k, p, q = WORKLOADS[args.workload]
    g = load_graph(args.workload)
    per_step = []
    sample = cores = None
    # each step is a bounded sample (~10-30 s of CPU work); at most 3 steps
    for _ in range(max(1, min(args.steps, 3))):
        ms, sample, cores, _ = oracle_sample(g, k, p, q)
        per_step.append(ms)
    value = float(np.mean(per_step))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "ms", "n_gpus": args.gpus,
            "steps": len(per_step), "warmup": 0, "ms_per_step": value, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "n": g.n, "nnz": g.nnz, "k": k, "oversample": p, "iters": q},
            "cpu_baseline": {"value": value, "unit": "ms", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
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

    def step():
        op.svd(k, p, q, seed=20211106312, precision=args.precision, U=U, S=S, V=V, info=info, check=False)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    st = isvd.info_dict(info)
    if st["status"] != "OK":
        raise RuntimeError(f"device status {st}")

    clocks = ClockSampler(torch.cuda.current_device())
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    evs = []
    torch.cuda.nvtx.range_push("timed_steps")
    for _ in range(args.steps):
        flush.zero_()  # untimed: leaves no operand of the next step in L2
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    ms = slowest_rank_ms(float(np.mean(step_ms)), world, dev)
    kernels_per_step = op.graph_kernel_nodes()

    # ---- SpMM step roofline: one M.Q apply of this operator at the SVD's block width ----
    # (K Horner SpMMs with fused epilogues plus the V^T G projection of the all-ones term),
    # in the storage type of the power iterations
    hbm, _, peak_src = measured_peaks()
    apply_dtype = torch.float32 if args.precision == "fp32" else torch.bfloat16
    es = 4 if apply_dtype == torch.float32 else 2
    Q = isvd.gaussian(1, g.n, l, device=dev).to(apply_dtype)
    Y = torch.empty_like(Q)
    for _ in range(3):
        op.apply(Q, out=Y)
    spmm_t = []
    for _ in range(10):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("roofline_apply")
        a.record(stream)
        op.apply(Q, out=Y)
        b.record(stream)
        torch.cuda.nvtx.range_pop()
        spmm_t.append((a, b))
    torch.cuda.synchronize()
    apply_ms = float(np.mean([a.elapsed_time(b) for a, b in spmm_t]))
    K = len(c5)
    csr_bytes = 4 * (g.n + 1) + 4 * g.nnz
    blk = es * g.n * l
    # per SpMM: CSR once, input block once, output block once; axpy operand in K-1 of K
    # steps; plus one read of Q for the projection c = 1^T Q
    alg_bytes = K * (csr_bytes + 2 * blk) + (K - 1) * blk + blk
    achieved = alg_bytes / (apply_ms * 1e-3) / 1e9
    kernel = op.tuning()["kernel"]
    traffic = recorded_traffic("f32" if es == 4 else "bf16", kernel)
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
                Ud, Sd, Vd, _ = op2.svd(k, p, q, seed=20211106312, precision=args.precision)
                U_h.copy_(Ud, non_blocking=True)
                V_h.copy_(Vd, non_blocking=True)
                S_h.copy_(Sd, non_blocking=True)
                torch.cuda.synchronize()
            if it > 0:  # the first call also compiles nothing but warms allocator pools
                e2e_ms.append((time.perf_counter() - t0) * 1e3)
        e2e = {"value": float(np.mean(e2e_ms)), "unit": "ms",
               "h2d_bytes_per_step": int(rp_h.numel() * 4 + ci_h.numel() * 4),
               "d2h_bytes_per_step": int((U_h.numel() + V_h.numel() + S_h.numel()) * 4),
               "includes": "H2D of the CSR, operator construction (validation, symmetry check, work lists), "
                           "SVD, D2H of U, S, V"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cms, sample, cores, _ = oracle_sample(g, k, p, q)
        cpu = {"value": cms, "unit": "ms", "cores": cores, "kind": "oracle", "sample": sample}

    op.close()
    if rank == 0:
        line = {
            "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "bf16+f32",
            "data": "synthetic",
            "config": {"workload": desc, "n": g.n, "nnz": g.nnz, "k": k, "oversample": p, "iters": q,
                       "precision": args.precision, "parallelism": f"replicas x{world}",
                       "l2": "256 MB buffer written between steps (untimed); per-step working set > 3 GB",
                       "construct_ms": construct_ms},
            "step_ms": step_ms,
            "spmm": {"ms_per_apply": apply_ms, "algorithmic_bytes": alg_bytes, "gbs": achieved, "width": l,
                     "spmm_per_apply": K, "storage": "f32" if es == 4 else "bf16"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": traffic, "peak_source": peak_src + " (copy, burst)",
                         "traffic_gbs": (traffic / (apply_ms * 1e-3) / 1e9) if traffic else None,
                         "traffic_frac": (traffic / (apply_ms * 1e-3) / 1e9 / hbm) if traffic else None,
                         "kernel": "SpMM: one M.Q apply = %d Horner SpMMs (%s kernel) + projection, width %d"
                                   % (K, kernel, l)},
            "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
            "gpu_launches": int(kernels_per_step * args.steps) if kernels_per_step > 0 else None,
            "device_status": st,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp32", "mixed"], default="fp32")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="ne_large")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
