"""Benchmark: matrix logarithms per second (and TFLOP/s) on GB300.

Default workload (synthetic stand-in for the paper's test sets, which are not
available): a batch of 512 real 256 x 256 matrices A = I + E, E seeded
Gaussian rescaled so ||E||_1 is uniform in [0.2, 5], plus one 4096 x 4096
A = Q T Q^T (T upper triangular, diag log-uniform in [1e-2, 1e2], off-diagonal
Gaussian of standard deviation 0.1/n; with 0.1 literally T is numerically
singular). One step = Algorithm 1 (plan, square roots, graph polynomial, 2^s
scaling) on all 513 matrices, FP64 path.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun, one rank per GPU) every rank runs its own batch (weak
scaling, no collective on the data path); value = matrices of all ranks / the
slowest rank's time. ``--impl reference`` times the CPU oracle on the host
cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "logm matrices/s and TFLOP/s at stated rel. error: mixed/batched vs plain FP64"
UNIT = "TFLOP/s"  # algorithmic FP64-equivalent work of the executed plan per second
COUNT, N = 512, 256
NBIG = 4096
WORKLOAD = ("512 x 256x256 A = I + E (||E||_1 ~ U[0.2, 5]) + one 4096x4096 A = Q T Q^T "
            "(diag T log-uniform [1e-2, 1e2], off-diag N(0, (0.1/n)^2)), seeded, FP64 path")


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def measure_gemm_peak(torch, dev, dtype, clocks_index, n=8192, seconds=2.5, tf32=False):
    """Dense peak measured here, outside the timed region: torch.matmul of two
    n x n matrices (cuBLAS DGEMM for float64, TF32 tensor cores for float32
    with TF32 allowed) back to back for about `seconds`, CUDA events on the
    current stream, nvidia-smi clocks sampled meanwhile. 2 n^3 flops per call."""
    old = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = bool(tf32)
    try:
        g = torch.Generator(device=dev)
        g.manual_seed(7)
        a = torch.randn((n, n), generator=g, device=dev, dtype=dtype)
        b = torch.randn((n, n), generator=g, device=dev, dtype=dtype)
        c = torch.empty((n, n), device=dev, dtype=dtype)
        torch.matmul(a, b, out=c)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b, out=c)
        e1.record()
        torch.cuda.synchronize(dev)
        reps = max(3, int(seconds / max(e0.elapsed_time(e1) * 1e-3, 1e-6)))
        with Clocks(clocks_index) as clk:
            torch.cuda.synchronize(dev)
            e0.record()
            for _ in range(reps):
                torch.matmul(a, b, out=c)
            e1.record()
            torch.cuda.synchronize(dev)
        t = e0.elapsed_time(e1) * 1e-3
        del a, b, c
        return {"tflops": 2.0 * n ** 3 * reps / t / 1e12, "n": n, "reps": reps, "seconds": t,
                "clocks": clk.summary()}
    finally:
        torch.backends.cuda.matmul.allow_tf32 = old


class Clocks:
    """nvidia-smi sampler for the timed region (reads settings only)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            with open(self.path) as f:
                for line in f:
                    parts = [p.strip() for p in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
        except OSError:
            pass
        finally:
            if self.path and os.path.exists(self.path):
                os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def algorithmic_flops(stats: np.ndarray, n: int) -> float:
    """2n^3 per inverse (LU 2/3 n^3 + inversion 4/3 n^3) and per product, 2n^2 per
    estimator matrix-vector product; O(n^2) lin-combs excluded (Sec. 2.2)."""
    st = stats.reshape(-1, 4).astype(np.float64)
    return float(((st[:, 1] + st[:, 2]) * 2.0 * n ** 3 + st[:, 3] * 2.0 * n ** 2).sum())


def oracle_flops(diags, n: int) -> float:
    """Algorithmic work of the oracle's executed plans, counted like the GPU's:
    2n^3 per inversion (the oracle's own count) and per graph product; the
    estimator's 2n^2 matrix-vector products are left out (negligible)."""
    tot = 0.0
    for d in diags:
        products = (d["k"] - 1) + (1 if d["s"] == 0 else 0)
        tot += 2.0 * n ** 3 * (d["n_inv"] + products)
    return tot


def cpu_baseline(A_np, sample: int):
    """The oracle as it stands, on the host cores, on `sample` matrices of the workload."""
    import oracle
    cores = len(os.sched_getaffinity(0))
    mats = [A_np[i] for i in range(sample)]
    oracle.logm_batch(mats[:1], nthreads=cores, reuse_root=1)  # build/load outside the timing
    t0 = time.perf_counter()
    Ls, ds = oracle.logm_batch(mats, nthreads=cores, reuse_root=1)
    dt = time.perf_counter() - t0
    return {"value": oracle_flops(ds, A_np.shape[1]) / dt / 1e12, "unit": UNIT, "matrices_per_s": sample / dt,
            "cores": cores, "kind": "oracle",
            "sample": (f"first {sample} of the {COUNT} 256x256 matrices (same seed), one OpenMP thread per matrix, "
                       "later square roots started from the previous root's Y as the CUDA path does"),
            "seconds": dt}, Ls, ds


def arm_config(count, big, big_n, world, fp64_products="pipe", n=N):
    """The `config` of the JSON line: what the arm runs each step."""
    return {"workload": WORKLOAD if (count == COUNT and n == N and big and big_n == NBIG) else
            f"{count} x {n}x{n} A = I + E (||E||_1 ~ U[0.2, 5])" + (f" + one {big_n}^2 Q T Q^T" if big else "")
            + ", seeded, FP64 path",
            "count": count, "n": n, "n_big": big_n if big else None, "precision": "fp64",
            "fp64_products": fp64_products,
            "l2": "inputs larger than the 129 MB L2; no flush", "parallelism": f"batch-sharded x{world}"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    from paper_2401_10089_gb300 import workloads
    A = workloads.identity_plus(COUNT, N, seed=1)
    sample = args.ref_sample
    cb, Ls, ds = cpu_baseline(A, sample)
    # warm-up / timed steps, each a bounded sample of the workload
    import oracle
    cores = cb["cores"]
    for _ in range(args.warmup):
        oracle.logm_batch([A[0]], nthreads=cores, reuse_root=1)
    times, flops = [], 0.0
    for s in range(args.steps):
        t0 = time.perf_counter()
        _, ds_s = oracle.logm_batch([A[(s * sample + i) % COUNT] for i in range(sample)], nthreads=cores,
                                    reuse_root=1)
        times.append(time.perf_counter() - t0)
        flops += oracle_flops(ds_s, N)
    value = flops / sum(times) / 1e12
    cb["value"] = value
    cb["sample"] = (f"each step the oracle on {sample} of the 512 256x256 matrices (same seed), one OpenMP thread "
                    "per matrix; the 4096x4096 matrix is not run (the oracle would need hours for it)")
    cb["matrices_per_s"] = sample * len(times) / sum(times)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "matrices_per_s": cb["matrices_per_s"],
           "config": arm_config(sample, False, None, world),
           "cpu_baseline": cb, "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-sample", type=int, default=COUNT)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the precision and differentiation forms")
    ap.add_argument("--no-batching", action="store_true", help="skip the 20,000-matrix ragged batching form")
    ap.add_argument("--count", type=int, default=COUNT, help="matrices per rank (smaller for profiling)")
    ap.add_argument("--no-big", action="store_true", help="leave out the 4096 x 4096 matrix")
    ap.add_argument("--big-n", type=int, default=NBIG, help="size of the large matrix (smaller for profiling)")
    ap.add_argument("--n", type=int, default=N, help="size of the batch's matrices (other sizes for profiling)")
    ap.add_argument("--no-peaks", action="store_true", help="skip the FP64 / TF32 peak measurements (profiling)")
    ap.add_argument("--config", type=int, default=None,
                    help="one-block kernel configuration for every size bucket that allows it (profiling; "
                         "default: the tuned table)")
    ap.add_argument("--fp64-products", default="tc_sliced", choices=["tc_sliced", "pipe"],
                    help="FP64 products of the whole-GPU kernel: exact BF16 digit products on the tensor cores "
                         "(default) or FP64 FMAs")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist

    import paper_2401_10089_gb300 as lg
    from paper_2401_10089_gb300 import shard, workloads

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    count, n = args.count, args.n
    if args.config is not None:
        from paper_2401_10089_gb300 import autotune
        lg.set_tuning([args.config if args.config in autotune.CANDIDATES[b] else t
                       for b, t in enumerate(lg.get_tuning())])
    A_np = workloads.identity_plus(count, n, seed=1 + rank)
    A_host = torch.from_numpy(A_np).pin_memory()
    A_dev = A_host.to(dev)
    big = not args.no_big
    if big:
        nbig = args.big_n
        B_host = torch.from_numpy(workloads.triangular_similar(nbig, seed=2 + rank)[None]).pin_memory()
        B_dev = B_host.to(dev)
        stats_b = torch.zeros(4, dtype=torch.int32, device=dev)
    stats = torch.zeros(4 * count, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    # the FP64 path: FP64 products of the whole-GPU kernel (the 4096^2 matrix)
    # formed exactly from BF16 digit products on the tensor cores; the
    # 256 x 256 matrices run on the FP64 pipe (one block per matrix)
    main = {"fp64_products": args.fp64_products}

    def step():
        out = lg.logm_execute(A_dev, stats=stats, **main)
        outb = lg.logm_execute(B_dev, stats=stats_b, **main) if big else None
        return out, outb

    for _ in range(args.warmup):
        step()
    barrier()

    # device-timed region: inputs resident in HBM (268 MB + 134 MB > 129 MB L2)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3 * args.steps)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        barrier()
        e0.record(stream)
        for i in range(args.steps):
            ev[3 * i].record(stream)
            L, s, k, info = lg.logm_execute(A_dev, stats=stats, **main)
            ev[3 * i + 1].record(stream)
            if big:
                Lb, sb, kb, infob = lg.logm_execute(B_dev, stats=stats_b, **main)
            ev[3 * i + 2].record(stream)
        e1.record(stream)
        barrier()
    ms = e0.elapsed_time(e1) / args.steps
    ms_a = sum(ev[3 * i].elapsed_time(ev[3 * i + 1]) for i in range(args.steps)) / args.steps
    ms_b = sum(ev[3 * i + 1].elapsed_time(ev[3 * i + 2]) for i in range(args.steps)) / args.steps
    clocks = clk.summary()
    ms_max = shard.max_over_ranks(ms, device=dev)  # the slowest rank's step

    flops_a = algorithmic_flops(stats.cpu().numpy(), n)
    flops_b = algorithmic_flops(stats_b.cpu().numpy(), args.big_n) if big else 0.0
    info_np = info.cpu().numpy()
    s_np, k_np = s.cpu().numpy(), k.cpu().numpy()
    n_mats = count + (1 if big else 0)

    # end to end through the C-ABI call on host buffers (logm_execute_host: the
    # copy of A to the device, Algorithm 1 and the copies of L, s, k, info back)
    e2e_steps = 0 if args.no_e2e else min(args.steps, 2)
    L_host = torch.empty_like(A_host).pin_memory()
    LB_host = torch.empty_like(B_host).pin_memory() if big else None
    ws_e2e = None
    if e2e_steps:  # one device workspace for both calls, allocated outside the timed region
        need = max(lg.logm_host_workspace_size(A_host), lg.logm_host_workspace_size(B_host) if big else 0)
        ws_e2e = torch.empty(need, dtype=torch.uint8, device=dev)
    if e2e_steps:  # one untimed call first, like the warm-up steps of the device timing
        lg.logm_execute_host(A_host, out=L_host, device=dev, workspace=ws_e2e, **main)
        if big:
            lg.logm_execute_host(B_host, out=LB_host, device=dev, workspace=ws_e2e, **main)
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        lg.logm_execute_host(A_host, out=L_host, device=dev, workspace=ws_e2e, **main)
        if big:
            lg.logm_execute_host(B_host, out=LB_host, device=dev, workspace=ws_e2e, **main)
    e2e_ms = (time.perf_counter() - t0) * 1e3 / e2e_steps if e2e_steps else float("nan")
    e2e_ms = shard.max_over_ranks(e2e_ms, device=dev)
    h2d = A_host.numel() * 8 + (B_host.numel() * 8 if big else 0)
    d2h = h2d + 3 * 4 * n_mats  # L, and s, k, info per matrix

    # precision forms: the same step with the graph products in split precision
    # on the tensor cores (square roots and plan stay FP64); error vs the FP64 result
    # The same step with one option changed: the graph products in split
    # precision on the tensor cores (square roots and plan stay FP64), the
    # product form of the Denman-Beavers iteration, and diagonal balancing;
    # each timed on the same inputs, error against the FP64 result.
    forms = {}
    other = "pipe" if args.fp64_products == "tc_sliced" else "tc_sliced"
    variants = [] if args.no_forms else [("fp64_" + other, {"fp64_products": other}, 1),
                                         ("tf32x3", {"precision": "tf32x3"}, 2), ("bf16x3", {"precision": "bf16x3"}, 2),
                                         ("db_product", {"db_form": "product"}, 1), ("balanced", {"balance": True}, 1)]
    st_fa = torch.zeros(4 * count, dtype=torch.int32, device=dev)
    st_fb = torch.zeros(4, dtype=torch.int32, device=dev)
    for name, vopts, vreps in variants:
        vopts = {**main, **vopts}  # each form changes one option of the FP64 step
        lg.logm_execute(A_dev, **vopts)
        if big:
            lg.logm_execute(B_dev, **vopts)
        barrier()
        fa0, fa1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        fb1 = torch.cuda.Event(enable_timing=True)
        reps = max(1, min(args.steps, vreps))
        fa0.record(stream)
        for _ in range(reps):
            Lp, sp, kp, ip = lg.logm_execute(A_dev, stats=st_fa, **vopts)
        fa1.record(stream)
        if big:
            for _ in range(reps):
                Lpb, _, _, _ = lg.logm_execute(B_dev, stats=st_fb, **vopts)
        fb1.record(stream)
        barrier()
        ms_fa = fa0.elapsed_time(fa1) / reps
        ms_fb = fa1.elapsed_time(fb1) / reps if big else 0.0
        # the split-precision forms run the same plan as the FP64 path (same s, k),
        # but their products are not in the FP64 kernel's tally: count the FP64 run's
        split = "precision" in vopts
        fl_a = flops_a if split else algorithmic_flops(st_fa.cpu().numpy(), n)
        errs_a = ((Lp - L).flatten(1).norm(dim=1) / L.flatten(1).norm(dim=1)).cpu().numpy()
        ent = {"options": vopts,
               "batch256": {"ms": ms_fa, "matrices_per_s": count / (ms_fa * 1e-3),
                            "tflops": fl_a / (ms_fa * 1e-3) / 1e12, "speedup_vs_fp64": ms_a / ms_fa,
                            "rel_err_vs_fp64": {"max": float(errs_a.max()), "median": float(np.median(errs_a))}}}
        if name in ("db_product",):
            sa = st_fa.cpu().numpy().reshape(-1, 4).sum(axis=0)
            ent["batch256"]["work"] = {"db_iterations": int(sa[0]), "inverses": int(sa[1]), "products": int(sa[2])}
        if big:
            fl_b = flops_b if split else algorithmic_flops(st_fb.cpu().numpy(), args.big_n)
            eb = float(((Lpb - Lb).norm() / Lb.norm()).item())
            ent["n4096"] = {"ms": ms_fb, "tflops": fl_b / (ms_fb * 1e-3) / 1e12, "speedup_vs_fp64": ms_b / ms_fb,
                            "rel_err_vs_fp64": eb}
            ent["step"] = {"ms": ms_fa + ms_fb, "tflops": (fl_a + fl_b) / ((ms_fa + ms_fb) * 1e-3) / 1e12,
                           "speedup_vs_fp64": ms / (ms_fa + ms_fb)}
        forms[name] = ent

    # the opt-in k = 6 order (k_max = 6, one-block-per-matrix kernels, n <= 256):
    # the batch part of the same step, against the k_max = 5 run above
    if not args.no_forms and n <= 256:
        vopts = {**main, "k_max": 6}
        try:
            lg.logm_execute(A_dev, **vopts)
            barrier()
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = max(1, args.steps)
            f0.record(stream)
            for _ in range(reps):
                L6, s6, k6, i6 = lg.logm_execute(A_dev, stats=st_fa, **vopts)
            f1.record(stream)
            barrier()
            ms6 = f0.elapsed_time(f1) / reps
            e6 = ((L6 - L).flatten(1).norm(dim=1) / L.flatten(1).norm(dim=1)).cpu().numpy()
            sa = st_fa.cpu().numpy().reshape(-1, 4).sum(axis=0)
            forms["k_max6"] = {
                "options": vopts,
                "note": "k_max = 6 is taken by the one-block-per-matrix kernels only (n <= 256)",
                "batch256": {"ms": ms6, "matrices_per_s": count / (ms6 * 1e-3),
                             "tflops": algorithmic_flops(st_fa.cpu().numpy(), n) / (ms6 * 1e-3) / 1e12,
                             "speedup_vs_fp64": ms_a / ms6,
                             "rel_err_vs_fp64": {"max": float(e6.max()), "median": float(np.median(e6))},
                             "s_hist": np.bincount(s6.cpu().numpy()).tolist(),
                             "k_hist": np.bincount(k6.cpu().numpy(), minlength=7).tolist(),
                             "info_nonzero": int((i6.cpu().numpy() != 0).sum()),
                             "work": {"db_iterations": int(sa[0]), "inverses": int(sa[1]), "products": int(sa[2])}}}
        except RuntimeError as e:  # a refused call is recorded, not fatal to the step's own line
            forms["k_max6"] = {"options": vopts, "error": str(e)}

    # differentiation form: 1024 SPD 64 x 64 (lambda log-uniform in [1e-2, 1e2]),
    # loss = sum(W o log A): forward with checkpoints, then the hand-written adjoint
    if not args.no_forms:
        Ad = torch.from_numpy(workloads.spd(1024, 64, seed=91 + rank, lo=1e-2, hi=1e2)).to(dev)
        Wd = torch.from_numpy(np.random.default_rng(92 + rank).standard_normal((1024, 64, 64))).to(dev)
        st_d = torch.zeros(4 * 1024, dtype=torch.int32, device=dev)
        for _ in range(2):
            Ld, _, _, _, cd = lg.logm_execute(Ad, with_ctx=True, stats=st_d)
            dAd, bi = lg.logm_backward(Ad, cd, Wd)
        barrier()
        d0, d1, d2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        reps = max(1, args.steps)
        fwd_ms = bwd_ms = 0.0
        for _ in range(reps):
            d0.record(stream)
            Ld, _, _, _, cd = lg.logm_execute(Ad, with_ctx=True, stats=st_d)
            d1.record(stream)
            dAd, bi = lg.logm_backward(Ad, cd, Wd)
            d2.record(stream)
            barrier()
            fwd_ms += d0.elapsed_time(d1) / reps
            bwd_ms += d1.elapsed_time(d2) / reps
        forms["differentiation"] = {
            "workload": "1024 SPD 64x64, lambda log-uniform [1e-2, 1e2], loss = sum(W o log A), FP64",
            "forward_ms": fwd_ms, "backward_ms": bwd_ms, "backward_over_forward": bwd_ms / fwd_ms,
            "matrices_per_s_fwd_bwd": 1024 / ((fwd_ms + bwd_ms) * 1e-3),
            "forward_tflops": algorithmic_flops(st_d.cpu().numpy(), 64) / (fwd_ms * 1e-3) / 1e12,
            "backward_info_nonzero": int((bi.cpu().numpy() != 0).sum())}
    # batching form: 20,000 SPD matrices, n uniform in {4, 8, ..., 256}, lambda
    # log-uniform in [1e-3, 1e3], FP32 storage, one logm_execute call (TF32x3 and
    # FP64 graph products); the inputs are drawn on the device
    if not args.no_batching and not args.no_forms:
        vals_d, ns_d, offs_d = workloads.ragged_spd_device(20000, dev, seed=4 + rank)
        ns_r = ns_d.cpu().numpy()
        R = lg.Ragged(vals_d, ns_d, offs_d, 256)
        st_r = torch.zeros(4 * 20000, dtype=torch.int32, device=dev)
        entry = {}
        for prec in ("tf32x3", "fp64"):
            lg.logm_execute(R, precision=prec, stats=st_r)
            barrier()
            r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            r0.record(stream)
            Lr_, sr_, kr_, ir_ = lg.logm_execute(R, precision=prec, stats=st_r)
            r1.record(stream)
            barrier()
            ms_r = r0.elapsed_time(r1)
            w = st_r.cpu().numpy().reshape(-1, 4).astype(np.float64)
            fl = float(((w[:, 1] + w[:, 2]) * 2.0 * ns_r.astype(np.float64) ** 3
                        + w[:, 3] * 2.0 * ns_r.astype(np.float64) ** 2).sum())
            entry[prec] = {"ms": ms_r, "matrices_per_s": 20000 / (ms_r * 1e-3), "tflops": fl / (ms_r * 1e-3) / 1e12,
                           "info_nonzero": int((ir_.cpu().numpy() != 0).sum()),
                           "s_hist": np.bincount(sr_.cpu().numpy()).tolist()}
        entry["workload"] = ("20000 SPD, n uniform over {4, 8, 16, 32, 64, 128, 256}, lambda log-uniform [1e-3, 1e3], FP32 storage, "
                             "one call (persistent FP64 stage + tcgen05 graph stage)")
        entry["speedup_tf32x3_vs_fp64"] = entry["fp64"]["ms"] / entry["tf32x3"]["ms"]
        forms["batching"] = entry

    if rank == 0:
        # FP64 and TF32 dense peaks measured on this GPU (cuBLAS GEMM loops of a
        # few seconds, outside the timed region, clocks sampled meanwhile)
        if args.no_peaks:  # profiling runs: no reference GEMM loops (the fractions are then NaN)
            peaks = {"fp64": {"tflops": float("nan"), "seconds": 0.0}, "tf32": {"tflops": float("nan")}}
        else:
            peaks = {"fp64": measure_gemm_peak(torch, dev, torch.float64, local),
                     "tf32": measure_gemm_peak(torch, dev, torch.float32, local, tf32=True)}
        peak = peak_a = peaks["fp64"]["tflops"]
        peak_note = ("FP64 dense of measured: cuBLAS DGEMM 8192^3 (torch.matmul float64) back to back for "
                     f"{peaks['fp64']['seconds']:.1f} s in this run")
        bound = "tensor"
        # dominant kernel: the whole-GPU 4096 kernel
        if big:
            ach = flops_b / (ms_b * 1e-3) / 1e12
            kname, fpl = "k_logm_large<execute> (cooperative, whole GPU on the 4096 matrix)", flops_b
            if args.fp64_products == "tc_sliced":
                # its FP64 products run on the BF16 tensor cores as 36 exact digit-pair
                # products each (8 digits per operand, pairs i + j <= 9): the ceiling of
                # that form is the sustained BF16 peak / 36
                pk = measured_peaks()
                bf16 = pk.get("bf16_tflops_sustained", 1700.0)
                peak = bf16 / 36.0
                peak_note = (f"FP64-equivalent ceiling of the 8-digit BF16 form: {'measured' if pk else 'fallback'} "
                             f"sustained BF16 {bf16:.1f} TFLOP/s / 36 digit-pair products per FP64 product "
                             f"({'of measured' if pk else 'of fallback'}); against the measured FP64 DGEMM peak "
                             f"{peak_a:.3f} TFLOP/s the kernel runs at {ach / peak_a:.2f}x")
        else:
            ach = flops_a / (ms_a * 1e-3) / 1e12
            kname, fpl = "k_logm_small<execute> (persistent, one block per matrix)", flops_a
        # DRAM bytes of the dominant kernel from ncu (dram__bytes_read.sum +
        # dram__bytes_write.sum). The 4096^2 launch is too long to capture; its
        # 2048^2 case (same plan: 27 iterations, 45 inversions, 4 products) moved
        # 96.62 GB, mostly the working matrix written back by every rank-32
        # update, which scales with n^3: x 8 for one 4096^2 launch.
        traffic, traffic_note = None, "not captured for this configuration"
        if big and args.big_n == NBIG and args.fp64_products == "pipe":
            traffic = 8 * (7.813095e9 + 88.806196e9)
            traffic_note = ("bytes per launch: 8 x the DRAM bytes ncu measured on the 2048^2 case of the same "
                            "kernel and plan (traffic grows with n^3); far below HBM bandwidth, FP64-pipe bound")
        elif big and args.big_n == NBIG and args.fp64_products == "tc_sliced":
            # ncu on the 2048^2 case of the tensor-core form (same plan): 20.66 GB
            # read + 34.37 GB written, mostly W read and written once per
            # 128-column super-panel and the digit tiles, both growing with n^3
            traffic = 8 * (20.661627e9 + 34.370699e9)
            traffic_note = ("bytes per launch: 8 x the DRAM bytes ncu measured on the 2048^2 case of the same "
                            "kernel and plan (traffic grows with n^3); far below HBM bandwidth, latency and "
                            "barrier bound (profiles/k_logm_large_tc_sliced_2048.md)")
        parts = {"batch256": {"ms": ms_a, "matrices_per_s": count / (ms_a * 1e-3),
                              "tflops": flops_a / (ms_a * 1e-3) / 1e12,
                              "frac": flops_a / (ms_a * 1e-3) / 1e12 / peak_a,
                              "peak_note": "of measured FP64 DGEMM peak (FP64 pipe, one block per matrix)",
                              "s_hist": np.bincount(s_np).tolist(), "k_hist": np.bincount(k_np, minlength=6).tolist(),
                              "info_nonzero": int((info_np != 0).sum()),
                              "work": dict(zip(("db_iterations", "inverses", "products"),
                                               stats.cpu().numpy().reshape(-1, 4).sum(axis=0)[:3].tolist()))}}
        if big:
            parts["n4096"] = {"ms": ms_b, "tflops": ach, "frac": ach / peak, "s": int(sb[0]), "k": int(kb[0]),
                              "info": int(infob[0]), "work": stats_b.cpu().numpy().tolist()}
        out = {
            "metric": METRIC, "value": (flops_a + flops_b) * world / (ms_max * 1e-3) / 1e12, "unit": UNIT,
            "matrices_per_s": n_mats * world / (ms_max * 1e-3), "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": arm_config(count, big, args.big_n, world, args.fp64_products, n),
            "parts": parts,
            "forms": forms,
            "roofline": {"bound": bound, "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                         "frac": ach / peak, "traffic": traffic, "traffic_note": traffic_note,
                         "peak_note": peak_note,
                         "kernel": kname, "flops_per_launch": fpl},
            "peaks_measured": peaks,
            "e2e": {"value": (flops_a + flops_b) * world / (e2e_ms * 1e-3) / 1e12 if e2e_steps else None,
                    "unit": UNIT, "matrices_per_s": n_mats * world / (e2e_ms * 1e-3) if e2e_steps else None,
                    "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": (4 + (1 if big else 0)) * args.steps,  # 3 queue-order kernels + persistent + cooperative
            "clocks": clocks,
        }
        if not args.no_cpu_baseline:
            cb, Ls, ds = cpu_baseline(A_np, min(args.ref_sample, count))
            Lg = L.cpu().numpy()
            errs = [np.linalg.norm(Lg[i] - Ls[i]) / np.linalg.norm(Ls[i]) for i in range(len(Ls))
                    if (ds[i]["s"], ds[i]["k"]) == (int(s_np[i]), int(k_np[i]))]
            cb["sample"] += "; the 4096 matrix is not run (the oracle would need hours for it)"
            out["cpu_baseline"] = cb
            out["rel_err_vs_oracle"] = {"max": float(max(errs)) if errs else None, "matrices": len(errs)}
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
