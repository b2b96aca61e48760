"""Benchmark of the CSRC product y = A x and y = A^T x on one GB300 (or N replicas).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]

One step is one y = A x and one y = A^T x (Fig. 2(a), Section 5) with the
library's window strategy: a band-kernel launch and an accumulation launch for
each product. The default workload is the Q1 hexahedral 27-point matrix on 96^3
nodes with 3 DOFs per node (n = 2,654,208, nnz = 210,542,904), RCM ordered,
FP64 values, synthetic and seeded. Its 2.15 GB per product is far larger than
L2 (129 MB), so no L2 flush is needed between steps.

The metric is GB/s over the CSRC working set (ia + ja + al + au + ad + x + y,
10 nnz + 18 n + 4 bytes per FP64 product, Table 1's ws) and its fraction of
the measured HBM bandwidth. Rank 0 prints one JSON line.

--impl reference times the CPU oracle (plain single-threaded FP64 C) on a
leading principal submatrix of the same matrix, sized so the run ends within a
few minutes, with the same metric and unit.

N > 1 (torchrun, one process per GPU) runs independent replicas: the product
has no exchange step on one matrix per GPU, so value = the bytes all ranks
processed / the slowest rank's time ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "CSRC SpMV GB/s and % of HBM roofline (FP64 vs mixed-prec batched, 1 GB300)"
FALLBACK_HBM_GBS = 6800.0
KERNEL_SOURCES = ["owner.cuh", "owner.cu", "internal.h"]


# ----------------------------------------------------------------------------- helpers
def model_bytes(n: int, pairs: int, value_bytes: int = 8, vec_bytes: int = 8) -> int:
    """ia + ja + al + au + ad + x + y of one product (Table 1's ws for FP64)."""
    return 4 * (n + 1) + 4 * pairs + 2 * value_bytes * pairs + value_bytes * n + 2 * vec_bytes * n


def flops(n: int, pairs: int) -> int:
    """2 nnz - n (Section 4.1): n multiplies on the diagonal and 2 multiply-adds per pair."""
    return n + 4 * pairs


def measured_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_sha() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1003_0952_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(workload: str):
    """DRAM bytes per launch of the product kernel from the committed ncu summary,
    or None when the kernel sources changed since that capture."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d.get(workload)
        if e and e.get("kernel_source_sha") == kernel_source_sha():
            return int(e["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi clock and throttle samples taken during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                p = [v.strip() for v in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max(v: float, world: int, device) -> float:
    if world <= 1:
        return v
    import torch
    import torch.distributed as dist

    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world: int, bytes_per_step: float, steps: int, seconds: float) -> float:
    """Whole-job GB/s of `world` replicas that each moved bytes_per_step per step for `steps`
    steps, timed by the slowest rank (seconds = max over ranks)."""
    return world * bytes_per_step * steps / seconds / 1e9


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


# ----------------------------------------------------------------------------- workload
def build_workload(name: str):
    import fe_inputs as fe

    builder, xseed = fe.CONFIGS[name]
    m = builder()
    x = fe.source_vector(m.n, xseed)
    return m, x


def describe(name: str, m) -> dict:
    return {"workload": f"{name}: " + {
        "q1v_96": "Q1 hex 27-point stencil, 96^3 nodes x 3 DOF (3x3 blocks), random then RCM order, "
                  "al != au U[-1,1], FP64 values, y = A x and y = A^T x",
        "q1s_96": "Q1 hex 27-point stencil, 96^3 nodes, scalar, random then RCM order, FP64, y = A x and y = A^T x",
        "q1v_64": "Q1 hex 27-point stencil, 64^3 nodes x 3 DOF (3x3 blocks), random then RCM order, FP64, "
                  "y = A x and y = A^T x (profiling case)",
        "p1_100x100": "P1 triangles on a 100x100 node grid, natural order, FP64, y = A x and y = A^T x",
    }.get(name, name), "n": int(m.n), "nnz": int(m.nnz), "pairs": int(m.pairs),
        "strategy": "window (shared-memory windows + deterministic accumulation)",
        "l2": "inputs larger than L2 (129 MB): no flush" if model_bytes(m.n, m.pairs) > 129e6
        else "fits in L2: no flush, L2-resident figure"}


# ----------------------------------------------------------------------------- CPU oracle timing
def oracle_gbs(m, x, budget_s: float, max_rows: int | None = None):
    """Time the oracle's Fig. 2(a) product (and its transpose) on the leading
    max_rows x max_rows principal submatrix, repeating until budget_s passes.
    Returns (GB/s, products, seconds, rows, y, y_t): the last A x and A^T x."""
    import oracle

    c = oracle.from_matrix(m)
    rows = m.n if max_rows is None else min(m.n, max_rows)
    if rows < m.n:
        c = oracle.CSRC(rows, c.ia[:rows + 1].copy(), c.ja[:int(c.ia[rows])], c.al[:int(c.ia[rows])],
                        c.au[:int(c.ia[rows])], c.ad[:rows])
    xs = x[:rows]
    nbytes = model_bytes(rows, c.pairs)
    done, t0 = 0, time.perf_counter()
    while True:
        y = oracle.csrc_spmv(c, xs)
        yt = oracle.csrc_spmv_t(c, xs)
        done += 2
        el = time.perf_counter() - t0
        if el >= budget_s:
            break
    return nbytes * done / el / 1e9, done, el, rows, y, yt


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    m, x = build_workload(args.workload)
    # calibrate: one product pair on a sample, then size each step to fit the budget
    total_budget = 120.0
    per_step = total_budget / max(1, args.steps + args.warmup)
    _, _, el, rows, _, _ = oracle_gbs(m, x, 0.0, max_rows=min(m.n, 200_000))
    rows_step = int(max(1000, min(m.n, rows * per_step / max(el, 1e-6))))
    import oracle

    c = oracle.from_matrix(m)
    c = oracle.CSRC(rows_step, c.ia[:rows_step + 1].copy(), c.ja[:int(c.ia[rows_step])],
                    c.al[:int(c.ia[rows_step])], c.au[:int(c.ia[rows_step])], c.ad[:rows_step])
    xs = x[:rows_step]
    for _ in range(args.warmup):
        oracle.csrc_spmv(c, xs)
        oracle.csrc_spmv_t(c, xs)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.csrc_spmv(c, xs)
        oracle.csrc_spmv_t(c, xs)
    el = time.perf_counter() - t0
    nbytes = 2 * model_bytes(rows_step, c.pairs)
    gbs = nbytes * args.steps / el / 1e9
    cfg = describe(args.workload, m)
    sample = (f"leading {rows_step}x{rows_step} principal submatrix ({c.pairs} pairs) of the workload, "
              f"y = A x and y = A^T x per step")
    line = {"impl": "reference", "metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": cfg,
            "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- GPU arm
def run_ours(args):
    import torch

    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    import paper_1003_0952_gb300 as cs

    m, x_np = build_workload(args.workload)
    strategy = cs.STRATEGIES[args.strategy]
    h = cs.csrc_create_from_csr(m.n, m.row_ptr, m.col, m.val, cs.STORAGE[args.storage])
    try:
        cs.csrc_partition(h, 0)
        if args.strategy == "color":
            cs.csrc_color(h, 12345)
        info = cs.csrc_get_info(h)
        stream = torch.cuda.current_stream()
        sptr = stream.cuda_stream
        vdt = torch.float64 if args.storage == "f64" else torch.float32
        x = torch.from_numpy(x_np).to(dev).to(vdt)
        y = torch.empty_like(x)
        yt = torch.empty_like(x)

        def step():
            cs.csrc_spmv(h, x, y, strategy, sptr)
            cs.csrc_spmv_t(h, x, yt, strategy, sptr)

        for _ in range(max(3, args.warmup)):
            step()
        torch.cuda.synchronize()
        st = cs.csrc_get_last_device_error(h)
        if st != cs.CSRC_OK:
            raise RuntimeError(f"device status after warm-up: {cs.csrc_status_string(st)}")

        # ---- timed region: device time with CUDA events on the launch stream
        clocks = ClockSampler(torch.cuda.current_device())
        clocks.start()
        time.sleep(0.3)
        cs.csrc_set_profiling(h, True)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        barrier(world)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        ms_local = ev0.elapsed_time(ev1)
        ktimes = cs.csrc_get_kernel_times(h)
        cs.csrc_set_profiling(h, False)
        clk = clocks.stop()
        ms = reduce_max(ms_local, world, dev)

        # ---- end to end through the public API with pinned host buffers
        xh = torch.from_numpy(x_np).to(vdt).pin_memory()
        yh = torch.empty_like(xh).pin_memory()
        yth = torch.empty_like(xh).pin_memory()

        def step_host():
            cs.csrc_spmv(h, xh, yh, strategy, sptr)
            cs.csrc_spmv_t(h, xh, yth, strategy, sptr)
            stream.synchronize()

        for _ in range(3):
            step_host()
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            step_host()
        e2e_s = reduce_max(time.perf_counter() - t0, world, dev)
        barrier(world)
        # the results of the last timed step, for the check against the oracle
        y_last = y.double().cpu().numpy()
        yt_last = yt.double().cpu().numpy()
        st = cs.csrc_get_last_device_error(h)
        if st != cs.CSRC_OK:
            raise RuntimeError(f"device status after the timed steps: {cs.csrc_status_string(st)}")
    finally:
        cs.csrc_destroy(h)

    nbytes_step = 2 * int(info["model_bytes"])
    value = replica_throughput(world, nbytes_step, args.steps, ms * 1e-3)
    e2e_value = replica_throughput(world, nbytes_step, args.steps, e2e_s)
    peak, peak_src = measured_hbm()
    nprod, ms_prod = ktimes["product"]
    # algorithmic bytes of one product-kernel launch: the CSRC working set (Table 1's ws) plus
    # the spill writes of the bands (the accumulation's traffic, counted explicitly); the colour
    # product writes y in place and spills nothing
    vec_bytes = 8 if args.storage == "f64" else 4
    colour = args.strategy == "color"
    kbytes = int(info["model_bytes"]) + (0 if colour else vec_bytes * int(info["spill_entries"]))
    launch_ms = ms_prod / max(nprod, 1)
    achieved = kbytes / (launch_ms * 1e-3) / 1e9 if nprod else None
    launches = sum(v[0] for v in ktimes.values())
    if rank != 0:
        return 0
    cfg = describe(args.workload, m)
    window = args.strategy in ("window", "auto") and info["tuned_strategy"] in (0, 1)
    arith = ("FP64 pipe: one FP64 multiply-add per stored value" if args.storage == "f64" and
             (window or info["arith"] == 1) else {0: "double-float (FP32 pairs)", 1: "FP64 pipe", 2: "FP32"}[info["arith"]])
    if colour and args.storage == "f64":
        arith = "FP64 pipe"
    cfg.update({"nbands": info["nbands"], "spill_entries": info["spill_entries"], "arith": arith,
                "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"})
    if args.strategy != "window":
        cfg["strategy"] = {"auto": "auto (the handle's tuned strategy)", "window_atomic": "window-atomic (stream order)",
                           "atomic": "atomic (stream order)",
                           "color": f"colour ({info['ncolors']} classes, one cooperative launch)"}[args.strategy]
    kname = ("owner_kernel (window strategy: target-sorted entry lists, one lane per window row)" if window
             else "color_persistent_kernel (colour strategy: all classes in one cooperative launch)" if colour
             else "band_kernel (stream-order strategy)")
    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.storage if args.storage == "f64" else f"{args.storage} storage, f32 compute",
        "data": "synthetic (seeded FE pattern and values)",
        "config": cfg,
        "gflops": world * flops(m.n, m.pairs) * 2 * args.steps / (ms * 1e-3) / 1e9,
        "pct_hbm_roofline": value / world / peak,
        "e2e": {"value": e2e_value, "unit": "GB/s", "h2d_bytes_per_step": 2 * xh.element_size() * m.n,
                "d2h_bytes_per_step": 2 * xh.element_size() * m.n},
        "roofline": {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": (achieved / peak) if achieved else None,
                     "peak_source": f"{peak_src} hbm_gbs", "traffic": ncu_traffic(args.workload) if window else None,
                     "algorithmic_bytes_per_launch": kbytes, "launch_ms": launch_ms,
                     # what the window strategy's kernel itself moves (entry slots and values, list
                     # metadata, x of every window slot, y and spill writes), for comparison
                     "kernel_bytes_per_launch": int(info["list_bytes"]) if window else None},
        "kernels": {k: {"launches": v[0], "ms": v[1]} for k, v in ktimes.items()},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if world == 1 and not args.no_cpu_baseline:
        import oracle

        xs64 = x.double().cpu().numpy() if args.storage != "f64" else x_np
        gbs, done, el, rows, yref, ytref = oracle_gbs(m, xs64, args.cpu_seconds)
        tol = {"f64": 1e-12, "f32": 1e-5, "bf16": 1e-2}[args.storage]
        err = {"A x": oracle.max_rel_err(m, xs64, y_last, yref),
               "A^T x": oracle.max_rel_err(m, xs64, yt_last, ytref, transpose=True)}
        line["cpu_baseline"] = {"value": gbs, "unit": "GB/s", "cores": 1, "kind": "oracle",
                                "sample": f"{done} full products (y = A x and y = A^T x alternating) of the "
                                          f"workload in {el:.1f} s, single-threaded FP64 C"}
        # the same oracle products check the timed steps' results: max_i |y_i - yref_i| / sum_j |a_ij||x_j|
        line["max_rel_err"] = {**err, "tolerance": tol, "ok": all(v <= tol for v in err.values())}
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


# ----------------------------------------------------------------------------- suite of every configuration
def _events_ms(fn, iters: int, runs: int = 3) -> float:
    """Median over `runs` runs of the mean device time of `iters` back-to-back calls of fn
    (CUDA events on the current stream, after three warm-up calls)."""
    import torch

    for _ in range(3):
        fn()
    torch.cuda.synchronize()
    times = []
    for _ in range(runs):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(iters):
            fn()
        b.record()
        b.synchronize()
        times.append(a.elapsed_time(b) / iters)
    return statistics.median(times)


def _oracle_leg(fn, nbytes: int):
    """CPU baseline of one suite row: the oracle's products timed once on the host (one
    core), returned with their results so that the row's GPU results can be checked."""
    t0 = time.perf_counter()
    out = fn()
    el = time.perf_counter() - t0
    return out, {"value": nbytes / el / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle", "seconds": el}


SUITE_TOL = {"f64": 1e-12, "f32": 1e-5, "bf16": 1e-2}


def run_suite(args):
    """One JSON line per configuration row of the contract (C1-C5) and of the next steps
    (N1-N4). Device time: median of three runs of --suite-iters calls, CUDA events on the
    launch stream. Every row carries a CPU baseline (the oracle timed on the host) and the
    max relative error of the row's GPU results against those oracle results. Inputs are
    larger than L2 except C1's, which is timed both L2-resident and over rotating copies."""
    import torch

    import fe_inputs as fe
    import oracle
    import paper_1003_0952_gb300 as cs

    torch.cuda.set_device(0)
    peak, _ = measured_hbm()
    st = torch.cuda.current_stream()
    sptr = st.cuda_stream

    def emit(d):
        d["frac_of_measured_hbm"] = d["GB/s"] / peak if "GB/s" in d else None
        print(json.dumps(d), flush=True)

    def gpu(t):
        return t.double().cpu().numpy()

    def spmv_rows(name, m, storages, strategies, colour=False, flags=0):
        xs = fe.source_vector(m.n, 7)
        c = oracle.from_matrix(m)
        for storage in storages:
            vb = {"f64": 8, "f32": 4, "bf16": 2}[storage]
            xb = 8 if storage == "f64" else 4
            x64 = xs if storage == "f64" else xs.astype(np.float32).astype(np.float64)
            mb = model_bytes(m.n, m.pairs, vb, xb)
            (yref, ytref), cpu = _oracle_leg(lambda: (oracle.csrc_spmv(c, x64), oracle.csrc_spmv_t(c, x64)),
                                             2 * model_bytes(m.n, m.pairs))
            h = cs.csrc_create_from_csr(m.n, m.row_ptr, m.col, m.val, cs.STORAGE[storage], flags)
            try:
                cs.csrc_partition(h, 0)
                if colour:
                    cs.csrc_color(h, 12345)
                dt = torch.float64 if storage == "f64" else torch.float32
                x = torch.from_numpy(x64).to(dt).cuda()
                y = torch.empty_like(x)
                yt = torch.empty_like(x)
                runs = [(st, st) for st in strategies if st != "color" or colour]
                if colour and "color" in strategies:
                    # the colour strategy again after the ascending greedy colouring of Section 3.2
                    # (csrc_color_stride with no bound): fewer classes than Jones-Plassmann's
                    runs.append(("color", "color (ascending greedy colouring)"))
                for strat, label in runs:
                    if label != strat:
                        cs.csrc_color_stride(h, 0)
                    code = cs.STRATEGIES[strat]
                    ms = _events_ms(lambda: (cs.csrc_spmv(h, x, y, code, sptr), cs.csrc_spmv_t(h, x, yt, code, sptr)),
                                    args.suite_iters) / 2
                    err = max(oracle.max_rel_err(m, x64, gpu(y), yref),
                              oracle.max_rel_err(m, x64, gpu(yt), ytref, transpose=True))
                    info = cs.csrc_get_info(h)
                    emit({"suite": name, "n": m.n, "nnz": m.nnz, "storage": storage, "strategy": label,
                          "ms_per_product": ms, "GB/s": mb / ms / 1e6, "GFLOP/s": flops(m.n, m.pairs) / ms / 1e6,
                          "model_bytes": mb, "nbands": info["nbands"] if strat == "window" else info["stream_nbands"],
                          "spill_entries": info["spill_entries"] if strat == "window" else info["stream_spill_entries"],
                          "ncolors": info["ncolors"], "max_rel_err": err, "tolerance": SUITE_TOL[storage],
                          "cpu_baseline": cpu})
                if cs.csrc_get_last_device_error(h) != cs.CSRC_OK:
                    raise RuntimeError("device status")
            finally:
                cs.csrc_destroy(h)

    def rotating_rows(name, m, copies):
        # the matrix fits in L2: time the window product over `copies` handles of it in turn,
        # so that each product reads its matrix from HBM (the copies together exceed L2 four times)
        xs = fe.source_vector(m.n, 7)
        c = oracle.from_matrix(m)
        (yref, ytref), cpu = _oracle_leg(lambda: (oracle.csrc_spmv(c, xs), oracle.csrc_spmv_t(c, xs)),
                                         2 * model_bytes(m.n, m.pairs))
        hs = [cs.csrc_create_from_csr(m.n, m.row_ptr, m.col, m.val, cs.CSRC_F64) for _ in range(copies)]
        try:
            for h in hs:
                cs.csrc_partition(h, 0)
            xd = [torch.from_numpy(xs).cuda() for _ in range(copies)]
            yd = [torch.empty_like(v) for v in xd]

            def run():
                for h, v, w in zip(hs, xd, yd):
                    cs.csrc_spmv(h, v, w, cs.CSRC_STRAT_WINDOW, sptr)

            ms = _events_ms(run, max(1, args.suite_iters // 10)) / copies
            err = oracle.max_rel_err(m, xs, gpu(yd[-1]), yref)
            cs.csrc_spmv_t(hs[0], xd[0], yd[0], cs.CSRC_STRAT_WINDOW, sptr)
            err = max(err, oracle.max_rel_err(m, xs, gpu(yd[0]), ytref, transpose=True))
            mb = model_bytes(m.n, m.pairs)
            emit({"suite": name, "n": m.n, "nnz": m.nnz, "storage": "f64", "strategy": "window",
                  "copies": copies, "ms_per_product": ms, "GB/s": mb / ms / 1e6,
                  "GFLOP/s": flops(m.n, m.pairs) / ms / 1e6, "max_rel_err": err, "tolerance": 1e-12,
                  "cpu_baseline": cpu})
        finally:
            for h in hs:
                cs.csrc_destroy(h)

    strategies = ["window", "window_atomic", "atomic", "color"]
    sel = set(args.suite.split(",")) if args.suite != "all" else {"c1", "c2", "c3", "c4", "c5", "n1", "n2", "n3", "n4"}
    if "c1" in sel:
        m, _ = build_workload("p1_100x100")
        spmv_rows("C1 p1_100x100 (fits in L2: L2-resident figure)", m, ["f64"], strategies, colour=True)
        rotating_rows("C1 p1_100x100 over rotating copies (HBM-resident figure)", m,
                      int(math.ceil(4 * 129e6 / model_bytes(m.n, m.pairs))))
    if "c2" in sel:
        for wl in ("q1s_96", "q1v_96"):
            m, _ = build_workload(wl)
            spmv_rows(f"C2 {wl}", m, ["f64", "f32", "bf16"] if wl == "q1v_96" else ["f64"], strategies,
                      colour=True)
            if wl == "q1v_96":
                # the stream-order kernel with double-float arithmetic (narrower than FP64:
                # about 2^-46 per operation), labelled as such
                spmv_rows("C2 q1v_96 double-float arithmetic (CSRC_FLAG_DF32_ARITH)", m, ["f64"],
                          ["window_atomic"], flags=cs.CSRC_FLAG_DF32_ARITH)
            del m
    if "c3" in sel:
        m = fe.tet_mesh(2_000_000, 1003, method=args.tet_method)
        spmv_rows(f"C3 tet_{args.tet_method}_2m", m, ["f64", "f32", "bf16"], ["window", "window_atomic"])
        del m

    if "c4" in sel:
        m, _ = build_workload("q1s_96")
        c = oracle.from_matrix(m)
        for storage in ("f64", "bf16"):
            vb = {"f64": 8, "bf16": 2}[storage]
            xb = 8 if storage == "f64" else 4
            h = cs.csrc_create_from_csr(m.n, m.row_ptr, m.col, m.val, cs.STORAGE[storage])
            try:
                cs.csrc_partition(h, 0)
                dt = torch.float64 if storage == "f64" else torch.float32
                x1 = torch.from_numpy(fe.source_vector(m.n, 8)).to(dt).cuda()
                y1 = torch.empty_like(x1)
                ms1 = _events_ms(lambda: cs.csrc_spmv(h, x1, y1, cs.CSRC_STRAT_WINDOW, sptr), args.suite_iters)
                for r in (4, 8, 16, 32):
                    Xn = fe.source_vector(m.n, 8, nrhs=r)
                    if storage != "f64":
                        Xn = Xn.astype(np.float32).astype(np.float64)
                    X = torch.from_numpy(Xn).to(dt).cuda()
                    Y = torch.empty_like(X)
                    cs.csrc_autotune_spmm(h, X, Y, r, sptr)
                    rk = cs.csrc_get_info(h)["tuned_rk"]
                    ms = _events_ms(lambda: cs.csrc_spmm_batched([h], [X], [Y], r, False, sptr), args.suite_iters)
                    Yref, cpu = _oracle_leg(lambda: oracle.csrc_spmm(c, Xn), r * model_bytes(m.n, m.pairs))
                    err = oracle.max_rel_err(m, Xn, gpu(Y), Yref)
                    matrix = 4 * (m.n + 1) + 4 * m.pairs + 2 * vb * m.pairs + vb * m.n
                    mb = matrix + 2 * r * m.n * xb
                    passes = (r + rk - 1) // rk if rk else 1
                    emit({"suite": "C4 q1s_96 several right-hand sides", "storage": storage, "nrhs": r,
                          "k_tile": rk, "ms": ms, "GB/s": mb / ms / 1e6,
                          "GFLOP/s": r * flops(m.n, m.pairs) / ms / 1e6,
                          "streamed_GB/s": (passes * matrix + 2 * r * m.n * xb) / ms / 1e6,
                          "single_vector_ms": ms1, "speedup_vs_r_single_products": r * ms1 / ms,
                          "max_rel_err": err, "tolerance": SUITE_TOL[storage], "cpu_baseline": cpu})
                    del X, Y
            finally:
                cs.csrc_destroy(h)
        del m, c
    if "n1" in sel:
        # rectangular CSRC (Section 2.1): the first half of q1v_96's rows as one subdomain of an
        # overlapping decomposition, its overlap columns in the auxiliary CSR
        g, _ = build_workload("q1v_96")
        a = fe.overlap_subdomain(g, g.n // 2, "q1v_96_half")
        del g
        r = oracle.csr_to_csrcr(a.n, a.m, a.row_ptr, a.col, a.val)
        h = cs.csrc_create_rect_from_csr(a.n, a.m, a.row_ptr, a.col, a.val, cs.CSRC_F64)
        try:
            cs.csrc_partition(h, 0)
            xmn, xnn = fe.source_vector(a.m, 10), fe.source_vector(a.n, 11)
            xm, xn = torch.from_numpy(xmn).cuda(), torch.from_numpy(xnn).cuda()
            yn = torch.empty(a.n, dtype=torch.float64, device="cuda")
            ym = torch.empty(a.m, dtype=torch.float64, device="cuda")
            info = cs.csrc_get_info(h)
            mb = info["model_bytes"]
            for tr in (False, True):
                if tr:
                    ms = _events_ms(lambda: cs.csrc_spmv_t(h, xn, ym, cs.CSRC_STRAT_WINDOW, sptr), args.suite_iters)
                    ref, cpu = _oracle_leg(lambda: oracle.csrcr_spmv_t(r, xnn), mb)
                    err = oracle.max_rel_err_rect(a.n, a.m, a.row_ptr, a.col, a.val, xnn, gpu(ym), ref, transpose=True)
                else:
                    ms = _events_ms(lambda: cs.csrc_spmv(h, xm, yn, cs.CSRC_STRAT_WINDOW, sptr), args.suite_iters)
                    ref, cpu = _oracle_leg(lambda: oracle.csrcr_spmv(r, xmn), mb)
                    err = oracle.max_rel_err_rect(a.n, a.m, a.row_ptr, a.col, a.val, xmn, gpu(yn), ref)
                emit({"suite": "N1 rectangular CSRC: q1v_96 half-domain with overlap", "n": a.n, "m": a.m,
                      "aux_nnz": info["rect_nnz"], "storage": "f64", "strategy": "window",
                      "product": "A^T x" if tr else "A x", "ms_per_product": ms, "GB/s": mb / ms / 1e6,
                      "max_rel_err": err, "tolerance": 1e-12, "cpu_baseline": cpu})
            if cs.csrc_get_last_device_error(h) != cs.CSRC_OK:
                raise RuntimeError("device status")
        finally:
            cs.csrc_destroy(h)
        del a, r
    if "n2" in sel:
        # numerically symmetric storage (Section 2.2): q1v_96's pattern with a_ji = a_ij, au not stored
        g, _ = build_workload("q1v_96")
        rows = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.row_ptr))
        g.val = fe.hash_uniform(1006, np.minimum(rows, g.col), np.maximum(rows, g.col))
        del rows
        c = oracle.from_matrix(g)
        xn = fe.source_vector(g.n, 12)
        h = cs.csrc_create_from_csr(g.n, g.row_ptr, g.col, g.val, cs.CSRC_F64, cs.CSRC_FLAG_SYMMETRIC_VALUES)
        try:
            cs.csrc_partition(h, 0)
            x = torch.from_numpy(xn).cuda()
            y = torch.empty_like(x)
            mb = cs.csrc_get_info(h)["model_bytes"]  # 6 nnz + 22 n + 4
            ref, cpu = _oracle_leg(lambda: oracle.csrc_spmv(c, xn), model_bytes(g.n, g.pairs))
            for strat in ("window", "window_atomic"):
                code = cs.STRATEGIES[strat]
                ms = _events_ms(lambda: cs.csrc_spmv(h, x, y, code, sptr), args.suite_iters)
                emit({"suite": "N2 numerically symmetric CSRC (au not stored): q1v_96 pattern", "n": g.n,
                      "nnz": g.nnz, "storage": "f64", "strategy": strat, "ms_per_product": ms, "model_bytes": mb,
                      "GB/s": mb / ms / 1e6, "GFLOP/s": flops(g.n, g.pairs) / ms / 1e6,
                      "max_rel_err": oracle.max_rel_err(g, xn, gpu(y), ref), "tolerance": 1e-12,
                      "cpu_baseline": cpu})
            if cs.csrc_get_last_device_error(h) != cs.CSRC_OK:
                raise RuntimeError("device status")
        finally:
            cs.csrc_destroy(h)
        del g, c
    if "n3" in sel:
        # index compression: 16-bit band-local window slots instead of 32-bit ones, q1v_96. The
        # window strategy's lists always use 16-bit slots; the stream-order kernel has both forms.
        g, _ = build_workload("q1v_96")
        c = oracle.from_matrix(g)
        xs = fe.source_vector(g.n, 13)
        for storage in ("f64", "bf16"):
            x64 = xs if storage == "f64" else xs.astype(np.float32).astype(np.float64)
            ref, cpu = _oracle_leg(lambda: oracle.csrc_spmv(c, x64), model_bytes(g.n, g.pairs))
            for flags, label, strat in ((0, "16-bit slots (entry lists)", "window"),
                                        (0, "32-bit slots", "window_atomic"),
                                        (cs.CSRC_FLAG_COMPRESS_INDICES, "16-bit slots", "window_atomic")):
                h = cs.csrc_create_from_csr(g.n, g.row_ptr, g.col, g.val, cs.STORAGE[storage], flags)
                try:
                    cs.csrc_partition(h, 0)
                    dt = torch.float64 if storage == "f64" else torch.float32
                    x = torch.from_numpy(x64).to(dt).cuda()
                    y = torch.empty_like(x)
                    code = cs.STRATEGIES[strat]
                    ms = _events_ms(lambda: cs.csrc_spmv(h, x, y, code, sptr), args.suite_iters)
                    info = cs.csrc_get_info(h)
                    mb = info["model_bytes"] if strat != "window" else info["model_bytes"] - 2 * g.pairs
                    emit({"suite": "N3 index compression: q1v_96", "storage": storage, "strategy": strat,
                          "indices": label, "ms_per_product": ms, "model_bytes": mb, "GB/s": mb / ms / 1e6,
                          "GFLOP/s": flops(g.n, g.pairs) / ms / 1e6,
                          "max_rel_err": oracle.max_rel_err(g, x64, gpu(y), ref), "tolerance": SUITE_TOL[storage],
                          "cpu_baseline": cpu})
                    if cs.csrc_get_last_device_error(h) != cs.CSRC_OK:
                        raise RuntimeError("device status")
                finally:
                    cs.csrc_destroy(h)
        del g, c
    if "n4" in sel:
        # BiCG (csrc_bicg) on q1v_96: one A p and one A^T p* per iteration plus two vector passes
        g, _ = build_workload("q1v_96")
        bn = fe.source_vector(g.n, 14)
        h = cs.csrc_create_from_csr(g.n, g.row_ptr, g.col, g.val, cs.CSRC_F64)
        try:
            cs.csrc_partition(h, 0)
            b = torch.from_numpy(bn).cuda()
            x = torch.zeros_like(b)
            cs.csrc_bicg(h, b, x, 1e-8, 3)  # warm-up (plans, scratch)
            x.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res = cs.csrc_bicg(h, b, x, 1e-8, 500)
            torch.cuda.synchronize()
            ms = (time.perf_counter() - t0) * 1e3
            it = max(res["iters"], 1)
            # true residual of the GPU solution, through the oracle's CSR product
            r_true, cpu = _oracle_leg(lambda: bn - oracle.csr_spmv(g.n, g.row_ptr, g.col, g.val, gpu(x)),
                                      model_bytes(g.n, g.pairs))
            # per iteration: two products (model bytes each) and 19 n vector reads/writes of 8 bytes
            per_it = 2 * cs.csrc_get_info(h)["model_bytes"] + 19 * 8 * g.n
            emit({"suite": "N4 BiCG on q1v_96 (csrc_bicg, FP64, window)", "status": res["status"],
                  "iters": res["iters"], "relres": res["relres"],
                  "true_relres": float(np.linalg.norm(r_true) / np.linalg.norm(bn)), "ms_total_host_clock": ms,
                  "ms_per_iteration": ms / it, "GB/s": per_it * it / ms / 1e6, "cpu_baseline": cpu})
        finally:
            cs.csrc_destroy(h)
        del g
    if "c5" in sel:
        ms_list = fe.batch_meshes(256, 1005)
        tot_n = sum(m.n for m in ms_list)
        tot_pairs = sum(m.pairs for m in ms_list)
        xs = [fe.source_vector(m.n, 9 + i) for i, m in enumerate(ms_list)]
        cs_list = [oracle.from_matrix(m) for m in ms_list]
        refs, cpu = _oracle_leg(lambda: [oracle.csrc_spmv(c, x) for c, x in zip(cs_list, xs)],
                                sum(model_bytes(m.n, m.pairs) for m in ms_list))
        res = {}
        for storage, tuned in (("f32", False), ("f32", True), ("f64", False)):
            hs = [cs.csrc_create_from_csr(m.n, m.row_ptr, m.col, m.val, cs.STORAGE[storage]) for m in ms_list]
            try:
                dt = torch.float64 if storage == "f64" else torch.float32
                X = [torch.from_numpy(x).to(dt).cuda() for x in xs]
                Y = [torch.empty_like(x) for x in X]
                if storage == "f32":
                    how = "one CUDA-graph replay over all 256 members"
                    if tuned:
                        # members keep the strategy csrc_autotune picked for their single products
                        for h, x, y in zip(hs, X, Y):
                            cs.csrc_autotune(h, x, y, sptr)
                        how += ", each member at the strategy csrc_autotune picked for its single products"
                    else:
                        how += ", window strategy for every member (the default)"
                    ms = _events_ms(lambda: cs.csrc_spmm_batched(hs, X, Y, 1, False, sptr), args.suite_iters)
                    vb, xb = 4, 4
                else:
                    for h in hs:
                        cs.csrc_partition(h, 0)

                    def separate():
                        for h, x, y in zip(hs, X, Y):
                            cs.csrc_spmv(h, x, y, cs.CSRC_STRAT_WINDOW, sptr)

                    ms = _events_ms(separate, max(3, args.suite_iters // 4))
                    vb, xb, how = 8, 8, "256 separate csrc_spmv calls (product + accumulation launches each)"
                torch.cuda.synchronize()
                err = max(oracle.max_rel_err(m, x if storage == "f64" else x.astype(np.float32).astype(np.float64),
                                             gpu(y), ref)
                          for m, x, y, ref in zip(ms_list, xs, Y, refs))
                mb = sum(model_bytes(m.n, m.pairs, vb, xb) for m in ms_list)
                res[storage + ("_tuned" if tuned else "")] = ms
                emit({"suite": "C5 batch_256", "storage": storage, "how": how, "members": len(ms_list),
                      "sum_n": tot_n, "sum_pairs": tot_pairs, "ms_per_batch": ms, "GB/s": mb / ms / 1e6,
                      "GFLOP/s": flops(tot_n, tot_pairs) / ms / 1e6, "max_rel_err": err,
                      "tolerance": SUITE_TOL[storage], "cpu_baseline": cpu})
            finally:
                for h in hs:
                    cs.csrc_destroy(h)
        # the mixed-precision batched form on double vectors: FP64 handles, each at the precision
        # csrc_autotune_precision picks under a componentwise budget of 1e-5, all in one graph
        hs = [cs.csrc_create_from_csr(m.n, m.row_ptr, m.col, m.val, cs.CSRC_F64) for m in ms_list]
        try:
            X = [torch.from_numpy(x).cuda() for x in xs]
            Y = [torch.empty_like(x) for x in X]
            picks = {}
            for h, x, y in zip(hs, X, Y):
                p_, _ = cs.csrc_autotune_precision(h, x, y, 1e-5, sptr)
                picks[p_] = picks.get(p_, 0) + 1
            ms = _events_ms(lambda: cs.csrc_spmm_batched(hs, X, Y, 1, False, sptr), args.suite_iters)
            torch.cuda.synchronize()
            err = max(oracle.max_rel_err(m, x, gpu(y), ref) for m, x, y, ref in zip(ms_list, xs, Y, refs))
            mb = sum(model_bytes(m.n, m.pairs) for m in ms_list)  # the FP64 model: what the FP64 path moves
            res["mixed"] = ms
            emit({"suite": "C5 batch_256", "storage": "f64 handles, per-matrix precision (budget 1e-5)",
                  "how": "one CUDA-graph replay over all 256 members, each at its tuned precision",
                  "precisions": {{0: "f64", 1: "f32", 2: "bf16"}[k]: v for k, v in picks.items()},
                  "members": len(ms_list), "ms_per_batch": ms, "GB/s (FP64 model)": mb / ms / 1e6,
                  "GFLOP/s": flops(tot_n, tot_pairs) / ms / 1e6, "max_rel_err": err, "tolerance": 1e-5,
                  "cpu_baseline": cpu})
        finally:
            for h in hs:
                cs.csrc_destroy(h)
        emit({"suite": "C5 batch_256 speedup", "f32_graph_vs_f64_separate": res["f64"] / res["f32"],
              "f32_graph_autotuned_members_vs_f64_separate": res["f64"] / res["f32_tuned"],
              "mixed_precision_graph_vs_f64_separate": res["f64"] / res["mixed"]})
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="q1v_96")
    ap.add_argument("--strategy", default="window", choices=["auto", "window", "window_atomic", "atomic", "color"])
    ap.add_argument("--storage", default="f64", choices=["f64", "f32", "bf16"],
                    help="value storage: f64 (the default workload), or f32 / bf16 with float vectors")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--suite", default=None,
                    help="all, or a comma list of c1..c5, n1..n4: one JSON line per configuration row")
    ap.add_argument("--suite-iters", type=int, default=20)
    ap.add_argument("--tet-method", default="delaunay", choices=["delaunay", "kuhn"])
    args = ap.parse_args(argv)
    if args.suite:
        return run_suite(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
