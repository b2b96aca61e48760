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
KERNEL_SOURCES = ["kernels.cu", "band.cuh", "df32.cuh", "internal.h"]


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
    Returns (GB/s, products, seconds, rows)."""
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
        oracle.csrc_spmv(c, xs)
        oracle.csrc_spmv_t(c, xs)
        done += 2
        el = time.perf_counter() - t0
        if el >= budget_s:
            break
    return nbytes * done / el / 1e9, done, el, rows


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    m, x = build_workload(args.workload)
    # calibrate: one product pair on a sample, then size each step to fit the budget
    total_budget = 120.0
    per_step = total_budget / max(1, args.steps + args.warmup)
    _, _, el, rows = oracle_gbs(m, x, 0.0, max_rows=min(m.n, 200_000))
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
    # algorithmic bytes of one band-kernel launch: the CSRC working set plus its spill writes
    vec_bytes = 8 if args.storage == "f64" else 4
    kbytes = int(info["model_bytes"]) + vec_bytes * int(info["spill_entries"])
    achieved = kbytes / (ms_prod / max(nprod, 1) * 1e-3) / 1e9 if nprod else None
    launches = sum(v[0] for v in ktimes.values())
    if rank != 0:
        return 0
    cfg = describe(args.workload, m)
    cfg.update({"nbands": info["nbands"], "spill_entries": info["spill_entries"],
                "arith": {0: "double-float (FP32 pairs)", 1: "FP64 pipe", 2: "FP32"}[info["arith"]],
                "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"})
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
        "roofline": {"bound": "hbm", "kernel": "band_kernel (product)", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": (achieved / peak) if achieved else None,
                     "peak_source": f"{peak_src} hbm_gbs", "traffic": ncu_traffic(args.workload),
                     "algorithmic_bytes_per_launch": kbytes,
                     "launch_ms": ms_prod / max(nprod, 1)},
        "kernels": {k: {"launches": v[0], "ms": v[1]} for k, v in ktimes.items()},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if world == 1 and not args.no_cpu_baseline:
        gbs, done, el, rows = oracle_gbs(m, x_np, args.cpu_seconds)
        line["cpu_baseline"] = {"value": gbs, "unit": "GB/s", "cores": 1, "kind": "oracle",
                                "sample": f"{done} full products (y = A x and y = A^T x alternating) of the "
                                          f"workload in {el:.1f} s, single-threaded FP64 C"}
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


# ----------------------------------------------------------------------------- suite of every configuration
def _events_ms(fn, iters: int) -> float:
    import torch

    for _ in range(3):
        fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(iters):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / iters


def run_suite(args):
    """One JSON line per configuration row: FP64 strategies, FP32 / BF16 storage, several
    right-hand sides and the batched graph launch. Device time with CUDA events; every
    row's inputs are larger than L2 except the P1 100x100 one (marked)."""
    import torch

    import fe_inputs as fe
    import paper_1003_0952_gb300 as cs

    torch.cuda.set_device(0)
    peak, _ = measured_hbm()
    st = torch.cuda.current_stream()
    sptr = st.cuda_stream

    def emit(d):
        d["frac_of_measured_hbm"] = d["GB/s"] / peak if "GB/s" in d else None
        print(json.dumps(d), flush=True)

    def spmv_rows(name, m, storages, strategies, colour=False):
        xs = fe.source_vector(m.n, 7)
        for storage in storages:
            vb = {"f64": 8, "f32": 4, "bf16": 2}[storage]
            xb = 8 if storage == "f64" else 4
            h = cs.csrc_create_from_csr(m.n, m.row_ptr, m.col, m.val, cs.STORAGE[storage])
            try:
                cs.csrc_partition(h, 0)
                if colour:
                    cs.csrc_color(h, 12345)
                dt = torch.float64 if storage == "f64" else torch.float32
                x = torch.from_numpy(xs).to(dt).cuda()
                y = torch.empty_like(x)
                mb = model_bytes(m.n, m.pairs, vb, xb)
                for strat in strategies:
                    if strat == "color" and not colour:
                        continue
                    code = cs.STRATEGIES[strat]
                    ms = _events_ms(lambda: (cs.csrc_spmv(h, x, y, code, sptr), cs.csrc_spmv_t(h, x, y, code, sptr)),
                                    args.suite_iters) / 2
                    info = cs.csrc_get_info(h)
                    emit({"suite": name, "n": m.n, "nnz": m.nnz, "storage": storage, "strategy": strat,
                          "ms_per_product": ms, "GB/s": mb / ms / 1e6, "GFLOP/s": flops(m.n, m.pairs) / ms / 1e6,
                          "nbands": info["nbands"], "spill_entries": info["spill_entries"],
                          "ncolors": info["ncolors"], "lanes_per_row": info["group"]})
                if cs.csrc_get_last_device_error(h) != cs.CSRC_OK:
                    raise RuntimeError("device status")
            finally:
                cs.csrc_destroy(h)

    sel = set(args.suite.split(",")) if args.suite != "all" else {"c1", "c2", "c3", "c4", "c5", "n1", "n2", "n3", "n4"}
    if "c1" in sel:
        m, _ = build_workload("p1_100x100")
        spmv_rows("C1 p1_100x100 (fits in L2)", m, ["f64"], ["window", "atomic", "color"], colour=True)
    if "c2" in sel:
        for wl in ("q1s_96", "q1v_96"):
            m, _ = build_workload(wl)
            spmv_rows(f"C2 {wl}", m, ["f64"], ["window", "atomic", "color"], colour=True)
            del m
    if "c3" in sel:
        m = fe.tet_mesh(2_000_000, 1003, method=args.tet_method)
        spmv_rows(f"C3 tet_{args.tet_method}_2m", m, ["f64", "f32"], ["window"])
        del m
    if "c4" in sel:
        m, _ = build_workload("q1s_96")
        for storage in ("f64", "bf16"):
            vb = {"f64": 8, "bf16": 2}[storage]
            xb = 8 if storage == "f64" else 4
            h = cs.csrc_create_from_csr(m.n, m.row_ptr, m.col, m.val, cs.STORAGE[storage])
            try:
                cs.csrc_partition(h, 0)
                dt = torch.float64 if storage == "f64" else torch.float32
                for r in (4, 8, 16, 32):
                    X = torch.from_numpy(fe.source_vector(m.n, 8, nrhs=r)).to(dt).cuda()
                    Y = torch.empty_like(X)
                    cs.csrc_autotune_spmm(h, X, Y, r, sptr)
                    rk = cs.csrc_get_info(h)["tuned_rk"]
                    ms = _events_ms(lambda: cs.csrc_spmm_batched([h], [X], [Y], r, False, sptr), args.suite_iters)
                    matrix = 4 * (m.n + 1) + 4 * m.pairs + 2 * vb * m.pairs + vb * m.n
                    mb = matrix + 2 * r * m.n * xb
                    passes = (r + rk - 1) // rk if rk else 1
                    emit({"suite": "C4 q1s_96 several right-hand sides", "storage": storage, "nrhs": r,
                          "k_tile": rk, "ms": ms, "GB/s": mb / ms / 1e6,
                          "GFLOP/s": r * flops(m.n, m.pairs) / ms / 1e6,
                          "streamed_GB/s": (passes * matrix + 2 * r * m.n * xb) / ms / 1e6})
                    del X, Y
            finally:
                cs.csrc_destroy(h)
        del m
    if "n1" in sel:
        # rectangular CSRC (Section 2.1): the first half of q1v_96's rows as one subdomain of an
        # overlapping decomposition, its overlap columns in the auxiliary CSR
        g, _ = build_workload("q1v_96")
        a = fe.overlap_subdomain(g, g.n // 2, "q1v_96_half")
        del g
        h = cs.csrc_create_rect_from_csr(a.n, a.m, a.row_ptr, a.col, a.val, cs.CSRC_F64)
        try:
            cs.csrc_partition(h, 0)
            xm = torch.from_numpy(fe.source_vector(a.m, 10)).cuda()
            xn = torch.from_numpy(fe.source_vector(a.n, 11)).cuda()
            yn = torch.empty(a.n, dtype=torch.float64, device="cuda")
            ym = torch.empty(a.m, dtype=torch.float64, device="cuda")
            info = cs.csrc_get_info(h)
            mb = info["model_bytes"]
            for tr in (False, True):
                if tr:
                    ms = _events_ms(lambda: cs.csrc_spmv_t(h, xn, ym, cs.CSRC_STRAT_WINDOW, sptr), args.suite_iters)
                else:
                    ms = _events_ms(lambda: cs.csrc_spmv(h, xm, yn, cs.CSRC_STRAT_WINDOW, sptr), args.suite_iters)
                emit({"suite": "N1 rectangular CSRC: q1v_96 half-domain with overlap", "n": a.n, "m": a.m,
                      "aux_nnz": info["rect_nnz"], "storage": "f64", "strategy": "window",
                      "product": "A^T x" if tr else "A x", "ms_per_product": ms, "GB/s": mb / ms / 1e6})
            if cs.csrc_get_last_device_error(h) != cs.CSRC_OK:
                raise RuntimeError("device status")
        finally:
            cs.csrc_destroy(h)
        del a
    if "n2" in sel:
        # numerically symmetric storage (Section 2.2): q1v_96's pattern with a_ji = a_ij, au not stored
        g, _ = build_workload("q1v_96")
        rows = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.row_ptr))
        g.val = fe.hash_uniform(1006, np.minimum(rows, g.col), np.maximum(rows, g.col))
        del rows
        h = cs.csrc_create_from_csr(g.n, g.row_ptr, g.col, g.val, cs.CSRC_F64, cs.CSRC_FLAG_SYMMETRIC_VALUES)
        try:
            cs.csrc_partition(h, 0)
            x = torch.from_numpy(fe.source_vector(g.n, 12)).cuda()
            y = torch.empty_like(x)
            mb = cs.csrc_get_info(h)["model_bytes"]  # 6 nnz + 22 n + 4
            ms = _events_ms(lambda: cs.csrc_spmv(h, x, y, cs.CSRC_STRAT_WINDOW, sptr), args.suite_iters)
            emit({"suite": "N2 numerically symmetric CSRC (au not stored): q1v_96 pattern", "n": g.n, "nnz": g.nnz,
                  "storage": "f64", "strategy": "window", "ms_per_product": ms, "model_bytes": mb,
                  "GB/s": mb / ms / 1e6, "GFLOP/s": flops(g.n, g.pairs) / ms / 1e6})
            if cs.csrc_get_last_device_error(h) != cs.CSRC_OK:
                raise RuntimeError("device status")
        finally:
            cs.csrc_destroy(h)
        del g
    if "n3" in sel:
        # index compression: 16-bit band-local window slots instead of 32-bit ones, q1v_96
        g, _ = build_workload("q1v_96")
        xs = fe.source_vector(g.n, 13)
        for storage in ("f64", "bf16"):
            for flags, label in ((0, "32-bit slots"), (cs.CSRC_FLAG_COMPRESS_INDICES, "16-bit slots")):
                h = cs.csrc_create_from_csr(g.n, g.row_ptr, g.col, g.val, cs.STORAGE[storage], flags)
                try:
                    cs.csrc_partition(h, 0)
                    dt = torch.float64 if storage == "f64" else torch.float32
                    x = torch.from_numpy(xs).to(dt).cuda()
                    y = torch.empty_like(x)
                    mb = cs.csrc_get_info(h)["model_bytes"]
                    ms = _events_ms(lambda: cs.csrc_spmv(h, x, y, cs.CSRC_STRAT_WINDOW, sptr), args.suite_iters)
                    emit({"suite": "N3 index compression: q1v_96", "storage": storage, "indices": label,
                          "ms_per_product": ms, "model_bytes": mb, "GB/s": mb / ms / 1e6,
                          "GFLOP/s": flops(g.n, g.pairs) / ms / 1e6})
                    if cs.csrc_get_last_device_error(h) != cs.CSRC_OK:
                        raise RuntimeError("device status")
                finally:
                    cs.csrc_destroy(h)
        del g
    if "n4" in sel:
        # BiCG (csrc_bicg) on q1v_96: one A p and one A^T p* per iteration plus two vector passes
        g, _ = build_workload("q1v_96")
        h = cs.csrc_create_from_csr(g.n, g.row_ptr, g.col, g.val, cs.CSRC_F64)
        try:
            cs.csrc_partition(h, 0)
            b = torch.from_numpy(fe.source_vector(g.n, 14)).cuda()
            x = torch.zeros_like(b)
            cs.csrc_bicg(h, b, x, 1e-8, 3)  # warm-up (plans, scratch)
            x.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res = cs.csrc_bicg(h, b, x, 1e-8, 500)
            torch.cuda.synchronize()
            ms = (time.perf_counter() - t0) * 1e3
            it = max(res["iters"], 1)
            # per iteration: two products (model bytes each) and 19 n vector reads/writes of 8 bytes
            per_it = 2 * cs.csrc_get_info(h)["model_bytes"] + 19 * 8 * g.n
            emit({"suite": "N4 BiCG on q1v_96 (csrc_bicg, FP64, window)", "status": res["status"],
                  "iters": res["iters"], "relres": res["relres"], "ms_total_host_clock": ms,
                  "ms_per_iteration": ms / it, "GB/s": per_it * it / ms / 1e6})
        finally:
            cs.csrc_destroy(h)
        del g
    if "c5" in sel:
        ms_list = fe.batch_meshes(256, 1005)
        tot_n = sum(m.n for m in ms_list)
        tot_pairs = sum(m.pairs for m in ms_list)
        res = {}
        for storage in ("f32", "f64"):
            hs = [cs.csrc_create_from_csr(m.n, m.row_ptr, m.col, m.val, cs.STORAGE[storage]) for m in ms_list]
            try:
                dt = torch.float64 if storage == "f64" else torch.float32
                X = [torch.from_numpy(fe.source_vector(m.n, 9 + i)).to(dt).cuda() for i, m in enumerate(ms_list)]
                Y = [torch.empty_like(x) for x in X]
                if storage == "f32":
                    for h, x, y in zip(hs, X, Y):
                        cs.csrc_autotune(h, x, y, sptr)
                    ms = _events_ms(lambda: cs.csrc_spmm_batched(hs, X, Y, 1, False, sptr), args.suite_iters)
                    vb, xb, how = 4, 4, "one CUDA-graph replay: persistent band kernels over all 256 members"
                else:
                    for h in hs:
                        cs.csrc_partition(h, 0)

                    def separate():
                        for h, x, y in zip(hs, X, Y):
                            cs.csrc_spmv(h, x, y, cs.CSRC_STRAT_WINDOW, sptr)

                    ms = _events_ms(separate, max(3, args.suite_iters // 4))
                    vb, xb, how = 8, 8, "256 separate csrc_spmv calls (band + accumulation launches each)"
                mb = sum(model_bytes(m.n, m.pairs, vb, xb) for m in ms_list)
                res[storage] = ms
                emit({"suite": "C5 batch_256", "storage": storage, "how": how, "members": len(ms_list),
                      "sum_n": tot_n, "sum_pairs": tot_pairs, "ms_per_batch": ms, "GB/s": mb / ms / 1e6,
                      "GFLOP/s": flops(tot_n, tot_pairs) / ms / 1e6})
            finally:
                for h in hs:
                    cs.csrc_destroy(h)
        emit({"suite": "C5 batch_256 speedup", "f32_graph_vs_f64_separate": res["f64"] / res["f32"]})
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="q1v_96")
    ap.add_argument("--strategy", default="window", choices=["auto", "window", "atomic"])
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
