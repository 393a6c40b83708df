"""Benchmark: SpMV GB/s per format and CG solves/s on the 27-point stencil.

Workload (HPCG problem, §II-B): 27-point stencil on a 128^3 grid, FP64 values,
int32 indices (N = 2,097,152 rows, 55,742,968 entries), x ~ U[-1, 1) from
SplitMix64 seed 2. One step = the hot path once:
  * y = A x in each format (COO, CSR, DIA, ELL, HYB), each preceded by an L2
    flush (a 256 MB read, which leaves L2 holding clean lines: a write would
    leave dirty ones whose write-back lands in the timed kernel; the matrix
    arrays alone are larger than L2 too);
  * one full FP64 CG solve to 1e-9 relative residual in the format the
    deterministic selector picks (DIA), b = A 1, x0 = 0.
`value` = GB/s of the selected format's SpMV: its algorithmic bytes (the
format's arrays once, x once, y once) / mean kernel time (CUDA events on the
launching stream), summed over ranks for N GPUs (independent replicas).

--impl reference times the CPU oracle (single-threaded C, FP64) on the same
workload, metric and unit: the paper's method has no public GPU reference to
install here, so the oracle is the reference arm.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

FMTS = ("coo", "csr", "dia", "ell", "hyb")
METRIC = "SpMV GB/s (selected format, % of HBM peak); CG solves/s (FP64, 1e-9)"


def algorithmic_bytes(fmt: str, N: int, nnz: int, ndiag: int, K: int, hyb_k: int, hyb_over: int,
                      vb: int = 8) -> int:
    """Bytes one SpMV must move: the format's arrays once (padding included),
    x once and y once (square matrix, N = ncols)."""
    vec = 2 * vb * N
    if fmt == "coo":
        return (8 + vb) * nnz + vec
    if fmt == "csr":
        return (4 + vb) * nnz + 4 * (N + 1) + vec
    if fmt == "dia":
        return vb * ndiag * N + 4 * ndiag + vec
    if fmt == "ell":
        return (4 + vb) * K * N + vec
    if fmt == "hyb":
        return (4 + vb) * hyb_k * N + (8 + vb) * hyb_over + vec
    raise ValueError(fmt)


# SpMV kernel launches per call, per format (DIA/ELL/CSR-vector: 1;
# COO: segmented + fix-up; HYB: ELL + segmented + fix-up).
def launches(fmt: str, info) -> int:
    """Kernels one SpMV of this format launches with its chosen variant:
    segmented kernels (COO variant 1, CSR merge variant 6, HYB's COO part)
    add a fix-up kernel; the others are one launch."""
    v = int(info.spmv_variant)
    if fmt == "coo":
        return 1 if v == 2 else 2
    if fmt == "csr":
        return 2 if v == 6 else 1
    if fmt == "hyb":
        return 1 + (2 if int(info.hyb_coo_nnz) > 0 else 0)
    return 1


def l2_evict(buf):
    """Replaces L2's contents by reading `buf` (twice L2's size) with a
    reduction. The lines left behind are clean, so none of their write-back
    falls into the next timed kernel (a write-based flush would leave 126 MB
    of dirty lines to write back while that kernel runs)."""
    return buf.sum()


def aggregate_ranks(total_ms: float, kernel_ms: float, units: float, world: int, device=None):
    """Whole-job figures of a run on `world` ranks (one process per GPU): the
    maximum over ranks of the timed region and of the kernel time, and the
    work units summed over ranks. Collective (torch.distributed) when
    world > 1; `device` holds the reduction tensors (a CUDA device under
    NCCL, None = CPU under gloo)."""
    import torch
    t = torch.tensor([total_ms, kernel_ms], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t[0]), float(t[1]), float(u[0])


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


# B300 FP64 pipe: 2 DFMA per clock per SM (4 flops), 148 SMs, at the maximum
# SM clock (2032 MHz): 1.203 TFLOP/s, the nominal 1.25 TFLOP/s at this clock.
SMS = 148
FP64_FLOPS_PER_CLK_SM = 4


def fp64_peak_tflops():
    mhz = 2032.0
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            mhz = float(json.load(f).get("sm_max_mhz", mhz))
    return SMS * FP64_FLOPS_PER_CLK_SM * mhz * 1e6 / 1e12


def executed_fmas(fmt: str, N: int, nnz: int, ndiag: int, K: int, hyb_k: int, hyb_over: int) -> int:
    """Multiply-adds one SpMV executes: DIA one per slot (padding included),
    ELL/HYB one per non-padding slot, CSR/COO one per entry."""
    if fmt == "dia":
        return ndiag * N
    return nnz


def kernel_source_hash() -> str:
    """Hash of the DIA SpMV kernel's source: its definition (from its header
    comment to the next kernel's), its tile-size rule, and the value-stream
    load it issues: the code that decides what one launch reads and writes.
    None when a marker is missing."""
    csrc = os.path.join(ROOT, "paper_2209_06478_b300", "csrc")
    spmv = open(os.path.join(csrc, "spmv.cu")).read()
    dev = open(os.path.join(csrc, "device.cuh")).read()
    parts = []
    for src, a, b in ((spmv, "// DIA: a thread owns", "// ELL: slot-major"),
                      (spmv, "static int64_t tile_rows_for(const dynmat_s* A) {", "\n}\n"),
                      (dev, "// The DIA value stream:", "\n\n")):
        i = src.find(a)
        j = src.find(b, i + 1) if i >= 0 else -1
        if i < 0 or j < 0:
            return None
        parts.append(src[i:j])
    return hashlib.sha256("\0".join(parts).encode()).hexdigest()[:16]


def ncu_traffic(kernel: str, workload: str, variant: int):
    """DRAM bytes (read + write) per launch of `kernel` in `variant` from the
    committed ncu summary, or None when the summary is missing, has no entry
    for the variant, or the kernel source changed since it was taken."""
    p = os.path.join(ROOT, "profiles", "ncu_summary.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(kernel, {}).get(workload)
    if not e or e.get("source_hash") != kernel_source_hash():
        return None
    v = e.get("variants", {}).get(str(variant))
    return None if v is None else v.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi samples (200 ms) while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def stencil_workload(n: int):
    N, r, c, v = synth.stencil27(n)
    x = synth.uniform_pm1(2, N)
    return N, r, c, v, x


# ---------------------------------------------------------------------------
# CPU oracle (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------

def oracle_spmv_gbs(N, r, c, v, x, budget_s: float, reps_max: int = 1000, omp: bool = False,
                    dia=None):
    """GB/s of the oracle's DIA product (algorithmic bytes / mean call time);
    omp=True times the same source's OpenMP build on all host cores."""
    import oracle
    oracle.build(omp=omp)
    if dia is None:
        dia = oracle.to_format("dia", N, N, r, c, v)
    nbytes = algorithmic_bytes("dia", N, r.size, dia["offsets"].size, 0, 0, 0)
    times = []
    t_end = time.perf_counter() + budget_s
    while len(times) < reps_max and (not times or time.perf_counter() < t_end):
        t0 = time.perf_counter()
        oracle.spmv("dia", N, N, dia, x, omp=omp)
        times.append(time.perf_counter() - t0)
    t = float(np.mean(times))
    return nbytes / t / 1e9, len(times), t


def run_reference(args):
    rank, world = int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    n = args.n
    N, r, c, v, x = stencil_workload(n)
    per_step = max(1.0, 20.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        oracle_spmv_gbs(N, r, c, v, x, budget_s=0.0, reps_max=1)
    gbs, reps, t = oracle_spmv_gbs(N, r, c, v, x, budget_s=per_step * args.steps,
                                   reps_max=max(1, args.steps))
    line = {
        "impl": "reference", "metric": METRIC, "value": round(gbs, 3), "unit": "GB/s",
        "n_gpus": args.gpus, "steps": reps, "warmup": args.warmup,
        "ms_per_step": round(t * 1e3, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "27-point stencil %d^3, FP64, DIA SpMV" % n, "nrows": N,
                   "nnz": int(r.size), "formats": ["dia"]},
        "cpu_baseline": {"value": round(gbs, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": "%d DIA SpMV calls of the single-threaded C oracle" % reps},
        "e2e": {"value": round(gbs, 3), "unit": "GB/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_dynmat(args):
    import torch
    import torch.distributed as dist
    from paper_2209_06478_b300 import build
    build.build()
    from paper_2209_06478_b300 import dynmat as dm

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    n = args.n
    N, r, c, v, x_host = stencil_workload(n)
    nnz = int(r.size)
    A = {}
    t0 = time.perf_counter()
    base = dm.dynmat_create(N, N, r, c, v)
    feats = base.features()
    chosen = FMTS[feats["choice"]]
    for f in FMTS:
        h = dm.dynmat_create(N, N, r, c, v)
        h.convert(f)
        h.tune_variant()
        A[f] = h
    setup_s = time.perf_counter() - t0
    info = {f: A[f].info() for f in FMTS}
    nbytes = {f: algorithmic_bytes(f, N, nnz, info["dia"].ndiag, info["ell"].ell_width,
                                   info["hyb"].ell_width, info["hyb"].hyb_coo_nnz)
              for f in FMTS}
    x = torch.from_numpy(x_host).to(dev)
    y = torch.empty(N, dtype=torch.float64, device=dev)
    ones = torch.ones(N, dtype=torch.float64, device=dev)
    b = torch.empty(N, dtype=torch.float64, device=dev)
    A[chosen].spmv(ones, b)
    xs = torch.zeros(N, dtype=torch.float64, device=dev)
    flush = torch.ones(64 << 20, dtype=torch.float32, device=dev)  # 256 MB

    def step(record):
        ev = {}
        for f in FMTS:
            l2_evict(flush)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            A[f].spmv(x, y)
            e1.record(stream)
            ev[f] = (e0, e1)
        xs.zero_()
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        res = A[chosen].cg_solve(b, xs, tol=1e-9, max_iters=5000, check_every=args.check_every)
        c1.record(stream)
        torch.cuda.synchronize()
        if record is not None:
            for f in FMTS:
                record.setdefault(f, []).append(ev[f][0].elapsed_time(ev[f][1]))
            record.setdefault("cg", []).append(c0.elapsed_time(c1))
            record.setdefault("cg_iters", []).append(res["iterations"])
            record.setdefault("cg_status", []).append(res["status"])
            record.setdefault("cg_true_res", []).append(res["true_rel_residual"])

    for _ in range(args.warmup):
        step(None)
    rec = {}
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for _ in range(args.steps):
            step(rec)
        s1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    total_ms = s0.elapsed_time(s1)
    ms = {f: float(np.mean(rec[f])) for f in FMTS}
    gbs = {f: nbytes[f] / (ms[f] * 1e-3) / 1e9 for f in FMTS}
    cg_ms = float(np.mean(rec["cg"]))
    iters = int(np.median(rec["cg_iters"]))

    # end to end through the public API with host buffers (H2D x, D2H y inside)
    # (host buffers from the library's allocator: huge pages, registered with CUDA)
    xh = dm.dynmat_host_alloc(N)
    xh[:] = x_host
    yh = dm.dynmat_host_alloc(N)
    # warm-up: at least 3 calls and 0.25 s (the first calls after the timed
    # region run up to 25% slower while the GPU settles)
    w0, nw = time.perf_counter(), 0
    while nw < 3 or time.perf_counter() - w0 < 0.25:
        A[chosen].spmv_host(xh, yh)
        nw += 1
    e2e_t = []
    n_e2e = max(50, args.steps)
    for _ in range(n_e2e):
        t1 = time.perf_counter()
        A[chosen].spmv_host(xh, yh)
        e2e_t.append(time.perf_counter() - t1)
    e2e_gbs = nbytes[chosen] / float(np.median(e2e_t)) / 1e9  # median of the calls

    # max over ranks of the timed region and kernel time; bytes summed over ranks
    total_ms, kernel_ms, all_bytes = aggregate_ranks(total_ms, ms[chosen], float(nbytes[chosen]),
                                                     world, dev)
    value = all_bytes / (kernel_ms * 1e-3) / 1e9

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    extras = {}
    if not args.no_extras and world == 1:
        wanted = set(args.extras.split(",")) if args.extras else None
        want = lambda name: wanted is None or name in wanted  # noqa: E731
        # Host-side inputs of the last two blocks (the 192^3 system for the
        # oracle's check, the served stream's 2M-row matrices) are generated
        # just before each of them, while nothing is timed. Generation beside
        # a timed block (numpy, the oracle's OpenMP product, the interpreter
        # lock they hold) delays the host's launches inside the timed region,
        # and the GPU waits there: the 16^3 CSR product read 422 us against
        # 10 us alone, a PCG solve 74.1 against 70.6 ms, the 64-matrix batch
        # 716 against 640 us.
        from concurrent.futures import ThreadPoolExecutor
        bg = ThreadPoolExecutor(max_workers=3)
        fut = {}

        def start_background(name):
            if name == "mixed" and want("mixed"):
                fut["mixed"] = bg.submit(oracle_system_192)
            if name == "serving" and want("serving"):
                fut["serving"] = bg.submit(serving_pool)

        for name, fn in (("selector", lambda: bench_selector(dm, torch, N, r, c, v, x_host)),
                         ("convert", lambda: bench_convert(dm, torch, N, r, c, v)),
                         ("small", lambda: bench_small(dm, torch)),
                         ("diag", lambda: bench_diag(dm, torch)),
                         ("hpcg", lambda: bench_hpcg(dm, torch)),
                         ("batch", lambda: bench_batch(dm, torch, kinds=tuple(args.batch_kinds.split(",")),
                                                       count=args.batch_count,
                                                       tune=not (args.batch_untuned or args.batch_format),
                                                       fixed=args.batch_format or "csr")),
                         ("split", lambda: bench_split(dm, torch)),
                         ("mixed", lambda: bench_mixed(dm, torch, fut["mixed"].result())),
                         ("serving", lambda: bench_serving(fut["serving"].result()))):
            if name in ("mixed", "serving"):
                start_background(name)  # its inputs, generated while nothing is timed
            if not want(name):
                continue
            try:
                extras[name] = fn()
            except Exception as e:  # reported, never hidden
                extras[name] = {"error": "%s: %s" % (type(e).__name__, e)}
        bg.shutdown(wait=False)
    peak, peak_kind = measured_peaks()
    # The bound of the selected kernel: whichever of HBM bytes and FP64
    # multiply-adds takes longer at peak.
    fp64_peak = fp64_peak_tflops()
    fmas = executed_fmas(chosen, N, nnz, info["dia"].ndiag, info["ell"].ell_width,
                         info["hyb"].ell_width, info["hyb"].hyb_coo_nnz)
    t_hbm = nbytes[chosen] / (peak * 1e9)
    t_alu = 2 * fmas / (fp64_peak * 1e12)
    kvar = int(info[chosen].spmv_variant)
    kname = "%s SpMV kernel, variant %d" % (chosen, kvar)
    if t_alu > t_hbm:
        ach = 2 * fmas / (kernel_ms * 1e-3) / 1e12
        roofline = {"bound": "alu", "achieved": round(ach, 4), "peak": round(fp64_peak, 4),
                    "unit": "TFLOP/s", "frac": round(ach / fp64_peak, 4),
                    "peak_source": "derived: 148 SMs x 2 DFMA/clk x 2 flop x %.0f MHz" % (
                        fp64_peak * 1e6 / (SMS * FP64_FLOPS_PER_CLK_SM)),
                    "hbm": {"achieved": round(gbs[chosen], 1), "peak": peak, "unit": "GB/s",
                            "frac": round(gbs[chosen] / peak, 4), "peak_source": peak_kind},
                    "kernel": kname, "flops_per_launch": 2 * fmas,
                    "bytes_per_launch": int(nbytes[chosen]),
                    "traffic": ncu_traffic("%s_spmv" % chosen, "stencil27_%d" % n, kvar)}
    else:
        roofline = {"bound": "hbm", "achieved": round(gbs[chosen], 1), "peak": peak,
                    "unit": "GB/s", "frac": round(gbs[chosen] / peak, 4),
                    "peak_source": peak_kind, "kernel": kname,
                    "bytes_per_launch": int(nbytes[chosen]),
                    "traffic": ncu_traffic("%s_spmv" % chosen, "stencil27_%d" % n, kvar)}
    every = args.check_every
    cg_launches = 3 * (1 + int(np.ceil(max(iters - 1, 0) / every)) * every) + 8
    launches_per_step = sum(launches(f, info[f]) for f in FMTS) + cg_launches
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        dia = oracle.to_format("dia", N, N, r, c, v)
        cg_bytes, reps, t = oracle_spmv_gbs(N, r, c, v, x_host, budget_s=args.cpu_seconds, dia=dia)
        cpu = {"value": round(cg_bytes, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
               "sample": "%d DIA SpMV calls (27-point %d^3, FP64) of the single-threaded C oracle, "
                         "%.1f s" % (reps, n, reps * t)}
        # The same oracle source built with OpenMP: the paper's multi-core CPU backend.
        oracle_spmv_gbs(N, r, c, v, x_host, budget_s=0.0, reps_max=2, omp=True, dia=dia)
        og, oreps, ot = oracle_spmv_gbs(N, r, c, v, x_host, budget_s=args.cpu_seconds / 4,
                                        omp=True, dia=dia)
        cpu["openmp"] = {"value": round(og, 3), "unit": "GB/s", "cores": oracle.threads(omp=True),
                         "sample": "%d DIA SpMV calls of the oracle's OpenMP build (rows split "
                                   "across threads; bit-identical to the serial build), %.1f s"
                                   % (oreps, oreps * ot)}
        # The oracle's FP64 CG (CSR, single thread), a fixed few iterations.
        rp = oracle.coo_to_csr(N, r)
        b_h = oracle.spmv("csr", N, N, {"rowptr": rp, "col": c, "val": v}, np.ones(N))
        k_cg = 5
        t_cg = time.perf_counter()
        oracle.cg(N, rp, c, v, b_h, tol=0.0, max_iters=k_cg)
        t_cg = time.perf_counter() - t_cg
        cpu["cg"] = {"us_per_iteration": round(t_cg / k_cg * 1e6, 1), "cores": 1,
                     "sample": "%d iterations of the oracle's FP64 CG (CSR) on the same system, "
                               "%.1f s" % (k_cg, t_cg)}
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(total_ms / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "27-point stencil %d^3, FP64 values, int32 indices" % n,
                   "nrows": N, "nnz": nnz, "selected_format": chosen,
                   "parallelism": "replicas" if world > 1 else "1 GPU",
                   "l2": "256 MB read before every timed SpMV (L2 left clean); matrix > L2"},
        "per_format": {f: {"gbs": round(gbs[f], 1), "us": round(ms[f] * 1e3, 2),
                           "us_median": round(float(np.median(rec[f])) * 1e3, 2),
                           "us_min": round(float(np.min(rec[f])) * 1e3, 2),
                           "variant": int(info[f].spmv_variant),
                           "bytes": int(nbytes[f]), "frac_of_peak": round(gbs[f] / peak, 4),
                           "gflops_useful": round(2 * nnz / (ms[f] * 1e-3) / 1e9, 1)}
                       for f in FMTS},
        "cg": {"format": chosen, "solves_per_s": round(1e3 / cg_ms, 3), "ms_per_solve": round(cg_ms, 3),
               "iterations": iters, "tol": 1e-9,
               "status": int(np.max(rec["cg_status"])),
               "true_rel_residual": float(np.max(rec["cg_true_res"])),
               "us_per_iteration": round(cg_ms * 1e3 / max(iters, 1), 2)},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": {"value": round(e2e_gbs, 3), "unit": "GB/s", "h2d_bytes_per_step": 8 * N,
                "d2h_bytes_per_step": 8 * N,
                "what": "dynmat_spmv_host on host x and y from dynmat_host_alloc (copies inside, "
                        "pipelined with the product), median of %d calls after 0.25 s of warm-up "
                        "calls" % n_e2e},
        "gpu_launches": int(launches_per_step * args.steps),
        "setup_s": round(setup_s, 2),
        "clocks": clk.summary(),
    }
    line.update(extras)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# Further measurements of the hot path (reported in the same line)
# ---------------------------------------------------------------------------

def cuda_time_ms(torch, fn, reps: int, warmup: int = 2):
    """Median CUDA-event time of fn() on the current stream. A 25 us
    device-side sleep precedes each start event, so the GPU is still busy
    while the host enqueues fn's work and the host's launch path (slower
    while background threads load the CPU) stays out of the timed region."""
    s = torch.cuda.current_stream()
    for _ in range(warmup):
        fn()
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda._sleep(50_000)
        e0.record(s)
        fn()
        e1.record(s)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(np.median(ts))


BATCH_KINDS = ("banded", "powerlaw", "uniform")


def bench_batch(dm, torch, reps: int = 10, kinds=BATCH_KINDS, count: int = 64, tune: bool = True,
                fixed: str = "csr"):
    """64 uneven FP64 matrices (1/3 banded, 1/3 power-law rows, 1/3 uniform;
    10k-500k rows, seeds 100-163) in one persistent launch, format and tile
    shape per matrix from the batch tuner; compared with one dynmat_spmv
    launch per matrix in the deterministic selector's format. `kinds` and
    `count` keep the first `count` matrices of those kinds, and tune=False
    sets every matrix in format `fixed` with its default tile shape (a
    reproducible case for a profiler: the tuner's choices depend on its
    timings)."""
    t0 = time.perf_counter()
    specs = [sp for sp in synth.batch_specs() if sp[1] in kinds][:count]
    B = dm.DynBatch(len(specs))
    keep, per = [], []
    for k, (seed, kind, n, extra) in enumerate(specs):
        N, r, c, v = synth.make(kind, seed, n, extra)
        A = dm.dynmat_create(N, N, r, c, v)
        A.convert("csr" if tune else fixed)
        x = torch.from_numpy(synth.uniform_pm1(seed, N)).cuda()
        y = torch.empty(N, dtype=torch.float64, device="cuda")
        B.set(k, A, x, y)
        keep.append((A, x, y, kind))
        P = dm.dynmat_create(N, N, r, c, v)
        f = P.select_format(dm.SELECT_FEATURES)
        P.convert(f)
        P.tune_variant()
        per.append((P, x, torch.empty_like(y)))
    gen_s = time.perf_counter() - t0
    t1 = time.perf_counter()
    choices = {}
    shape_counts = {}  # per kind: "format lanes/rows/entries" -> slots
    total_bytes = 0
    shapes = []  # per slot: tuned shape, algorithmic bytes, entries
    for k, (A, x, y, kind) in enumerate(keep):
        fmt, shape = B.autotune(k) if tune else (dm.FORMATS.index(fixed), None)
        i = A.info()
        name = dm.FORMATS[fmt]
        choices.setdefault(kind, {}).setdefault(name, 0)
        choices[kind][name] += 1
        if shape is not None:  # (lanes, rows per tile, entries per tile)
            key = "%s %d/%d/%d" % (name, *shape)
            shape_counts.setdefault(kind, {}).setdefault(key, 0)
            shape_counts[kind][key] += 1
        nb = algorithmic_bytes(name, i.nrows, i.nnz, i.ndiag, i.ell_width, 0, 0)
        total_bytes += nb
        shapes.append((shape, nb, int(i.nnz)))
    tune_s = time.perf_counter() - t1
    ms = cuda_time_ms(torch, B.spmv, reps)
    # each kind alone in a batch of its own (the same handles, formats and
    # shapes): the per-format breakdown of the launch above
    per_kind = {}
    for kd in kinds:
        idx = [k for k, e in enumerate(keep) if e[3] == kd]
        if not idx:
            continue
        Bk = dm.DynBatch(len(idx))
        for j, k in enumerate(idx):
            A, x, y, _ = keep[k]
            Bk.set(j, A, x, y, shape=shapes[k][0])
        kms = cuda_time_ms(torch, Bk.spmv, reps)
        kb = sum(shapes[k][1] for k in idx)
        knnz = sum(shapes[k][2] for k in idx)
        per_kind[kd] = {"matrices": len(idx), "formats": choices.get(kd, {}),
                        "us": round(kms * 1e3, 1), "gbs": round(kb / (kms * 1e-3) / 1e9, 1),
                        "g_entries_per_s": round(knnz / (kms * 1e-3) / 1e9, 1)}
        del Bk
    per_bytes = 0
    for P, x, y in per:
        i = P.info()
        per_bytes += algorithmic_bytes(dm.FORMATS[i.format], i.nrows, i.nnz, i.ndiag,
                                       i.ell_width, i.ell_width, i.hyb_coo_nnz)

    def per_matrix():
        for P, x, y in per:
            P.spmv(x, y)
    ms_per = cuda_time_ms(torch, per_matrix, reps)
    nnz = sum(k[0].info().nnz for k in keep)
    if tuple(kinds) == BATCH_KINDS and count == 64:
        workload = "64 FP64 matrices, 10k-500k rows (banded / power-law / uniform), seeds 100-163"
    else:
        workload = "%d FP64 matrices of the 64 (%s)" % (len(specs), " / ".join(kinds))
    return {"workload": workload + ("" if tune else ", %s, default tile shape" % fixed.upper()),
            "nnz": int(nnz), "batched_us": round(ms * 1e3, 1),
            "batched_gbs": round(total_bytes / (ms * 1e-3) / 1e9, 1),
            "per_matrix_us": round(ms_per * 1e3, 1),
            "per_matrix_gbs": round(per_bytes / (ms_per * 1e-3) / 1e9, 1),
            "speedup_vs_per_matrix": round(ms_per / ms, 3),
            "tuner_choices": choices, "tuner_shapes": shape_counts, "per_kind_alone": per_kind,
            "generate_s": round(gen_s, 1), "tune_s": round(tune_s, 1)}


def format_bytes(fmt: str, info, nnz: int, vb: int = 8) -> int:
    """Bytes of a format's arrays (what a conversion reads from its source or
    writes to its target): COO row, col, val; CSR rowptr, col, val; DIA
    offsets and ndiag x N values; ELL K x N columns and values; HYB's ELL
    part and its COO overflow."""
    N = int(info.nrows)
    if fmt == "coo":
        return (8 + vb) * nnz
    if fmt == "csr":
        return (4 + vb) * nnz + 4 * (N + 1)
    if fmt == "dia":
        return vb * int(info.ndiag) * N + 4 * int(info.ndiag)
    if fmt == "ell":
        return (4 + vb) * int(info.ell_width) * N
    return (4 + vb) * int(info.ell_width) * N + (8 + vb) * int(info.hyb_coo_nnz)


def bench_convert(dm, torch, N, r, c, v, reps: int = 3):
    """Create, the selector and every conversion pair (§III-B: source -> COO
    -> target, in place) on the 27-point stencil. Each is a blocking call
    (sizes are read back to the host between kernels), timed as wall time
    with the device idle before and after, median of `reps`. GB/s counts the
    source format's arrays read once and the target's written once."""
    nnz = int(r.size)
    out = {"workload": "27-point stencil, %d rows, %d entries, FP64" % (N, nnz), "pairs": {}}

    def wall(fn):
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        return float(np.median(ts))

    # create from device arrays: canonical input (check only) and shuffled (radix sort)
    dr, dc, dv = (torch.from_numpy(a).cuda() for a in (r, c, v))
    perm = torch.from_numpy(np.argsort(synth.uniform01(11, nnz), kind="stable")).cuda()
    sr, sc, sv = dr[perm].contiguous(), dc[perm].contiguous(), dv[perm].contiguous()
    del perm
    for name, args in (("create_sorted", (dr, dc, dv)), ("create_shuffled", (sr, sc, sv))):
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h = dm.dynmat_create(N, N, *args)
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
            del h
        t = float(np.median(ts))
        out[name] = {"us": round(t * 1e6, 1), "gbs": round(2 * 16 * nnz / t / 1e9, 1),
                     "bytes": 2 * 16 * nnz}
    del sr, sc, sv
    H = dm.dynmat_create(N, N, dr, dc, dv)
    t = wall(lambda: H.features())
    out["features_select"] = {"us": round(t * 1e6, 1), "gbs": round(8 * nnz / t / 1e9, 1),
                              "bytes": 8 * nnz}
    infos = {}
    for f in FMTS:
        H.convert(f)
        infos[f] = H.info()
    for src in FMTS:
        H.convert(src)
        for dst in FMTS:
            if dst == src:
                continue
            ts = []
            for _ in range(reps):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                H.convert(dst)
                torch.cuda.synchronize()
                ts.append(time.perf_counter() - t0)
                H.convert(src)
            t = float(np.median(ts))
            nb = format_bytes(src, infos[src], nnz) + format_bytes(dst, infos[dst], nnz)
            out["pairs"]["%s->%s" % (src, dst)] = {"us": round(t * 1e6, 1),
                                                   "gbs": round(nb / t / 1e9, 1), "bytes": nb}
    return out


def bench_small(dm, torch, n: int = 16, reps: int = 50):
    """The 16^3 configuration (4096 rows, 97,336 entries): every format's
    SpMV after an L2 flush (cold) and back to back (warm, the matrix resident
    in L2), 50 CG iterations on b = A 1 in the selected format, and the
    conversions. Small enough to be latency-bound: reported in microseconds
    and GB/s, not against the roofline."""
    N, r, c, v = synth.stencil27(n)
    x_host = synth.uniform_pm1(1, N)
    nnz = int(r.size)
    x = torch.from_numpy(x_host).cuda()
    y = torch.empty_like(x)
    flush = torch.ones(64 << 20, dtype=torch.float32, device="cuda")
    out = {"workload": "27-point stencil %d^3, FP64, x from seed 1" % n, "nrows": N, "nnz": nnz,
           "spmv": {}}
    s = torch.cuda.current_stream()
    handles = {}
    for f in FMTS:
        A = dm.dynmat_create(N, N, r, c, v)
        A.convert(f)
        handles[f] = A
        info = A.info()
        nb = algorithmic_bytes(f, N, nnz, int(info.ndiag), int(info.ell_width),
                               int(info.ell_width), int(info.hyb_coo_nnz))
        # Each product is timed between two events with the GPU kept busy
        # while the host enqueues it (the L2 flush, or a 25 us device-side
        # sleep when warm), so a microsecond kernel is not timed together with
        # the host's launch latency.
        cold, warm_t = [], []
        for mode, out_t in (("cold", cold), ("warm", warm_t)):
            for _ in range(reps):
                if mode == "cold":
                    l2_evict(flush)
                else:
                    torch.cuda._sleep(50_000)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(s)
                A.spmv(x, y)
                e1.record(s)
                torch.cuda.synchronize()
                out_t.append(e0.elapsed_time(e1))
        warm = float(np.median(warm_t))
        c_ms = float(np.median(cold))
        out["spmv"][f] = {"variant": int(info.spmv_variant), "bytes": nb,
                          "us_cold": round(c_ms * 1e3, 2), "gbs_cold": round(nb / c_ms / 1e6, 1),
                          "us_warm": round(warm * 1e3, 2), "gbs_warm": round(nb / warm / 1e6, 1)}
    chosen = FMTS[handles["coo"].features()["choice"]]
    ones = torch.ones(N, dtype=torch.float64, device="cuda")
    b = torch.empty_like(ones)
    handles[chosen].spmv(ones, b)
    xs = torch.zeros_like(b)
    res = {}

    def cg50():
        xs.zero_()
        res.update(handles[chosen].cg_solve(b, xs, tol=0.0, max_iters=50, check_every=50))
    ms = cuda_time_ms(torch, cg50, 10)
    out["cg_50_iterations"] = {"format": chosen, "ms": round(ms, 3),
                               "us_per_iteration": round(ms * 1e3 / 50, 2),
                               "iterations": res["iterations"]}
    conv = bench_convert(dm, torch, N, r, c, v, reps=5)
    out["convert"] = {k: conv[k] for k in ("create_sorted", "create_shuffled", "features_select",
                                          "pairs")}
    return out


def oracle_system_192(n: int = 192):
    """The 192^3 stencil from the generator with its CSR arrays and b = A 1
    from the CPU oracle (the inputs of bench_mixed's check)."""
    import oracle
    oracle.build(omp=True)
    N, r, c, v = synth.stencil27(n)
    a = {"rowptr": oracle.coo_to_csr(N, r), "col": c, "val": v}
    b = oracle.spmv("csr", N, N, a, np.ones(N), omp=True)
    return n, N, a, b


def serving_pool():
    """The served stream's irregular matrices (2M-row ones included)."""
    from paper_2209_06478_b300 import serve
    return serve.irregular_pool()


def bench_selector(dm, torch, N, r, c, v, x, reps: int = 20):
    """The format choice both ways (§IV-B run-time choice, §V-E tuner): the
    deterministic FEATURES rule (modelled bytes) and PROFILE mode (every
    admissible format and kernel variant timed), each with its SpMV time on
    the 128^3 stencil (CUDA events, L2 flushed before each call)."""
    import time as _t
    A = dm.dynmat_create(N, N, r, c, v)
    t0 = _t.perf_counter()
    f_feat = A.select_format(dm.SELECT_FEATURES)
    t_feat = _t.perf_counter() - t0
    t0 = _t.perf_counter()
    f_prof, var_prof = A.autotune()
    t_prof = _t.perf_counter() - t0
    flush = torch.ones(64 << 20, dtype=torch.float32, device="cuda")
    xt = torch.from_numpy(x).cuda()
    y = torch.empty_like(xt)
    s = torch.cuda.current_stream()

    def spmv_us(H):
        ts = []
        for _ in range(reps):
            l2_evict(flush)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            H.spmv(xt, y)
            e1.record(s)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) * 1e3)
        return round(float(np.median(ts)), 2)
    prof_us = spmv_us(A)
    B = dm.dynmat_create(N, N, r, c, v)
    B.convert(f_feat)
    B.tune_variant()
    feat_us = spmv_us(B)
    return {"features": {"format": FMTS[f_feat], "variant": int(B.info().spmv_variant),
                         "spmv_us": feat_us, "select_s": round(t_feat, 4)},
            "profile": {"format": FMTS[f_prof], "variant": int(var_prof), "spmv_us": prof_us,
                        "select_s": round(t_prof, 3)},
            "agree": FMTS[f_feat] == FMTS[f_prof]}


def bench_mixed(dm, torch, system, reps: int = 3):
    """27-point stencil 192^3 (7,077,888 rows), b = A 1, to 1e-10: FP32
    values + FP32 inner CG with FP64 residual / refinement vs plain FP64 CG,
    both in DIA on the same GPU. b comes from the CPU oracle, and the true
    relative residual of every returned x is recomputed by the oracle's FP64
    product (its OpenMP build, bit-identical to the serial one). The oracle's
    own CG is timed over 20 iterations beside it."""
    import oracle
    n, N, a_host, b_host = system
    A64 = dm.dynmat_create_stencil(n, 27, dm.DIA, dm.F64)
    A32 = dm.dynmat_create_stencil(n, 27, dm.DIA, dm.F32)
    assert A64.info().nrows == N
    b = torch.from_numpy(b_host).cuda()
    out = {"workload": "27-point stencil %d^3, b = A 1, tol 1e-10" % n, "nrows": N}
    for name, A, prec in (("fp64", A64, dm.CG_FP64), ("mixed_restarted", A32, dm.CG_MIXED),
                          ("mixed_reliable", A32, dm.CG_MIXED_RELIABLE)):
        x = torch.zeros_like(b)
        res = {}

        def run():
            x.zero_()
            res.update(A.cg_solve(b, x, tol=1e-10, max_iters=5000, precision=prec,
                                  inner_tol=1e-5, check_every=32))
        ms = cuda_time_ms(torch, run, reps, warmup=1)
        err = float(torch.linalg.norm(x - 1) / N ** 0.5)
        xh = x.cpu().numpy()
        ores = float(np.linalg.norm(b_host - oracle.spmv("csr", N, N, a_host, xh, omp=True))
                     / np.linalg.norm(b_host))
        out[name] = {"ms_per_solve": round(ms, 2), "solves_per_s": round(1e3 / ms, 3),
                     "iterations": res["iterations"], "outer": res["outer_iterations"],
                     "true_rel_residual": res["true_rel_residual"],
                     "oracle_true_rel_residual": ores,
                     "status": res["status"], "rms_error_vs_ones": err}
    for name in ("mixed_restarted", "mixed_reliable"):
        out["speedup_%s_vs_fp64" % name] = round(
            out["fp64"]["ms_per_solve"] / out[name]["ms_per_solve"], 3)
    # the CPU oracle's FP64 CG on the same system, a fixed 20 iterations (a
    # whole solve would take minutes), single-threaded as the oracle stands
    t0 = time.perf_counter()
    ref = oracle.cg(N, a_host["rowptr"], a_host["col"], a_host["val"], b_host, tol=0.0,
                    max_iters=20)
    dt = time.perf_counter() - t0
    out["cpu_oracle_cg"] = {"us_per_iteration": round(dt * 1e6 / max(ref["iterations"], 1), 1),
                            "iterations": ref["iterations"], "cores": 1,
                            "gpu_fp64_us_per_iteration": round(
                                out["fp64"]["ms_per_solve"] * 1e3 / out["fp64"]["iterations"], 1)}
    return out


def bench_split(dm, torch, n: int = 128, grids=((2, 2, 2), (4, 4, 4)), reps: int = 20):
    """The 128^3 stencil partitioned over a process grid as HPCG does (§IV-B,
    §V-E), each rank's product timed on this GPU as if it had one of its own
    (L2 flushed before every run), for the paper's versions:
      original: the local system matrix unsplit (remote columns appended) in
        CSR, after the halo gather;
      morpheus: local part DIA, remote part CSR;
      ghost: local part CSR, remote part COO;
      multi: the (local, remote) format pair whose split product is fastest
        for the rank (the per-process optimum).
    Each rank's product is captured once in a CUDA graph and replayed, so the
    times are device times (no host launch cost), as a native caller that
    replays its solver step would see them.
    The fixed versions run each format's automatic kernel variant; only the
    multi-format version tunes (formats and variants).
    Reported per version: the slowest rank's time (the parallel SpMV time)
    and the ratio original / version (> 1: faster than the original)."""
    flush = torch.ones(64 << 20, dtype=torch.float32, device="cuda")  # 256 MB
    s = torch.cuda.current_stream()

    def timed(fn):
        side = torch.cuda.Stream()
        side.wait_stream(s)
        with torch.cuda.stream(side):
            for _ in range(3):
                fn()  # first calls size the work buffers outside the capture
        s.wait_stream(side)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            fn()
        ts = []
        for k in range(reps + 3):
            l2_evict(flush)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(s)
            g.replay()
            e1.record(s)
            torch.cuda.synchronize()
            if k >= 3:
                ts.append(e0.elapsed_time(e1))
        return float(np.median(ts)) * 1e3

    out = {"workload": "27-point stencil %d^3 over a process grid, one rank's product per GPU" % n}
    N = n ** 3
    xh = synth.uniform_pm1(2, N)
    x = torch.from_numpy(xh).cuda()
    for grid in grids:
        P = grid[0] * grid[1] * grid[2]
        times = {"original": [], "morpheus": [], "ghost": [], "multi": []}
        tuned = {}
        choices = {}
        dia_unsplit = None
        for r in range(P):
            part = synth.partition_stencil(n, grid, r)
            nl, off, h = part["nloc"], part["offset"], part["halo"]
            lr, lc, lv = part["local"]
            rr, rc, rv = part["remote"]
            halo = torch.from_numpy(h).cuda()
            x_loc = x[off:off + nl]
            y = torch.empty(nl, dtype=torch.float64, device="cuda")
            # original: one CSR matrix over [local | halo] columns
            W = dm.dynmat_create(nl, nl + h.size, np.concatenate([lr, rr]),
                                 np.concatenate([lc, rc + nl]).astype(np.int32),
                                 np.concatenate([lv, rv]))
            if dia_unsplit is None:
                try:
                    W.convert("dia")
                    dia_unsplit = "converted"
                except dm.DynmatError as e:
                    dia_unsplit = dm.status_string(e.status)
            W.convert("csr")  # the automatic kernel variant: no per-rank tuning
            xw = torch.empty(nl + h.size, dtype=torch.float64, device="cuda")
            xw[:nl].copy_(x_loc)

            def original():
                dm.dynmat_gather(x, halo, xw[nl:])
                W.spmv(xw, y)
            times["original"].append(timed(original))
            x_ext = torch.empty(max(h.size, 1), dtype=torch.float64, device="cuda")
            for ver, lf, rf in (("morpheus", "dia", "csr"), ("ghost", "csr", "coo")):
                Al = dm.dynmat_create(nl, nl, lr, lc, lv)
                Al.convert(lf)
                Ar = dm.dynmat_create(nl, h.size, rr, rc, rv) if h.size else None
                if Ar is not None:
                    Ar.convert(rf)
                times[ver].append(timed(lambda: dm.dynmat_split_spmv(Al, Ar, halo, x, x_loc,
                                                                     x_ext, y)))
            # multi-format: the per-process optimum, by timing the whole split
            # product for each (local, remote) pair, each part's kernel
            # variant tuned; ranks with the same structure (halo size and
            # entry counts) share the choice
            key = (h.size, len(lr), len(rr))
            if key not in tuned:
                best = None
                for lf in ("dia", "ell", "csr"):
                    for rf in (("coo", "csr", "hyb") if h.size else ("-",)):
                        Al = dm.dynmat_create(nl, nl, lr, lc, lv)
                        try:
                            Al.convert(lf)
                        except dm.DynmatError:
                            continue
                        Al.tune_variant()
                        Ar = None
                        if h.size:
                            Ar = dm.dynmat_create(nl, h.size, rr, rc, rv)
                            Ar.convert(rf)
                            Ar.tune_variant()
                        t = timed(lambda: dm.dynmat_split_spmv(Al, Ar, halo, x, x_loc, x_ext, y))
                        if best is None or t < best[0]:
                            best = (t, lf, rf)
                tuned[key] = best
            t, lf, rf = tuned[key]
            name = "%s+%s" % (lf, rf)
            choices[name] = choices.get(name, 0) + 1
            times["multi"].append(t)
        worst = {k: max(v) for k, v in times.items()}
        out["%dx%dx%d" % grid] = {
            "ranks": P, "rows_per_rank": N // P,
            "us_slowest_rank": {k: round(v, 2) for k, v in worst.items()},
            "ratio_vs_original": {k: round(worst["original"] / v, 3) for k, v in worst.items()},
            "multi_format_choices": choices,
            "dia_of_unsplit_local_system_matrix": dia_unsplit}
    return out


def bench_hpcg(dm, torch, n: int = 128, levels: int = 4, reps: int = 3):
    """HPCG's preconditioned CG (§II-B) on the 27-point stencil n^3 with a
    `levels`-level V-cycle (colour-ordered symmetric Gauss-Seidel, injection)
    against plain CG on the same system (b = A 1, tol 1e-9), and one V-cycle
    alone."""
    M = dm.DynMG(n, n, n, levels=levels)
    A, _ = M.level(0)
    N = n ** 3
    ones = torch.ones(N, dtype=torch.float64, device="cuda")
    b = torch.empty_like(ones)
    A.spmv(ones, b)
    out = {"workload": "27-point stencil %d^3, %d-level V-cycle, b = A 1, tol 1e-9" % (n, levels)}
    for name, run in (("pcg", lambda x: M.pcg_solve(b, x, tol=1e-9, max_iters=1000)),
                      ("cg", lambda x: A.cg_solve(b, x, tol=1e-9, max_iters=5000))):
        x = torch.zeros_like(ones)
        res = run(x)
        ts = []
        for _ in range(reps):
            x.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res = run(x)
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        ms = float(np.median(ts)) * 1e3
        out[name] = {"iterations": res["iterations"], "status": res["status"],
                     "true_rel_residual": res["true_rel_residual"],
                     "ms_per_solve": round(ms, 3), "solves_per_s": round(1e3 / ms, 3),
                     "us_per_iteration": round(ms * 1e3 / max(res["iterations"], 1), 1),
                     "max_error_vs_ones": float(torch.max(torch.abs(x - 1.0)).item())}
    z = torch.empty_like(ones)
    out["vcycle_us"] = round(cuda_time_ms(torch, lambda: M.apply(b, z), 10) * 1e3, 1)
    out["pcg_vs_cg_time"] = round(out["cg"]["ms_per_solve"] / out["pcg"]["ms_per_solve"], 3)
    return out


def bench_diag(dm, torch, n: int = 128, reps: int = 20):
    """Diagonal extraction and update (§III-D; §IV-B: HPCG's CG test rewrites
    the matrix diagonal) on the 27-point stencil n^3 in every format: wall
    time per (blocking) call through the ABI, and GB/s over the bytes that
    locate and move each diagonal entry once."""
    N = n ** 3
    nnz = (3 * n - 2) ** 3
    below = (nnz - N) // 2  # entries left of the diagonal (symmetric pattern)
    index = {"dia": 0, "csr": 4 * (N + 1) + 4 * N, "ell": 4 * (below + N), "hyb": 4 * (below + N),
             "coo": 8 * nnz}
    peak, _ = measured_peaks()
    out = {"workload": "27-point stencil %d^3, FP64, every format; median of %d calls" % (n, reps),
           "bytes": "index bytes that find a(i,i) (DIA none; CSR the row pointer and one column per row; "
                    "ELL and HYB the slots up to the diagonal; COO every row and column index) + 8 B "
                    "read and 8 B written per row"}
    d = torch.empty(N, dtype=torch.float64, device="cuda")

    def wall_us(fn):
        for _ in range(3):
            fn()
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            fn()
            ts.append(time.perf_counter() - t0)
        return float(np.median(ts)) * 1e6

    for f in FMTS:
        A = dm.dynmat_create_stencil(n, 27, f)
        te = wall_us(lambda: A.diagonal(d))
        ok = bool(torch.all(d == 26.0).item())
        d2 = torch.full_like(d, 26.0)
        tu = wall_us(lambda: A.set_diagonal(d2))
        b = index[f] + 16 * N
        out[f] = {"extract_us": round(te, 1), "update_us": round(tu, 1),
                  "extract_gbs": round(b / te / 1e3, 1), "update_gbs": round(b / tu / 1e3, 1),
                  "extract_frac_of_measured_hbm": round(b / te / 1e3 / peak, 3),
                  "update_frac_of_measured_hbm": round(b / tu / 1e3 / peak, 3),
                  "diagonal_reads_26": ok}
        A.destroy()
        del A
    return out


def bench_serving(pool, rate: float = 400.0, count: int = 96):
    """Served stream: Poisson arrivals (seed 7), 7-/27-point stencils 32^3-160^3
    and banded / power-law SPD matrices of 50k-2M rows, random right-hand
    sides, tol 1e-10, 150 GB budget: mixed-precision batched vs plain FP64
    per-matrix (serial) path, and mixed batched with the online tuner (a
    short probe in the batch kernel when a matrix is first admitted). The
    mixed stream runs again under a budget of a few GB, which forces
    admission to wait and the matrix cache to evict."""
    from paper_2209_06478_b300 import serve
    reqs = serve.make_requests(count, rate)
    out = {"workload": "%d requests, Poisson %.0f/s, stencils 32^3-160^3 + irregular 50k-2M rows, "
                       "tol 1e-10, budget 150 GB, least estimated work admitted first, "
                       "8 batch slots" % (count, rate),
           "irregular_rows": sorted({q.size for q in reqs if not q.kind.startswith("stencil")})}
    # warm-up of both engines (graph instantiation, first launches) on a
    # short stream, so that neither timed run pays it
    warm = serve.make_requests(6, rate, seed=3, stencil_sizes=(32, 48))
    for mode in ("mixed_batched", "fp64_serial"):
        serve.serve(mode, warm, pool=pool)
    for mode in ("mixed_batched", "fp64_serial"):
        out[mode] = serve.serve(mode, reqs, pool=pool)
    # the same stream with the online tuner probing each new matrix at admission
    out["mixed_batched_online_tuned"] = serve.serve("mixed_batched", reqs, pool=pool,
                                                    online_tune=True)
    # shortest remaining work: ticks run only the least remaining work until
    # it fills the GPU, the other admitted solves are paused
    out["mixed_batched_srpt"] = serve.serve("mixed_batched", reqs, pool=pool, policy="srpt")
    tight = 6 * 10**9
    out["mixed_batched_budget_6gb"] = serve.serve("mixed_batched", reqs, budget=tight, pool=pool)
    out["solves_per_s_ratio"] = round(out["mixed_batched"]["solves_per_s"] /
                                      out["fp64_serial"]["solves_per_s"], 3)
    # latency ratios: serial FP64 over batched mixed (above 1: the batched
    # engine answers sooner)
    out["p50_ratio"] = round(out["fp64_serial"]["p50_ms"] / out["mixed_batched"]["p50_ms"], 3)
    out["p99_ratio"] = round(out["fp64_serial"]["p99_ms"] / out["mixed_batched"]["p99_ms"], 3)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="dynmat", choices=["dynmat", "reference"])
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--check-every", type=int, default=32)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batch, mixed-precision and serving measurements")
    ap.add_argument("--extras", default="",
                    help="comma-separated subset of selector,convert,small,batch,split,hpcg,"
                         "diag,mixed,serving to run (default all)")
    ap.add_argument("--batch-kinds", default=",".join(BATCH_KINDS),
                    help="batch extra: matrix kinds kept from the 64 (banded,powerlaw,uniform)")
    ap.add_argument("--batch-count", type=int, default=64,
                    help="batch extra: number of matrices kept")
    ap.add_argument("--batch-untuned", action="store_true",
                    help="batch extra: CSR with the default tile shape instead of the tuner's choice")
    ap.add_argument("--batch-format", choices=("csr", "ell", "dia"), default=None,
                    help="batch extra: every matrix in this format with its default tile shape, "
                         "instead of the tuner's choice")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_dynmat(args)


if __name__ == "__main__":
    main()
