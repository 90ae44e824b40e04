"""Benchmark of the balance-check hot path: balance-checked assignments per second.

Workload: n = 1000 units, n1 = 500, d = 1000 covariates (half N(0,1), a quarter
Bernoulli(0.3), a quarter lognormal(0,1), standardised), ridge-whitened, and one
step = one accepted pool of B = 200,000 Philox draws at q = 1e-3 (K = 200):
regenerate every assignment, score it, stream the selection, re-check the
candidates exactly and return the accepted keys. Inputs are synthetic.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl frr|reference]

``--impl reference`` times the FP64 CPU oracle on this machine's cores on a
bounded sample of the same workload (the paper ships no reusable reference
program; the oracle is the reference arm). Under torchrun every rank runs its
own draw ranges (weak scaling, no collective on the data path); rank 0 prints
one JSON line.
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
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
# library kernels per frr_select step of the precision workload (one chunk): k_sel_init,
# k_balance_tc, k_sel_level1, k_sel_keep, k_bits, k_recheck_tc, k_finish
LAUNCHES_PER_STEP = 7
sys.path.insert(0, str(ROOT))

METRIC = "balance-checked assignments/s at n=d=1000; split-BF16 vs FP32 path, same B300"
WORKLOAD = "precision_n1000_d1000"
L2_FLUSH_BYTES = 256 << 20


def _peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        return json.loads(p.read_text()), "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0, "sm_max_mhz": 2032.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 10 ms while the steps run. The sampler
    is started (and its first sample awaited) before the warm-up; summary() keeps the samples
    taken inside [t0, t1] (wall clock), or all of them when none falls inside."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.tmp = None
        self.window = None

    def __enter__(self):
        self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "10"],
                                         stdout=self.tmp, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        # the first sample marks a running sampler (nvidia-smi takes a moment to start)
        t0 = time.perf_counter()
        while self.proc is not None and time.perf_counter() - t0 < 5.0:
            self.tmp.flush()
            if Path(self.tmp.name).stat().st_size > 0:
                break
            time.sleep(0.01)
        return self

    def mark(self, t0: float, t1: float):
        """Wall-clock window (time.time()) of the timed steps."""
        self.window = (t0, t1)

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        self.tmp.flush()

    def summary(self) -> dict:
        import datetime
        rows = []
        try:
            for line in Path(self.tmp.name).read_text().splitlines():
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 10:
                    rows.append(parts)
        finally:
            os.unlink(self.tmp.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}

        def stamp(r):
            try:
                return datetime.datetime.strptime(r[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                return None

        inside = rows
        if self.window is not None:
            lo, hi = self.window
            w = [r for r in rows if (t := stamp(r)) is not None and lo - 0.005 <= t <= hi + 0.005]
            if w:
                inside = w
        sm = [float(r[2]) for r in inside if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in inside if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in inside for i in range(4) if r[6 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "samples_in_timed_steps": len(inside) if inside is not rows else 0}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# --------------------------------------------------------------- CPU oracle --
def oracle_zc(X):
    from oracle import oracle as O
    Zc, *_ = O.prep(X, "ridge", 0.1)
    return Zc


def oracle_rate(Zc, n1, seed, target_s: float, first: int = 0, full: int = 200_000):
    """Oracle draws/s on the first `full` draws, or on a sample sized to take about target_s
    seconds when they would take longer (an 8192-draw calibration: with fewer, the threads'
    start-up and the sort inflate the per-draw time)."""
    from oracle import oracle as O
    cal = min(8192, full)
    t0 = time.perf_counter()
    O.select(Zc, n1, seed, first, cal, q=1e-3)
    per = (time.perf_counter() - t0) / cal
    S = int(max(64, min(full, target_s / max(per, 1e-7))))
    t0 = time.perf_counter()
    O.select(Zc, n1, seed, first + cal, S, q=1e-3)
    dt = time.perf_counter() - t0
    return S / dt, S, O.threads()


def oracle_rate_1t(Zc, n1, seed, target_s: float, first: int = 0):
    """The same oracle selection on one host thread (balance with threads=1, then the sort)."""
    from oracle import oracle as O
    t0 = time.perf_counter()
    O.select_from_M(O.balance(Zc, n1, seed, first, 16, threads=1), first, q=1e-3)
    per = (time.perf_counter() - t0) / 16
    S = int(max(16, min(50_000, target_s / max(per, 1e-7))))
    t0 = time.perf_counter()
    O.select_from_M(O.balance(Zc, n1, seed, first + 16, S, threads=1), first + 16, q=1e-3)
    return S / (time.perf_counter() - t0), S


def oracle_full_mc() -> dict:
    """The whole n = d = 100 workload (2e5 draws, q = 0.01) through the FP64 oracle on all host
    cores: preparation, M of every draw and the selection."""
    from oracle import oracle as O
    from paper_2501_07642_b300.workloads import workload
    w = workload("mc_n100_d100")
    X = w.covariates()
    t0 = time.perf_counter()
    Zc, *_ = O.prep(X, w.whiten, 0.1)
    keys, _ = O.select(Zc, w.n1, w.philox_seed, 0, w.draws, q=w.q)
    dt = time.perf_counter() - t0
    return {"value": w.draws / dt, "unit": "draws/s", "s": dt, "draws": w.draws, "K": int(len(keys)),
            "cores": O.threads(), "workload": "mc_n100_d100 (n = d = 100, q = 0.01), every draw"}


def cpu_model() -> str:
    try:
        for line in Path("/proc/cpuinfo").read_text().splitlines():
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    from paper_2501_07642_b300.workloads import workload
    w = workload(WORKLOAD)
    Zc = oracle_zc(w.covariates())
    from oracle import oracle as O
    rates, samples = [], []
    # per-step sample: at most ref_step_s seconds, and the whole run within about ref_total_s;
    # its size comes from the first (calibrating) call and is kept for every step
    step_s = min(args.ref_step_s, args.ref_total_s / max(1, args.warmup + args.steps))
    _, S, cores = oracle_rate(Zc, w.n1, w.philox_seed, step_s, first=0)
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        O.select(Zc, w.n1, w.philox_seed, (i + 1) * 1_000_000, S, q=1e-3)
        r = S / (time.perf_counter() - t0)
        if i >= args.warmup:
            rates.append(r)
            samples.append(S)
    value = len(rates) / sum(1.0 / r for r in rates)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "draws/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(samples) / len(samples) / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": w.n, "n1": w.n1, "d": w.d, "q": w.q, "whiten": "ridge 0.1",
                       "draws_per_step": int(statistics.median(samples))},
            "cpu_baseline": {"value": value, "unit": "draws/s", "cores": cores, "kind": "oracle",
                             "sample": f"FP64 oracle select (M of every draw + sort) on {int(statistics.median(samples))} "
                                       f"draws per step of the {WORKLOAD} workload"},
            "e2e": {"value": value, "unit": "draws/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# -------------------------------------------------------------------- GPU --
def run_frr(args):
    import torch
    import torch.distributed as dist

    from paper_2501_07642_b300 import frr
    from paper_2501_07642_b300.workloads import workload

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl")
    w = workload(WORKLOAD)
    X = w.covariates()
    B, q = w.draws, w.q
    K = math.ceil(q * B - 1e-9 * q * B)
    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    peaks, peak_kind = _peaks()

    precisions = [p for p in args.precision.split(",") if p]
    results = {}
    draw_base = rank * (1 << 40)  # disjoint draw ranges per rank
    for prec in precisions:
        try:
            ctx = frr.Context(X, w.n1, precision=prec, whiten="ridge", ridge=0.1, stream=stream)
        except frr.FrrError as e:
            results[prec] = {"error": str(e)}
            continue
        keys = torch.empty(K, dtype=torch.int64, device="cuda")
        m64 = torch.empty(K, dtype=torch.float64, device="cuda")
        try:
            frr.frr_select(ctx, w.philox_seed, draw_base, B, q=q, keys_out=keys, M64_out=m64, cap=K)
        except frr.FrrError as e:
            results[prec] = {"error": str(e)}
            ctx.close()
            continue
        step_ms, bal_ms, sel_ms, rck_ms = [], [], [], []
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        with ClockSampler(torch.cuda.current_device()) as clk:
            t_wall = time.perf_counter()
            n_warm = args.warmup
            i = 0
            t_timed0 = None
            while i < n_warm + args.steps:
                if i == n_warm:
                    t_timed0 = time.time()
                with torch.cuda.stream(stream):
                    flush.zero_()  # L2 flush between steps, outside the timed events
                    ev0.record(stream)
                first = draw_base + (i + 1) * B
                frr.frr_select(ctx, w.philox_seed, first, B, q=q, keys_out=keys, M64_out=m64, cap=K)
                ev1.record(stream)  # (on the library's stream; no stream switch inside the timed interval)
                ev1.synchronize()
                i += 1
                if i > n_warm:
                    step_ms.append(ev0.elapsed_time(ev1))
                    stt = frr.frr_last_stats(ctx)
                    bal_ms.append(stt["ms_balance"])
                    sel_ms.append(stt["ms_select"])
                    rck_ms.append(stt["ms_recheck"])
            torch.cuda.synchronize()
            clk.mark(t_timed0, time.time())
            wall = time.perf_counter() - t_wall
        stats = frr.frr_last_stats(ctx)
        total_ms = sum(step_ms)
        if ws > 1:
            t = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            total_ms = float(t.item())
        # end to end through the public API with host buffers: upload X from pinned
        # memory, prepare, select, read the keys back
        e2e = None
        if args.e2e:
            Xp = torch.from_numpy(X).pin_memory().numpy()
            hk = np.empty(K, dtype=np.uint64)
            hm = np.empty(K, dtype=np.float64)
            e2e_t = []
            for i in range(max(1, args.e2e_steps) + 1):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                c2 = frr.Context(Xp, w.n1, precision=prec, whiten="ridge", ridge=0.1)
                frr.frr_select(c2, w.philox_seed, draw_base + (1 << 30) + i * B, B, q=q, keys_out=hk, M64_out=hm, cap=K)
                c2.close()
                if i > 0:
                    e2e_t.append(time.perf_counter() - t0)
            e2e = {"value": ws * B / statistics.median(e2e_t), "unit": "draws/s",
                   "h2d_bytes_per_step": int(X.nbytes), "d2h_bytes_per_step": int(K * 16),
                   "includes": "frr_init (X upload, FP64 prep) + frr_select + key read-back"}
        results[prec] = {"value": ws * B * args.steps / (total_ms / 1e3), "ms_per_step": total_ms / args.steps,
                         "ms_per_step_median": statistics.median(step_ms), "ms_per_step_min": min(step_ms),
                         "ms_per_step_max": max(step_ms),
                         "ms_balance": statistics.mean(bal_ms), "ms_select": statistics.mean(sel_ms),
                         "ms_recheck": statistics.mean(rck_ms), "clocks": clk.summary(), "stats": stats, "e2e": e2e,
                         "wall_s": wall}
        ctx.close()

    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank != 0:
        return
    ok = [p for p in precisions if "value" in results.get(p, {})]
    if not ok:
        print(json.dumps({"metric": METRIC, "error": {p: results[p].get("error") for p in precisions}}))
        sys.exit(1)
    prim = ok[0]
    r = results[prim]
    n, d, n1 = w.n, w.d, w.n1
    f32_peak = fp32_lane_peak() if "f32" in ok else None

    def roofline(path, res):
        if path == "split_bf16":
            flops = 2.0 * 2.0 * n * d  # two BF16 parts, dense 0/1 x Zc per draw (multiply-add = 2)
            achieved = flops * B / (res["ms_balance"] / 1e3) / 1e12
            peak = peaks["bf16_tflops"]
            return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                    "traffic": tc_traffic(B, WORKLOAD), "kernel": "k_balance_tc",
                    "peak_source": f"bf16_tflops (burst, {peak_kind})", "flop_per_draw": flops}
        # FP32 CUDA-core path: the algorithmic work is n1 * d additions per draw (the treated rows;
        # the kernel executes n * d predicated ones), against the FP32 lane rate measured with a
        # cuBLAS FP32 GEMM in this run (one lane operation per multiply-add)
        adds = float(n1) * d
        achieved = adds * B / (res["ms_balance"] / 1e3) / 1e12
        return {"bound": "alu", "achieved": achieved, "peak": f32_peak, "unit": "Tadd/s", "frac": achieved / f32_peak,
                "traffic": None, "kernel": "k_balance_f32",
                "peak_source": "FP32 lane operations/s of a cuBLAS FP32 GEMM (8192^3, TF32 off), measured in this run",
                "adds_per_draw": adds, "executed_adds_per_draw": float(n) * d,
                "executed_frac": 2.0 * achieved / f32_peak}

    roof = roofline(prim, r)
    dtype = "bf16" if prim == "split_bf16" else "f32"
    for p in ok:
        results[p]["roofline"] = roofline(p, results[p])
    dist_line = distance_bench(peaks["bf16_tflops"]) if args.distance else None
    batch_line = batched_bench(args.batched_reps) if args.batched else None
    stream_line = stream_bench() if args.stream else None
    cpu = None
    if args.cpu_baseline:
        Zc = oracle_zc(X)
        rate, S, cores = oracle_rate(Zc, n1, w.philox_seed, args.cpu_s, full=B)
        rate1, S1 = oracle_rate_1t(Zc, n1, w.philox_seed, args.cpu_s / 4, first=10_000_000)
        cpu = {"value": rate, "unit": "draws/s", "cores": cores, "kind": "oracle",
               "sample": (f"FP64 oracle select (M of every draw + sort) on "
                          + (f"all {S} draws of one step" if S == B else f"{S} of the {B} draws of a step")
                          + f" of the {WORKLOAD} workload"),
               "single_thread": {"value": rate1, "sample": f"{S1} draws on one thread"},
               "mc_n100_d100_full": oracle_full_mc(),
               "cpu_model": cpu_model(), "nproc": os.cpu_count()}
    line = {"metric": METRIC, "value": r["value"], "unit": "draws/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype, "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": n, "n1": n1, "d": d, "draws_per_step": B, "q": q, "K": K,
                       "whiten": "ridge 0.1", "path": prim, "l2": "flushed (256 MiB write) between timed steps"},
            "paths": {p: ({k: results[p][k] for k in ("value", "ms_per_step", "ms_per_step_median", "ms_per_step_min",
                                                       "ms_per_step_max", "ms_balance", "ms_select", "ms_recheck",
                                                       "roofline")}
                          if "value" in results[p] else results[p])
                      for p in precisions},
            "roofline": roof, "cpu_baseline": cpu, "e2e": r["e2e"], "gpu_launches": LAUNCHES_PER_STEP * args.steps * ws,
            "clocks": {k: r["clocks"][k] for k in ("sm_mhz", "sm_max_mhz", "reasons", "samples", "samples_in_timed_steps")},
            "selection": {k: r["stats"][k] for k in ("candidates", "accepted", "max_rel_err", "max_err_over_band",
                                                     "band_violations", "parity_at_risk")},
            "fast_distance": dist_line, "batched": batch_line, "stream": stream_line}
    print(json.dumps(line), flush=True)



def fp32_lane_peak(size: int = 8192, reps: int = 5) -> float:
    """FP32 lane operations per second (T/s) of this GPU, measured: a cuBLAS FP32 GEMM with TF32
    off does one FP32 multiply-add per lane operation; best of `reps` after two warm-ups."""
    import torch
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        a = torch.randn(size, size, device="cuda")
        b = torch.randn(size, size, device="cuda")
        for _ in range(2):
            torch.mm(a, b)
        best = float("inf")
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.mm(a, b)
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        del a, b
        torch.cuda.empty_cache()
        return float(size) ** 3 / (best / 1e3) / 1e12
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev


def distance_bench(peak_tflops: float, n: int = 16384, d: int = 768, reps: int = 5) -> dict:
    """fast_distance on n x n pairs of d-dimensional FP32 rows (device in / out), one call =
    operand split, norms and the tensor-core kernel; median of `reps` calls after 2 warm-ups."""
    import torch

    from paper_2501_07642_b300 import frr

    g = torch.Generator(device="cuda").manual_seed(768)
    X = torch.randn((n, d), device="cuda", generator=g)
    Y = torch.randn((n, d), device="cuda", generator=g)
    D = torch.empty((n, n), device="cuda")
    for _ in range(2):
        frr.frr_fast_distance(X, Y, D_out=D)
    ts = []
    for _ in range(reps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        frr.frr_fast_distance(X, Y, D_out=D)
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms = statistics.median(ts)
    dp = 64 * ((d + 63) // 64)
    executed = 2.0 * n * n * 3 * dp  # three BF16 products per FP32 product (split operands)
    del X, Y, D
    torch.cuda.empty_cache()
    return {"workload": f"embedding_n{n}_m{n}_d{d}", "ms_per_call": ms,
            "pairs_per_s": n * n / (ms / 1e3),
            "roofline": {"bound": "tensor", "achieved": executed / (ms / 1e3) / 1e12, "peak": peak_tflops,
                         "unit": "TFLOP/s", "frac": executed / (ms / 1e3) / 1e12 / peak_tflops,
                         "flop_per_pair": 2.0 * 3 * dp, "note": "whole call (split + norms + kernel)"},
            "fp32_equivalent_tflops": 2.0 * n * n * d / (ms / 1e3) / 1e12,
            "output_gbs": n * n * 4 / (ms / 1e3) / 1e9}


def batched_bench(reps: int = 3) -> dict:
    """frr_batch_run over the 256-experiment batched workload (n log-uniform on [50, 2000],
    d on [10, 500], 1e5 draws and q = 0.01 each, then each experiment's randomization test
    over its 201-point tau grid): batched preparation, one persistent balance launch per
    class of n (autotuned, replayed as one CUDA graph), per-experiment selection and test;
    host covariates and outcomes, host results; median of `reps` runs after one warm-up run
    (which also tunes)."""
    from paper_2501_07642_b300 import frr
    from paper_2501_07642_b300.workloads import batched_workloads, outcome

    ws = batched_workloads(256)
    exps = []
    for w in ws:
        X = w.covariates()
        # outcome with no treatment effect (the test's w_obs is the first accepted key)
        Y = outcome(X, np.zeros(w.n), 0.0, w.y_seed)
        exps.append(dict(X=X, n1=w.n1, whiten=w.whiten, ridge=w.ridge, seed=w.philox_seed, B=w.draws, q=w.q,
                         cap=2048, Y=Y, tau=w.tau_grid, alpha=0.05))
    frr.frr_batch_run(exps, autotune=True)
    runs = []
    for _ in range(reps):
        t0 = time.perf_counter()
        _, st = frr.frr_batch_run(exps, autotune=True)
        runs.append((time.perf_counter() - t0, st))
    runs.sort(key=lambda r: r[0])
    dt, st = runs[len(runs) // 2]
    return {"workload": "batched_256", "experiments": 256, "draws": int(st["draws"]), "s_per_batch": dt,
            "draws_per_s": st["draws"] / dt, "ms_prep": st["ms_init"], "ms_balance": st["ms_balance"],
            "ms_select_and_tests": st["ms_select"], "randomization_tests": "201-point tau grid per experiment",
            "note": "wall time of frr_batch_run with host inputs and outputs; the selection and tests are issued "
                    "while the balance runs, and ms_select_and_tests is the wall time beyond the balance's device time"}


def stream_bench() -> dict:
    """The streaming workload (stream_n1000_d1000): 1e8 draws in 1e6-draw chunks through
    frr_stream_begin / frr_stream_chunk / frr_stream_end at q = 1.2e-5 (K = 1200), split BF16;
    wall time of the whole stream after a two-chunk warm-up stream, device inputs resident."""
    import torch
    from paper_2501_07642_b300 import frr
    from paper_2501_07642_b300.workloads import workload

    w = workload("stream_n1000_d1000")
    X = w.covariates()
    K = math.ceil(w.q * w.draws - 1e-9 * w.q * w.draws)
    with frr.Context(X, w.n1, precision="split_bf16", whiten=w.whiten, ridge=w.ridge) as ctx:
        frr.frr_stream_begin(ctx, w.philox_seed, 2 * w.chunk, q=w.q)
        for c in range(2):
            frr.frr_stream_chunk(ctx, (1 << 40) + c * w.chunk, w.chunk)
        frr.frr_stream_end(ctx, 4096)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        frr.frr_stream_begin(ctx, w.philox_seed, w.draws, q=w.q)
        for c in range(w.draws // w.chunk):
            frr.frr_stream_chunk(ctx, c * w.chunk, w.chunk)
        keys, _ = frr.frr_stream_end(ctx, 2 * K)
        dt = time.perf_counter() - t0
        st = frr.frr_last_stats(ctx)
    return {"workload": "stream_n1000_d1000", "draws": w.draws, "chunk": w.chunk, "K": int(len(keys)),
            "s": dt, "draws_per_s": w.draws / dt, "candidates_rechecked": int(st["candidates"]),
            "ms_balance": st["ms_balance"], "ms_select": st["ms_select"], "ms_recheck": st["ms_recheck"],
            "note": "wall time of the stream (one read-back per chunk bounds the retained set)"}


def tc_traffic(B, workload_name):
    """DRAM bytes per k_balance_tc launch from the committed ncu summary, or None when the
    kernel's sources changed since the capture, or the workload or launch size differs."""
    md = ROOT / "profiles" / "k_balance_tc_precision_n1000_d1000.md"
    try:
        text = md.read_text()
        rec = json.loads(text[text.rindex("```json") + 7:text.rindex("```")])
        h = hashlib.sha256()
        for f in rec["sources"]:
            h.update((ROOT / f).read_bytes())
        if (h.hexdigest() != rec["source_sha256"] or int(rec["draws_per_launch"]) != int(B)
                or rec.get("workload") != workload_name):
            return None
        return int(rec["dram_bytes_per_launch"])
    except (OSError, ValueError, KeyError):
        return None


def main():
    global WORKLOAD
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("frr", "reference"), default="frr")
    ap.add_argument("--precision", default="split_bf16,f32")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--cpu-s", type=float, default=20.0)
    ap.add_argument("--ref-step-s", type=float, default=8.0)
    ap.add_argument("--ref-total-s", type=float, default=120.0)
    ap.add_argument("--no-e2e", dest="e2e", action="store_false")
    ap.add_argument("--e2e-steps", type=int, default=15)
    ap.add_argument("--no-distance", dest="distance", action="store_false")
    ap.add_argument("--no-batched", dest="batched", action="store_false")
    ap.add_argument("--no-stream", dest="stream", action="store_false")
    ap.add_argument("--workload", default=WORKLOAD,
                    help="workload of the main leg (for profiling other shapes; the headline is the default)")
    ap.add_argument("--batched-only", action="store_true",
                    help="run only the 256-experiment batched leg and print its record (for profiling)")
    ap.add_argument("--batched-reps", type=int, default=3)
    args = ap.parse_args()
    WORKLOAD = args.workload
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.batched_only:
        print(json.dumps({"batched": batched_bench(args.batched_reps)}), flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_frr(args)


if __name__ == "__main__":
    main()
