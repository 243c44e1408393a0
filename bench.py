"""Benchmark of the (min,+) power path on GB300.

Prints ONE JSON line (rank 0).  Headline: add-min throughput of the (min,+)
product C = A (x) B at N = 16384 (synthetic operands, int16, entries uniform in
[0, 32], each infinite with probability 1/2, seeds 1 and 2), with inputs resident
in HBM; the step is one rd_minplus_gemm call (DPX product + fused minimum
reduction).  Operands (2 x 512 MiB) exceed the 129 MB L2, so no flush is needed
between steps.  Beside it, in the same line:
  * e2e: the same product through the C ABI with host operands, the pinned
    host->device copies of A and B and the device->host copy of C inside the
    timed region;
  * roofline of the product kernel against the DPX add-min peak;
  * time_to_period: the whole hot path (enumerate + build A(G), power until the
    first repeat, gamma_R closed form) for m = 3, 7, 9, with the oracle's time;
  * cpu_baseline: the oracle's product on a bounded sample of rows.

--impl reference times the oracle (the plain CPU restatement of the method) on
the same workload, one bounded row sample per step.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_HEAD = 16384
SEED_A, SEED_B = 1, 2
# Nominal DPX rate from unit counts and clock: 152 SMs x 64 __viaddmin_s16x2 lanes per clock x 2 add-mins per
# lane x 2070 MHz.  The roofline's peak is the measured one (rd_measure_addmin_peak, run by this script before
# the timed region); the nominal figure is printed beside it.
SMS, DPX_LANES_PER_CLK, ADDMIN_PER_LANE, SM_MAX_MHZ = 152, 64, 2, 2070.0
PEAK_GOPS = SMS * DPX_LANES_PER_CLK * ADDMIN_PER_LANE * SM_MAX_MHZ * 1e6 / 1e9
# DRAM bytes (read + write) per launch of the product kernel at N = 16384, from a one-pass ncu capture of
# dram__bytes_read.sum and dram__bytes_write.sum on that launch (8.60 GB read + 0.552 GB written).
GEMM_TRAFFIC_BYTES = 9.152e9
CONFIG_NAME = "synthetic dense (min,+) GEMM N=16384, int16 uniform[0,32], P(inf)=0.5"


def _measured_hbm_gbs() -> float:
    """The measured copy bandwidth of the GB300s (MEASURED_PEAKS.json beside this script, read + write
    bytes), else the earlier measurement of 6652.3 GB/s."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return 6652.3


HBM_GBS = _measured_hbm_gbs()


def max_over_ranks(value_ms: float, dist, device) -> float:
    """The slowest rank's time: the whole job is done when its last rank is."""
    if dist is None:
        return value_ms
    import torch

    t = torch.tensor([value_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, steps: int, ops_per_step: float, max_ms: float) -> float:
    """Whole-job rate in G per second: every rank did `steps` steps of `ops_per_step` in max_ms."""
    return world * steps * ops_per_step / (max_ms * 1e-3) / 1e9


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []
        self.reader = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.reader = threading.Thread(target=self._read, daemon=True)
            self.reader.start()
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            if self.reader is not None:
                self.reader.join(timeout=2)

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[3:7]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline_gemm(a: np.ndarray, b: np.ndarray, rows: int) -> dict:
    """The oracle's textbook product on the first `rows` rows of A against all of B."""
    import oracle

    n = b.shape[1]
    t0 = time.perf_counter()
    oracle.minplus_i16(a[:rows], b)
    dt = time.perf_counter() - t0
    ops = rows * a.shape[1] * n
    return {"value": ops / dt / 1e9, "unit": "G add-min/s", "cores": oracle.threads(), "kind": "oracle",
            "sample": f"rows 0..{rows - 1} of C = A (x) B at N={n} ({ops:.3g} add-mins, {dt:.1f} s)"}


def closed_form(r: dict, n: int) -> int:
    """gamma_R(n) from the boundary values and (k, p, q) (Prop. 7)."""
    k, p, q = r["k"], r["p"], r["q"]
    if n < k + p:
        return int(r["gamma"][n])
    return int(r["gamma"][k + (n - k) % p]) + q * ((n - k) // p)


def time_to_period(rd, torch, ms: list[int], with_oracle: bool) -> dict:
    """The whole hot path for each m: build A(G), power until the first repeat, closed form for n = 3..1000.

    The power step is the row-split one (A(G) (x) P_k from the row rules in two passes); its plan is
    built inside the timed region.  For comparison the dense x sparse step (rows per block R from
    the native autotuner, outside the timed region) is timed at m >= 7, and the dense DPX step at m = 9.
    One row-split product is also timed alone (CUDA events) against the measured HBM bandwidth:
    it moves (2 N + 2 X rows) x N x 2 bytes (B in, X out, X in, R out).
    """
    out = {}
    for m in ms:
        n = rd.state_count(m)
        ld = rd.padded_dim(n)
        kmax = 64
        work = rd.power_workspace(n, ld, kmax, 8)
        A = torch.empty((n, ld), dtype=torch.int16, device="cuda")
        rd.build_transfer(m, A)
        nnz = int((A[:, :n] != rd.RD_INF).sum().item())
        # one untimed pass (first touch of allocations, module load), then the timed one; N <= 128 runs
        # the single-CTA search of rd_power_until_periodic (no plan), larger N the row-split step
        small = n <= 128
        tuned = None
        if not small:
            # the native autotuner picks the passes' launch shape (outside the timed region); the plan
            # built inside the timed region then takes it from the library's tuning table
            tplan = rd.split_plan(m, x_ld=ld)
            T = torch.empty_like(A)
            tuned = rd.tune_split(tplan, A, T, reps=2)
            del tplan, T
        for _ in range(2):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rd.build_transfer(m, A)
            if small:
                r = rd.power_until_periodic(A, n, kmax, work)
            else:
                plan = rd.split_plan(m, x_ld=ld)
                r = rd.power_until_periodic_split(A, plan, kmax, work)
            gam = [closed_form(r, nn) for nn in range(3, 1001)]
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
        products = r["j"] - 1
        # the A(G) builder alone (a store stream: 2 N ld bytes written)
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        b0.record()
        for _ in range(3):
            rd.build_transfer(m, A)
        b1.record()
        torch.cuda.synchronize()
        build_ms = b0.elapsed_time(b1) / 3
        if small:
            plan = rd.split_plan(m, x_ld=ld)  # for the product timed alone below
        info = plan["info"]
        C = torch.empty_like(A)
        rd.split_minplus(plan, A, C)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            rd.split_minplus(plan, A, C)
        e1.record()
        torch.cuda.synchronize()
        prod_ms = e0.elapsed_time(e1) / 3
        moved = (2 * n + 2 * info.x_rows) * n * 2
        entry = {"N": n, "nnz_A": nnz, "k": r["k"], "p": r["p"], "q": r["q"], "products": products, "gpu_s": dt,
                 "step": ("single-CTA search (N <= 128)" if small else
                          f"row split j={info.j} (w {info.w1}/{info.w2}, slabs per CTA {info.k1}/{info.k2})"),
                 "us_per_power": dt / r["j"] * 1e6, "tuned_shape": tuned,
                 "build_ms": build_ms, "build_GBps": 2.0 * n * ld / (build_ms * 1e-3) / 1e9,
                 "build_frac_of_measured_hbm": 2.0 * n * ld / (build_ms * 1e-3) / 1e9 / HBM_GBS,
                 "split_product_ms": prod_ms, "split_x_rows": info.x_rows,
                 "split_product_GBps": moved / (prod_ms * 1e-3) / 1e9,
                 "split_product_frac_of_measured_hbm": moved / (prod_ms * 1e-3) / 1e9 / HBM_GBS,
                 "addmin_gops": products * nnz * n / dt / 1e9,
                 "dense_equivalent_gops": products * float(n) ** 3 / dt / 1e9, "gamma_R_n3_to_12": gam[:10]}
        del C
        if m >= 4:
            entry["remark13_holds_n5_to_1000"] = all(5 * gam[nn - 3] == 2 * (m + 1) * nn for nn in range(5, 1001, 5))
        if m >= 7:
            R, tune_ms = rd.sparse_tune(A, n, work)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rd.build_transfer(m, A)
            sp = rd.sparse_plan(A, n, n, R)
            s = rd.power_until_periodic_sparse(A, n, sp, kmax, work)
            torch.cuda.synchronize()
            entry["sparse_step_gpu_s"] = time.perf_counter() - t0
            entry["sparse_R"] = R
            entry["sparse_ms_per_product"] = tune_ms
            entry["sparse_matches_split"] = bool(np.array_equal(s["gamma"], r["gamma"]))
            del sp
        if m == 9:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rd.build_transfer(m, A)
            d = rd.power_until_periodic(A, n, kmax, work)
            torch.cuda.synchronize()
            entry["dense_step_gpu_s"] = time.perf_counter() - t0
            entry["dense_matches_split"] = bool((d["k"], d["p"], d["q"]) == (r["k"], r["p"], r["q"]))
        if with_oracle:
            import oracle

            if m <= 7:
                t0 = time.perf_counter()
                o = oracle.power_until_periodic(m, kmax=kmax)
                entry["oracle_s"] = time.perf_counter() - t0
                entry["oracle_matches"] = bool(o["found"] and (o["k"], o["p"], o["q"]) == (r["k"], r["p"], r["q"]))
                # the same search on one host thread, in a child process (OpenMP reads its thread count at start)
                code = (f"import sys, time; sys.path.insert(0, {ROOT!r}); import oracle; oracle.build(); "
                        f"t = time.perf_counter(); oracle.power_until_periodic({m}, kmax={kmax}); "
                        f"print(time.perf_counter() - t)")
                one = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                                     env=dict(os.environ, OMP_NUM_THREADS="1"), timeout=600)
                if one.returncode == 0:
                    entry["oracle_s_one_thread"] = float(one.stdout.strip().splitlines()[-1])
            else:
                rows = max(16, oracle.threads())  # one row per host thread at least, so every core works
                t0 = time.perf_counter()
                oracle.power_rows(m, np.arange(rows), r["j"])
                dt_o = time.perf_counter() - t0
                entry["oracle_s_extrapolated"] = dt_o * n / rows
                entry["oracle_sample"] = f"rows 0..{rows - 1} of A^1..A^{r['j']} ({dt_o:.1f} s), scaled by N/{rows}"
            entry["oracle_cores"] = oracle.threads()
        out[f"m={m}"] = entry
        del work, A, plan
        torch.cuda.empty_cache()
    return out


def small_case(rd, torch, m: int = 3, kmax: int = 32, reps: int = 20) -> dict:
    """The small case (m = 3, n = 3..30): microseconds per power and per search, A(G) built once.
    'single_cta' is rd_power_until_periodic, whose whole search runs in one CTA for N <= 128; for
    comparison the step kernels through rd_power_until_periodic_multi with one run, from a captured CUDA
    graph ('graph', 16 steps per graph, capture and instantiation inside each call) or launched
    directly ('direct', state read every 8 steps)."""
    A, n = rd.transfer_matrix(m)
    plan = rd.sparse_plan(A, n, n, 1)
    work = rd.power_workspace(n, A.stride(0), kmax, 8)
    runs = [(A, n, plan, work)]
    out = {"m": m, "N": n}
    single = rd.power_until_periodic(A, n, kmax, work)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        single = rd.power_until_periodic(A, n, kmax, work)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / reps
    out["single_cta"] = {"s_per_search": dt, "us_per_power": dt / single["j"] * 1e6}
    for name, gsteps in (("multi_graph", 16), ("multi_direct", 0)):
        res = rd.power_until_periodic_multi(runs, 1, kmax, graph_steps=gsteps)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            res = rd.power_until_periodic_multi(runs, 1, kmax, graph_steps=gsteps)
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / reps
        r = res[0]
        out[name] = {"s_per_search": dt, "us_per_power": dt / r["j"] * 1e6}
        assert (r["k"], r["p"], r["q"]) == (single["k"], single["p"], single["q"])
    out.update({"k": single["k"], "p": single["p"], "q": single["q"], "powers": single["j"],
                "gamma_n3_to_30": [closed_form(single, nn) for nn in range(3, 31)]})
    return out


def run_sparse_only(rd, torch, args) -> None:
    """One dense x sparse product A (x) P with P = A^2, repeated: the kernel of the power step."""
    m, R = args.sparse_only, args.rows_per_block
    A, n = rd.transfer_matrix(m)
    P = torch.empty_like(A)
    C = torch.empty_like(A)
    plan = rd.sparse_plan(A, n, n, R)
    rd.sparse_minplus(plan, A, P)  # P = A (x) A, dense enough to stand for a power
    for _ in range(args.warmup):
        rd.sparse_minplus(plan, P, C)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for s0, s1 in evs:
        s0.record()
        rd.sparse_minplus(plan, P, C)
        s1.record()
    torch.cuda.synchronize()
    ms = float(np.mean([s0.elapsed_time(s1) for s0, s1 in evs]))
    nnz = int((A[:, :n] != rd.RD_INF).sum().item())
    print(json.dumps({"sparse_only_m": m, "N": n, "R": R, "entries": plan["entries"], "nnz": nnz, "ms": ms,
                      "useful_addmin_gops": nnz * n / (ms * 1e-3) / 1e9,
                      "b_row_bytes_per_launch": plan["entries"] * n * 2,
                      "b_row_TBps": plan["entries"] * n * 2 / (ms * 1e-3) / 1e12}))


def run_batched_only(rd, torch, args) -> None:
    """The 64-product batch alone: `--warmup` untimed batched launches, then `--steps` timed ones."""
    from paper_2409_17658_gb300 import inputs

    sizes = inputs.log_uniform_sizes(64, 128, 8192, seed=4)
    probs = []
    for i, n in enumerate(sizes):
        ld = (n + 7) // 8 * 8
        A = inputs.matrix_torch(n, n, seed=1000 + 2 * i, ld=ld, device="cuda")
        B = inputs.matrix_torch(n, n, seed=1001 + 2 * i, ld=ld, device="cuda")
        probs.append((A, B, torch.empty_like(A), n, n, n))
    for _ in range(args.warmup):
        rd.minplus_gemm_batched(probs)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        rd.minplus_gemm_batched(probs)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(1, args.steps)
    ops = float(sum(n ** 3 for n in sizes))
    print(json.dumps({"batched_only": len(sizes), "ms": ms, "gops": ops / (ms * 1e-3) / 1e9,
                      "frac_of_peak": ops / (ms * 1e-3) / 1e9 / PEAK_GOPS}))


def run_split_only(rd, torch, args) -> None:
    """One row-split product A(G) (x) P with P = A(G)^2, repeated: the kernel pair of the power step."""
    m = args.split_only
    A, n = rd.transfer_matrix(m)
    P = torch.empty_like(A)
    C = torch.empty_like(A)
    plan = rd.split_plan(m, x_ld=A.stride(0))
    rd.split_minplus(plan, A, P)  # P = A (x) A, dense enough to stand for a power
    tuned = rd.tune_split(plan, P, C, reps=2) if args.tune else None
    for _ in range(args.warmup):
        rd.split_minplus(plan, P, C)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for s0, s1 in evs:
        s0.record()
        rd.split_minplus(plan, P, C)
        s1.record()
    torch.cuda.synchronize()
    ms = float(np.mean([s0.elapsed_time(s1) for s0, s1 in evs]))
    info = plan["info"]
    moved = (2 * n + 2 * info.x_rows) * n * 2
    print(json.dumps({"split_only_m": m, "N": n, "plan": info.as_dict(), "tuned": tuned, "ms": ms,
                      "bytes_per_product": moved,
                      "GBps": moved / (ms * 1e-3) / 1e9, "frac_of_measured_hbm": moved / (ms * 1e-3) / 1e9 / HBM_GBS}))


def run_search_only(rd, torch, args) -> None:
    """The period search with the row-split step at m = M, repeated (--tune: the plan's launch shape from the
    autotuner first): the kernel sequence of one power step, for profiling."""
    m = args.search_only
    A, n = rd.transfer_matrix(m)
    plan = rd.split_plan(m, x_ld=A.stride(0))
    if args.tune:
        P = torch.empty_like(A)
        C = torch.empty_like(A)
        rd.split_minplus(plan, A, P)
        rd.tune_split(plan, P, C, reps=2)
        del P, C
    kmax = 48
    work = rd.power_workspace(n, A.stride(0), kmax, 8)
    for _ in range(args.warmup):
        rd.power_until_periodic_split(A, plan, kmax, work)
    torch.cuda.synchronize()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = rd.power_until_periodic_split(A, plan, kmax, work)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    info = plan["info"]
    print(json.dumps({"search_only_m": m, "N": n, "k": r["k"], "p": r["p"], "q": r["q"], "powers": r["j"],
                      "shape": [info.w1, info.k1, info.w2, info.k2], "s_per_search": float(np.median(times)),
                      "ms_per_power": float(np.median(times)) * 1e3 / r["j"]}))


def gemv_leg(rd, torch, B, n: int, reps: int = 20) -> dict:
    """The matrix-vector form of the synthetic workload: y = x (x) B at N = 16384, against HBM bandwidth."""
    from paper_2409_17658_gb300 import inputs

    x = inputs.matrix_torch(1, n, seed=3, device="cuda")[0].contiguous()
    y = torch.empty(n, dtype=torch.int16, device="cuda")
    for _ in range(3):
        rd.minplus_gemv(x, B, y)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        rd.minplus_gemv(x, B, y)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    nbytes = n * B.stride(0) * 2 + 2 * n * 2  # B once, x in, y out
    return {"N": n, "ms": ms, "GB_per_s": nbytes / (ms * 1e-3) / 1e9, "bound": "hbm",
            "frac_of_measured_hbm": nbytes / (ms * 1e-3) / 1e9 / HBM_GBS, "addmin_gops": float(n) * n / (ms * 1e-3) / 1e9,
            "l2": "B is 512 MiB > L2; consecutive calls re-read it from HBM"}


def gemm_sweep(rd, torch, sizes=(1024, 2048, 4096, 32768)) -> dict:
    """The dense product at the sweep's other sizes (the headline size is the main line): the native
    autotuner picks the output tile and split-K factor per size class (outside the timed region), then
    CUDA events time the product as a caller launches it."""
    from paper_2409_17658_gb300 import inputs

    out = {}
    for n in sizes:
        A = inputs.matrix_torch(n, n, seed=SEED_A, device="cuda")
        B = inputs.matrix_torch(n, n, seed=SEED_B, device="cuda")
        C = torch.empty((n, n), dtype=torch.int16, device="cuda")
        reps = 2 if n > 16384 else 10
        tuned = rd.tune_gemm(A, B, C, reps=1 if n > 16384 else 3)
        rd.minplus_gemm(A, B, C)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            rd.minplus_gemm(A, B, C)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        gops = float(n) ** 3 / (ms * 1e-3) / 1e9
        out[f"N={n}"] = {"ms": ms, "gops": gops, "frac_of_peak": gops / PEAK_GOPS, "split_k": tuned["p"][0],
                         "tile": "128x128" if tuned["p"][1] else "128x256", "tuner_ms": tuned["ms"]}
        if n <= 4096:
            # the stream-K form: the resident CTAs share the (tile, k-tile) units evenly
            work = rd.minplus_gemm_streamk_workspace(n, n, n)
            C2 = torch.empty_like(C)
            rd.minplus_gemm_streamk(A, B, C2, work)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(reps):
                rd.minplus_gemm_streamk(A, B, C2, work)
            e1.record()
            torch.cuda.synchronize()
            ms_sk = e0.elapsed_time(e1) / reps
            gops_sk = float(n) ** 3 / (ms_sk * 1e-3) / 1e9
            out[f"N={n}"]["streamk"] = {"ms": ms_sk, "gops": gops_sk, "frac_of_peak": gops_sk / PEAK_GOPS,
                                        "same_result": bool(torch.equal(C, C2))}
            del work, C2
        del A, B, C
        torch.cuda.empty_cache()
    return out


def time_to_period_low_memory(rd, torch, m: int = 11, chunk_cols: int = 8192) -> dict:
    """The whole path for m = 11 (N = 191476, 73 GB per power) on one GPU: a 3-slot ring with A(G) built in
    its first slot, the row split's intermediate in column chunks, and the repeat verified by re-deriving
    the earlier power (it has left the ring).  One untimed pass, then the timed one (wall clock)."""
    torch.cuda.empty_cache()
    n = rd.state_count(m)
    ld = rd.padded_dim(n)
    kmax = 48
    work = rd.power_workspace(n, ld, kmax, 3)
    off0 = rd.power_slot(n, ld, kmax, work.numel(), 0)
    A = work[off0:off0 + n * ld * 2].view(torch.int16).view(n, ld)
    for _ in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rd.build_transfer(m, A)
        plan = rd.split_plan(m, chunk_cols=chunk_cols)
        r = rd.power_until_periodic_split(A, plan, kmax, work)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
    gam = [closed_form(r, nn) for nn in range(3, 1001)]
    out = {"N": n, "bytes_per_power": 2 * n * ld, "ring_slots": 3, "chunk_cols": chunk_cols, "k": r["k"],
           "p": r["p"], "q": r["q"], "gpu_s": dt, "products": r["j"] - 1 + r["k"] - 1,
           "gamma_R_n3_to_12": gam[:10],
           "cor12_holds_n10_to_1000": all(5 * gam[nn - 3] == 24 * nn for nn in range(10, 1001, 5)),
           "how": "3-slot ring (A(G) in slot 0), chunked intermediate, earlier power re-derived to verify"}
    del A, work, plan
    torch.cuda.empty_cache()
    return out


def batched_products(rd, torch, count: int = 64, seed: int = 4) -> dict:
    """64 independent products, N_i = round(exp(U[ln 128, ln 8192])) (seeded): one persistent
    batched launch against one launch per product, both on the same stream, results compared."""
    from paper_2409_17658_gb300 import inputs

    sizes = inputs.log_uniform_sizes(count, 128, 8192, seed=seed)
    ops = float(sum(n ** 3 for n in sizes))
    probs, refs = [], []
    for i, n in enumerate(sizes):
        ld = (n + 7) // 8 * 8
        A = inputs.matrix_torch(n, n, seed=1000 + 2 * i, ld=ld, device="cuda")
        B = inputs.matrix_torch(n, n, seed=1001 + 2 * i, ld=ld, device="cuda")
        probs.append((A, B, torch.empty_like(A), n, n, n))
        refs.append(torch.empty_like(A))
    stream = torch.cuda.current_stream()

    def one_by_one():
        for (A, B, _, n, _, _), R in zip(probs, refs):
            rd.minplus_gemm(A, B, R, n, n, n)

    def batched():
        rd.minplus_gemm_batched(probs)

    out = {"products": count, "sizes_min_median_max": [min(sizes), int(np.median(sizes)), max(sizes)],
           "addmins": ops}
    for name, fn in (("one_launch_per_product", one_by_one), ("batched_persistent", batched)):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 3
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out[name] = {"ms": ms, "gops": ops / (ms * 1e-3) / 1e9, "launches": count if name.startswith("one") else 2}
    out["speedup"] = out["one_launch_per_product"]["ms"] / out["batched_persistent"]["ms"]
    out["results_identical"] = bool(all(torch.equal(p[2][:, :p[4]], r[:, :p[4]]) for p, r in zip(probs, refs)))
    del probs, refs
    torch.cuda.empty_cache()

    # A(G) for m = 1..9 powered until periodic: all together (CUDA graph of 8 steps) vs one after another;
    # the large ones (m = 8, 9) with the row-split step, the others with the sparse step
    kmax, R = 64, 2
    runs = []
    for m in range(1, 10):
        A, n = rd.transfer_matrix(m)
        plan = rd.split_plan(m, x_ld=A.stride(0)) if m >= 8 else rd.sparse_plan(A, n, n, R)
        runs.append((A, n, plan, rd.power_workspace(n, A.stride(0), kmax, 8)))

    def one(A, n, plan, w):
        if "info" in plan:
            return rd.power_until_periodic_split(A, plan, kmax, w)
        return rd.power_until_periodic_sparse(A, n, plan, kmax, w)

    timings = {}
    for name in ("sequential", "together_graph", "together_graph_launches_per_phase"):
        # the multi-run search advances all runs one power per launch of its step kernel; the third
        # variant runs the same steps as launches per phase (products, normaliser, finalize, compare)
        if name.endswith("per_phase"):
            os.environ["RD_MULTI_STEP"] = "launches"
        for _ in range(2):  # first pass untimed
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if name == "sequential":
                res = [one(*run) for run in runs]
            else:
                res = rd.power_until_periodic_multi(runs, R, kmax, graph_steps=8)
            torch.cuda.synchronize()
            timings[name] = time.perf_counter() - t0
        os.environ.pop("RD_MULTI_STEP", None)
        timings[name + "_triples"] = [(r["k"], r["p"], r["q"]) for r in res]
    out["periods_m1_to_9"] = {"sequential_s": timings["sequential"], "together_graph_s": timings["together_graph"],
                              "together_launches_per_phase_s": timings["together_graph_launches_per_phase"],
                              "speedup": timings["sequential"] / timings["together_graph"],
                              # per step: one multi_step_kernel launch for the sparse runs (m = 1..7), and per
                              # row-split run (m = 8, 9) its two passes, finalize and compare
                              "launches_per_step": 1 + 4 * sum(1 for run in runs if "info" in run[2]),
                              "launches_how": "sparse runs m = 1..7: one multi_step_kernel launch; row-split runs "
                                              "m = 8, 9: two passes + finalize + compare each",
                              "same_results": (timings["sequential_triples"] == timings["together_graph_triples"] ==
                                               timings["together_graph_launches_per_phase_triples"]),
                              "triples": timings["together_graph_triples"]}
    # the runs that the persistent step kernel carries alone (m = 1..7, sparse step): one launch per step for
    # all seven, eight steps per replay of the captured graph, against each search on its own
    small = runs[:7]
    t_small = {}
    for name in ("sequential", "together"):
        for _ in range(2):  # first pass untimed
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if name == "sequential":
                res = [one(*run) for run in small]
            else:
                res = rd.power_until_periodic_multi(small, R, kmax, graph_steps=8)
            torch.cuda.synchronize()
            t_small[name] = time.perf_counter() - t0
        t_small[name + "_triples"] = [(r["k"], r["p"], r["q"]) for r in res]
    out["periods_m1_to_7_one_launch"] = {
        "sequential_s": t_small["sequential"], "together_graph_s": t_small["together"],
        "speedup": t_small["sequential"] / t_small["together"], "launches_per_step": 1,
        "launches_how": "one multi_step_kernel launch per step for all seven runs, 8 steps per graph replay; "
                        "alone, m <= 4 run the single-CTA search and m = 5..7 the sparse step",
        "same_results": t_small["sequential_triples"] == t_small["together_triples"]}
    del runs, small
    torch.cuda.empty_cache()
    return out


def query_mix(queries: int, seed: int):
    """Config 5's query mix: m uniform in {2..9}, n uniform in [3, 200]; one query in 20 is m = 10 with
    n = 0 mod 5 in [10, 200] (N(10)^2 int16 = 8.4 GB fits HBM).  Also unit exponential gaps for the arrivals."""
    from paper_2409_17658_gb300 import inputs

    x = inputs.splitmix64((np.uint64(seed) << np.uint64(32)) + np.arange(4 * queries, dtype=np.uint64))
    u = (x >> np.uint64(11)).astype(np.float64) / float(1 << 53)
    gaps = -np.log1p(-u[:queries])
    ms = (2 + (u[queries:2 * queries] * 8).astype(np.int64)).astype(np.int32)
    ns = (3 + (u[2 * queries:3 * queries] * 198).astype(np.int64)).astype(np.int64)
    ten = u[3 * queries:] < 0.05
    ms[ten] = 10
    ns[ten] = 10 + 5 * (ns[ten] % 39)
    return ms, ns, gaps


def serve_stream(rd, ms, ns, arrivals, budget_gb: float, server=None) -> dict:
    """Submits the queries at their arrival times to a server (a fresh one unless given) and waits for all."""
    sv = server or rd.Server(hbm_budget_bytes=int(budget_gb * (1 << 30)), kmax=128)
    try:
        tickets = []
        t0 = time.perf_counter()
        i, q = 0, len(ms)
        while i < q:
            now = time.perf_counter() - t0
            j = int(np.searchsorted(arrivals, now, side="right"))
            if j <= i:
                time.sleep(max(0.0, min(arrivals[i] - now, 0.001)))
                continue
            tickets.append(sv.submit(ms[i:j], ns[i:j]))
            i = j
        g, st, lat = sv.wait(np.concatenate(tickets), timeout_s=900)
        wall = time.perf_counter() - t0
        stats = sv.stats()
    finally:
        if server is None:
            sv.close()
    return {"gamma": g, "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "max_ms": float(lat.max() * 1e3), "queries_per_s": q / wall, "wall_s": wall,
            "all_ok": bool(np.all(st == rd.RD_OK)), "jobs": int(stats["jobs_admitted"]),
            "peak_gb": stats["bytes_peak"] / 2 ** 30}


def plain_stream(rd, ms, ns, arrivals) -> dict:
    """The plain path on the same stream: one rd_gamma_R call per query, in arrival order, one at a time, from
    a cleared cache (each m's first query runs its whole period search before the next query starts)."""
    rd.gamma_R_clear()
    q = len(ms)
    g = np.zeros(q, dtype=np.int64)
    lat = np.zeros(q)
    t0 = time.perf_counter()
    for i in range(q):
        now = time.perf_counter() - t0
        if arrivals[i] > now:
            time.sleep(arrivals[i] - now)
        g[i] = rd.gamma_R(int(ms[i]), int(ns[i]))
        lat[i] = time.perf_counter() - t0 - arrivals[i]
    wall = time.perf_counter() - t0
    return {"gamma": g, "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "max_ms": float(lat.max() * 1e3), "queries_per_s": q / wall, "wall_s": wall}


def serving(rd, queries: int = 3000, rates=(1e3, 1e4, 1e5, 1e6), seed: int = 7, budget_gb: float = 120.0) -> dict:
    """Config 5: Poisson streams of gamma_R(P_m box C_n) queries through the query server, swept over the
    offered rate.  Every rate starts a fresh server, so each m's first queries trigger its period search
    (searches of different m share the GPU step by step, admitted by HBM footprint) and the rest wait for
    it or are answered from its result.  Beside the sweep, at the highest rate: the plain path (one
    rd_gamma_R per query, one at a time, cleared cache) on the same stream, whose answers every served
    answer must equal; and a warm replay against a settled server.  Latency is submit to answer.
    """
    ms, ns, gaps = query_mix(queries, seed)
    out = {"queries": queries, "budget_gb": budget_gb, "mix": "m uniform 2..9, n uniform 3..200; 5 % m = 10, n = 0 mod 5"}
    sweep, answers = [], []
    for rate in rates:
        arrivals = np.cumsum(gaps / rate)
        r = serve_stream(rd, ms, ns, arrivals, budget_gb)
        answers.append(r.pop("gamma"))
        sweep.append({"offered_per_s": rate, **r})
    out["sweep"] = sweep
    arrivals = np.cumsum(gaps / rates[-1])
    plain = plain_stream(rd, ms, ns, arrivals)
    want = plain.pop("gamma")
    out["plain_at_max_rate"] = plain
    out["served_over_plain_at_max_rate"] = sweep[-1]["queries_per_s"] / plain["queries_per_s"]
    # the plain path without a cache (Algorithm 2 and the closed form for every query, one at a time), on a
    # bounded sample: the first queries of the stream, all arrived at once
    sample = 60
    uncached_ok = True
    t0 = time.perf_counter()
    for i in range(sample):
        rd.gamma_R_clear()
        uncached_ok &= rd.gamma_R(int(ms[i]), int(ns[i])) == want[i]
    dt = time.perf_counter() - t0
    out["plain_uncached_sample"] = {"queries": sample, "queries_per_s": sample / dt, "wall_s": dt,
                                    "m10_queries": int(np.sum(ms[:sample] == 10))}
    out["served_over_plain_uncached"] = sweep[-1]["queries_per_s"] / (sample / dt)
    out["answers_equal_plain"] = bool(uncached_ok and all(np.array_equal(a, want) for a in answers))
    tens = np.nonzero(ms == 10)[0]
    out["m10_cor12_holds"] = bool(all(5 * want[i] == 22 * ns[i] for i in tens))
    sv = rd.Server(hbm_budget_bytes=int(budget_gb * (1 << 30)), kmax=128)
    try:
        serve_stream(rd, ms, ns, np.zeros(queries), budget_gb, server=sv)  # settle every m
        warm = serve_stream(rd, ms, ns, arrivals, budget_gb, server=sv)
        warm.pop("gamma")
        out["warm_at_max_rate"] = warm
        out["restart_from_records"] = restart_from_records(rd, sv, ms, ns, arrivals, budget_gb, want)
    finally:
        sv.close()
    return out


def restart_from_records(rd, sv, ms, ns, arrivals, budget_gb: float, want) -> dict:
    """Checkpoint and resume: the settled server's relation records (first repeat and gamma table per m)
    go to a JSON file; a fresh server imports them and serves the same stream at the highest rate with no
    period search at all (jobs = 0).  The answers must equal the plain path's."""
    import tempfile

    from paper_2409_17658_gb300 import relations

    t0 = time.perf_counter()
    recs = [sv.export_relation(int(m)) for m in sorted(set(ms.tolist()))]
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "relations.json")
        relations.save(path, recs)
        nbytes = os.path.getsize(path)
        loaded = relations.load(path)
    fresh = rd.Server(hbm_budget_bytes=int(budget_gb * (1 << 30)), kmax=128)
    try:
        for r in loaded:
            fresh.import_relation(r)
        t_ckpt = time.perf_counter() - t0
        r = serve_stream(rd, ms, ns, arrivals, budget_gb, server=fresh)
    finally:
        fresh.close()
    g = r.pop("gamma")
    return {**r, "answers_equal_plain": bool(np.array_equal(g, want)), "records": len(recs), "file_bytes": nbytes,
            "export_save_load_import_ms": t_ckpt * 1e3}


def run_reference(args, rank, world) -> None:
    """--impl reference: the oracle on the same workload, one bounded row sample per step."""
    if rank != 0:
        return
    import oracle
    from paper_2409_17658_gb300 import inputs

    n = N_HEAD
    rows = oracle.threads()  # one output row per thread, so every core counted below is busy
    a = inputs.matrix(rows, n, seed=SEED_A)
    b = inputs.matrix_torch(n, n, seed=SEED_B, device="cpu").numpy()  # same values as inputs.matrix, multithreaded
    for _ in range(args.warmup):
        oracle.minplus_i16(a[:1], b)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.minplus_i16(a, b)
    dt = time.perf_counter() - t0
    ops = args.steps * rows * n * n
    value = ops / dt / 1e9
    line = {"metric": "(min,+) add-min GOPS and % of GB300 DPX/INT peak at N=16384; gamma_R time-to-period vs oracle",
            "value": value, "unit": "G add-min/s", "impl": "reference", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": CONFIG_NAME, "N": n, "sample_rows_per_step": rows},
            "cpu_baseline": {"value": value, "unit": "G add-min/s", "cores": min(rows, oracle.threads()), "kind": "oracle",
                             "sample": f"{rows} rows of C per step ({rows * n * n:.3g} add-mins)"},
            "e2e": {"value": value, "unit": "G add-min/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-period", action="store_true", help="skip the time-to-period leg")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle timings")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-products leg")
    ap.add_argument("--no-serving", action="store_true", help="skip the query-server leg")
    ap.add_argument("--streamk", action="store_true", help="with --gemm-only: time rd_minplus_gemm_streamk")
    ap.add_argument("--gemm-only", type=int, default=0, metavar="N",
                    help="time only the product at size N (used for profiler captures)")
    ap.add_argument("--sparse-only", type=int, default=0, metavar="M",
                    help="time only the dense x sparse product A(G) (x) A(G)^2 for m = M (profiler captures)")
    ap.add_argument("--rows-per-block", type=int, default=2, help="R of the sparse form for --sparse-only")
    ap.add_argument("--gemv-only", type=int, default=0, metavar="N",
                    help="time only the one-row product against an N x N operand (profiling aid)")
    ap.add_argument("--split-only", type=int, default=0, metavar="M",
                    help="time only the row-split product at m = M (profiling aid)")
    ap.add_argument("--search-only", type=int, default=0, metavar="M",
                    help="run only the row-split period search at m = M (profiling aid)")
    ap.add_argument("--tune", action="store_true",
                    help="with --split-only or --search-only: run the autotuner on the plan first")
    ap.add_argument("--batched-only", action="store_true", help="time only the 64-product batch (profiling aid)")
    ap.add_argument("--build-only", type=int, default=0, metavar="M",
                    help="time only the A(G) builder at m = M (profiling aid)")
    ap.add_argument("--multi-only", type=int, default=0, metavar="M",
                    help="time only the period searches of m = 1..M advanced together (profiling aid)")
    ap.add_argument("--tune-table", default="", metavar="PATH",
                    help="load a saved tuning table (JSON, paper_2409_17658_gb300.tuning) before running")
    ap.add_argument("--no-sweep", action="store_true", help="skip the dense sweep at the other sizes")
    args = ap.parse_args()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch

    import paper_2409_17658_gb300 as rd
    from paper_2409_17658_gb300 import build, inputs

    build.build()
    torch.cuda.set_device(local)
    if args.tune_table:
        from paper_2409_17658_gb300 import tuning

        tuning.load(args.tune_table)
    if args.sparse_only:
        return run_sparse_only(rd, torch, args)
    if args.split_only:
        return run_split_only(rd, torch, args)
    if args.search_only:
        return run_search_only(rd, torch, args)
    if args.batched_only:
        return run_batched_only(rd, torch, args)
    if args.multi_only:
        kmax, R = 64, 2
        runs = []
        for m in range(1, args.multi_only + 1):
            A, n = rd.transfer_matrix(m)
            plan = rd.split_plan(m, x_ld=A.stride(0)) if m >= 8 else rd.sparse_plan(A, n, n, R)
            runs.append((A, n, plan, rd.power_workspace(n, A.stride(0), kmax, 8)))
        for _ in range(max(args.warmup, 1)):
            rd.power_until_periodic_multi(runs, R, kmax, graph_steps=8)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            res = rd.power_until_periodic_multi(runs, R, kmax, graph_steps=8)
        torch.cuda.synchronize()
        print(json.dumps({"multi_only": args.multi_only, "s_per_search": (time.perf_counter() - t0) / args.steps,
                          "triples": [(r["k"], r["p"], r["q"]) for r in res]}))
        return
    if args.build_only:
        m = args.build_only
        n = rd.state_count(m)
        ld = rd.padded_dim(n)
        A = torch.empty((n, ld), dtype=torch.int16, device="cuda")
        for _ in range(max(args.warmup, 1)):
            rd.build_transfer(m, A)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            rd.build_transfer(m, A)
        e1.record()
        torch.cuda.synchronize()
        ms_ = e0.elapsed_time(e1) / args.steps
        print(json.dumps({"build_only": m, "N": n, "ms": ms_, "GBps": 2.0 * n * ld / (ms_ * 1e-3) / 1e9,
                          "frac_of_measured_hbm": 2.0 * n * ld / (ms_ * 1e-3) / 1e9 / HBM_GBS}))
        return
    if args.gemv_only:
        from paper_2409_17658_gb300 import inputs

        B = inputs.matrix_torch(args.gemv_only, args.gemv_only, seed=SEED_B, device="cuda")
        print(json.dumps({"gemv_only": args.gemv_only, **gemv_leg(rd, torch, B, args.gemv_only, reps=args.steps)}))
        return
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    n = args.gemm_only or N_HEAD
    A = inputs.matrix_torch(n, n, seed=SEED_A, device="cuda")
    B = inputs.matrix_torch(n, n, seed=SEED_B, device="cuda")
    C = torch.empty((n, n), dtype=torch.int16, device="cuda")
    mn = torch.empty(1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()

    if args.gemm_only and args.streamk:
        sk_work = rd.minplus_gemm_streamk_workspace(n, n, n)

        def product():
            rd.minplus_gemm_streamk(A, B, C, sk_work, min_out=mn)
    else:

        def product():
            rd.minplus_gemm(A, B, C, min_out=mn)

    for _ in range(max(args.warmup, 3)):
        product()
    torch.cuda.synchronize()
    # the roofline's denominator, measured on this GPU (a 17 ms register-resident DPX loop)
    with ClockSampler(local) as peak_clocks:
        peak = rd.measure_addmin_peak(trips=8192)
    peak["clocks"] = peak_clocks.summary()

    # ---- device-resident timed region: events around every launch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        start = torch.cuda.Event(enable_timing=True)
        stop = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        for i in range(args.steps):
            ev[i][0].record(stream)
            product()
            ev[i][1].record(stream)
        stop.record(stream)
        torch.cuda.synchronize()
    barrier()
    total_ms = max_over_ranks(start.elapsed_time(stop), dist, "cuda")
    per_launch_ms = float(np.mean([s.elapsed_time(e) for s, e in ev]))
    ops_per_step = float(n) ** 3
    value = job_throughput(world, args.steps, ops_per_step, total_ms)
    clk = clocks.summary()
    if args.gemm_only:
        if rank == 0:
            print(json.dumps({"gemm_only": n, "streamk": bool(args.streamk), "steps": args.steps,
                              "ms_per_launch": per_launch_ms,
                              "gops": ops_per_step / (per_launch_ms * 1e-3) / 1e9, "clocks": clk}))
        return
    a = A.cpu().numpy()
    b = B.cpu().numpy()

    # ---- end to end through the C ABI with host buffers: every step is one rd_minplus_gemm_host call,
    # which copies A and B in from pinned host memory, runs the product and copies C back out.  Steps
    # alternate between two streams with their own staging buffers, so one step's copies overlap the
    # neighbouring step's product.
    del C
    a_pin = torch.from_numpy(a).pin_memory()
    b_pin = torch.from_numpy(b).pin_memory()
    c_pin = [torch.empty((n, n), dtype=torch.int16).pin_memory() for _ in range(2)]
    wbytes = rd.minplus_gemm_host_work_bytes(n, n, n)
    works = [torch.empty(wbytes, dtype=torch.uint8, device="cuda") for _ in range(2)]
    e2e_streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    e2e_steps = max(2, min(args.steps, 6))
    for i in range(e2e_steps):  # one untimed pass: both streams, staging buffers and pinned pages warm
        rd.minplus_gemm_host(a_pin, b_pin, c_pin[i % 2], works[i % 2], stream=e2e_streams[i % 2])
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for st_ in e2e_streams:
        st_.wait_stream(stream)
    for i in range(e2e_steps):
        rd.minplus_gemm_host(a_pin, b_pin, c_pin[i % 2], works[i % 2], stream=e2e_streams[i % 2])
    for st_ in e2e_streams:
        stream.wait_stream(st_)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
    e2e_value = job_throughput(world, e2e_steps, ops_per_step, e2e_ms)
    C_check = torch.empty((2, n), dtype=torch.int16, device="cuda")
    rd.minplus_gemm(A[:2], B, C_check)
    assert np.array_equal(c_pin[0][:2].numpy(), C_check.cpu().numpy())
    del works, C_check

    extra = {}
    if rank == 0:
        extra["gemv"] = gemv_leg(rd, torch, B, n)
    if rank == 0 and not args.no_sweep:
        extra["gemm_sweep"] = gemm_sweep(rd, torch)
    if rank == 0 and not args.no_period:
        extra["time_to_period"] = time_to_period(rd, torch, [3, 7, 9, 10], with_oracle=not args.no_cpu)
        extra["time_to_period"]["m=11"] = time_to_period_low_memory(rd, torch)
        extra["small_case"] = small_case(rd, torch)
    if rank == 0 and not args.no_serving:
        extra["serving"] = serving(rd)  # its row-split plans take the shapes tuned above
    if rank == 0 and not args.no_batched:
        extra["batched"] = batched_products(rd, torch)
    if rank == 0:
        extra["tuning_table"] = rd.tune_table()
    if rank == 0 and not args.no_cpu:
        extra["cpu_baseline"] = cpu_baseline_gemm(a, b, rows=128)  # about 10 s of CPU work on 16 cores

    if rank == 0:
        achieved = ops_per_step / (per_launch_ms * 1e-3) / 1e9
        per_clk = peak["addmin_per_clk_per_sm"]
        peak_max = per_clk * peak["sm_count"] * SM_MAX_MHZ * 1e6 / 1e9  # measured rate per clock at the max clock
        roof = {"bound": "alu", "achieved": achieved, "peak": peak_max, "unit": "G add-min/s",
                "frac": achieved / peak_max, "traffic": GEMM_TRAFFIC_BYTES,
                "kernel": "minplus_gemm_kernel<false>", "per_launch_ms": per_launch_ms,
                "peak_basis": "measured",
                "peak_how": (f"rd_measure_addmin_peak: {per_clk:.2f} add-min/clk/SM (clock64 spans of a full wave "
                             f"of __viaddmin_s16x2 chains) x {peak['sm_count']} SMs x {SM_MAX_MHZ:.0f} MHz"),
                "peak_measured_run": {"addmin_per_clk_per_sm": per_clk, "gops_at_run_clock": peak["addmin_per_s"] / 1e9,
                                      "run_sm_mhz": peak["sm_mhz"], "ms": peak["ms"], "clocks": peak["clocks"]},
                "peak_nominal": PEAK_GOPS,
                "peak_nominal_formula": "152 SMs x 64 DPX s16x2 lanes/clk x 2 add-min x 2070 MHz",
                "frac_of_nominal": achieved / PEAK_GOPS}
        if clk.get("sm_mhz"):
            roof["frac_at_sampled_clock"] = achieved / (per_clk * peak["sm_count"] * clk["sm_mhz"] * 1e6 / 1e9)
        line = {"metric": "(min,+) add-min GOPS and % of GB300 DPX/INT peak at N=16384; gamma_R time-to-period vs oracle",
                "value": value, "unit": "G add-min/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "int16", "data": "synthetic",
                "config": {"workload": CONFIG_NAME, "N": n, "seeds": [SEED_A, SEED_B], "parallelism": f"replicas{world}",
                           "l2": "operands 2 x 512 MiB > 129 MB L2; no flush"},
                "frac_of_peak": value / world / peak_max,
                "e2e": {"value": e2e_value, "unit": "G add-min/s", "h2d_bytes_per_step": 2 * a.nbytes,
                        "d2h_bytes_per_step": a.nbytes, "steps": e2e_steps,
                        "how": "one rd_minplus_gemm_host call per step (pinned host A, B in; C out); steps "
                               "alternate two streams and staging buffers, so copies overlap the neighbouring "
                               "step's product"},
                "gpu_launches": 2 * args.steps,
                "roofline": roof, "clocks": clk}
        line.update(extra)
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
