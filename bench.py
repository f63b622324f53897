"""Benchmark of the loop-program hot path on GB300.

One step = one run of the six-loop program (init, GEMM, scale-add, transpose, row
sums, Frobenius norm) on n x n binary32 matrices under the all-GPU gene, through
the C ABI (prog_run).  Default workload: n = 4096 (the size of the all-64-genes
configuration), GEMM as the three-term split-bfloat16 product with binary32
accumulation (the path that meets 1e-6).  value = 2 n^3 / step time (TFLOP/s of
the whole program).  Inputs never leave the device inside the timed region for
`value`; `e2e` repeats the measurement with A, B, C0 coming from pinned host
memory and the results (row sums, norm) read back every step.

Launch: python bench.py [--gpus N --steps K --warmup W]; for N > 1 under
torch.distributed.run, each rank runs its own replica on its own GPU (replicas
only: the path has no exchange step); value sums the ranks' work over the max
time.  --impl reference times the FP64 CPU oracle on a bounded sample instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

PREC = {"fp32_simt": 0, "bf16": 1, "bf16x3": 2, "bf16x6": 3, "fp8": 4}
PRODUCTS = {"fp32_simt": 1, "bf16": 1, "bf16x3": 3, "bf16x6": 6, "fp8": 1}
FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        d["source"] = "measured"
        return d
    d = dict(FALLBACK)
    d["source"] = "fallback"
    return d


class Clocks:
    """Samples nvidia-smi every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark(self):
        return time.time()

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self, t0=None, t1=None):
        """Median SM clock and active throttle reasons of the samples taken in [t0, t1]."""
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ts, l in self.lines:
            if t0 is not None and not (t0 <= ts <= t1):
                continue
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def profile_traffic(kernel_file: str, name: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the
    current source of the kernel (else None)."""
    path = os.path.join(ROOT, "profiles", name)
    src = os.path.join(ROOT, "paper_1806_01430_gb300", "csrc", kernel_file)
    if not (os.path.exists(path) and os.path.exists(src)):
        return None
    text = open(path).read()
    m = re.search(r"source_sha256:\s*([0-9a-f]{64})", text)
    t = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not (m and t):
        return None
    if hashlib.sha256(open(src, "rb").read()).hexdigest() != m.group(1):
        return None
    return float(t.group(1))


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _reduce(x: float, op: str) -> float:
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def allmax(world, x: float) -> float:
    """Max over ranks (the slowest rank's time is the job's time)."""
    return x if world == 1 else _reduce(x, "max")


def allsum(world, x: float) -> float:
    """Sum over ranks (the whole job's work)."""
    return x if world == 1 else _reduce(x, "sum")


# ---- CPU oracle baseline -------------------------------------------------------------------

def oracle_rows(n: int, seed: int, r: int, B) -> float:
    """Seconds the FP64 oracle takes for rows [0, r) of the six-loop program: INIT of
    those rows of A and C, their GEMM rows (against the full B, initialised outside),
    scale-add, transpose, row sums and norm."""
    import oracle
    t0 = time.perf_counter()
    A = oracle.init_matrix(seed, 0, r, n)
    C0 = oracle.init_matrix(seed, 2, r, n)
    C = oracle.gemm(A, B, C0, 1.5, 0.5)
    D = oracle.axpy(C, 2.0, A)
    E = oracle.transpose(D)
    oracle.rowsum(E)
    oracle.frobenius(E)
    return time.perf_counter() - t0


def oracle_calibrate(n: int, seed: int, target_s: float):
    """Rows r whose oracle time is about target_s (at most n); returns (r, B)."""
    import oracle
    B = oracle.init_matrix(seed, 1, n, n)
    r = 8
    while True:
        dt = oracle_rows(n, seed, r, B)
        if dt >= 0.5 * target_s or r >= n:
            r = max(1, min(n, int(r * target_s / max(dt, 1e-4))))
            return r, B
        r = min(n, r * 4)


def oracle_sample(n: int, seed: int, target_s: float):
    """(flop-equivalent per s, rows, seconds, threads) of one bounded oracle sample."""
    import oracle
    r, B = oracle_calibrate(n, seed, target_s)
    dt = oracle_rows(n, seed, r, B)
    return 2.0 * r * n * n / dt, r, dt, oracle.num_threads()


def reference_arm(args, world, rank):
    """The oracle, as it stands, on the host cores: each step is the same bounded
    sample (rows 0..r-1 of the program), r sized so that the whole run takes about
    two minutes whatever --steps/--warmup are."""
    if rank != 0:
        return
    import oracle
    n = args.n
    per_step = max(0.02, min(args.ref_target_s, 120.0 / (args.steps + args.warmup)))
    r, B = oracle_calibrate(n, W.six_loop_seed(n), per_step)
    secs = []
    for i in range(args.warmup + args.steps):
        dt = oracle_rows(n, W.six_loop_seed(n), r, B)
        if i >= args.warmup:
            secs.append(dt)
    ms = statistics.median(secs) * 1e3
    val = 2.0 * r * n * n / (ms / 1e3) / 1e12
    sample = (f"rows 0..{r - 1} of the n={n} six-loop program per step (their init, GEMM rows against the full B, "
              f"scale-add, transpose, row sums, norm) in FP64")
    line = {"impl": "reference", "metric": "gemm_program_tflops", "value": val, "unit": "TFLOP/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded counter hash)",
            "config": {"workload": f"six_loop_n{n}_all_gpu_bf16x6", "n": n, "sample": sample},
            "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def fused_groups(prog, stats):
    """Loops that ran as one pass: a loop that ran on the GPU (placement 1) and the loops
    right after it that ran inside its pass (placement 2).  A fused norm belongs to a GEMM
    chain, which is not a memory-bound pass, and is left out."""
    groups, head = {}, None
    for i, s_ in enumerate(stats):
        if s_["placement"] == 2 and head is not None and prog.loops[i].kind != W.FROBENIUS:
            groups[head].append(i)
        else:
            head = i if s_["placement"] == 1 else None
            if head is not None:
                groups[head] = [i]
    return groups


def group_bytes(prog, idx) -> float:
    """Algorithmic bytes of loops run as one pass: the buffers it reads that it does not
    produce, read once, and the buffers it produces that are OUTPUTs or read after it,
    written once."""
    def nbytes(b):
        B = prog.buffers[b]
        return B.rows * B.cols * (8 if B.dtype == W.F64 else 4)
    produced, reads, writes = set(), set(), []
    for i in idx:
        lp = prog.loops[i]
        for b in ([] if lp.kind == W.INIT else [x for x in lp.ins if x >= 0]):
            if b not in produced:
                reads.add(b)
        for o in (lp.outs if lp.kind == W.INIT else lp.outs[:1]):
            if o >= 0:
                produced.add(o)
                writes.append(o)
    after = {b for lp in prog.loops[max(idx) + 1:] for b in (lp.ins if lp.kind != W.INIT else []) if b >= 0}
    live = {o for o in writes if prog.buffers[o].role == W.OUTPUT or o in after}
    return float(sum(nbytes(b) for b in reads) + sum(nbytes(o) for o in live))


def pass_gbs(prog, stats, loop_ms, steps, hbm):
    """GB/s of every memory-bound pass (a loop, or loops fused into one pass) from the
    per-loop CUDA-event times; a fused pass is keyed by its first loop and its length."""
    out = {}
    for head, idx in fused_groups(prog, stats).items():
        lp = prog.loops[head]
        if lp.kind == W.GEMM or loop_ms[head] <= 0:
            continue
        g = group_bytes(prog, idx) / (loop_ms[head] / steps / 1e3) / 1e9
        key = f"L{head}_{W.KIND_NAMES[lp.kind]}" + (f"+{len(idx) - 1}fused" if len(idx) > 1 else "")
        out[key] = {"gbs": round(g, 1), "hbm_frac": round(g / hbm, 3)}
    return out


# ---- our arm --------------------------------------------------------------------------------------

# flags of the timed runs: outputs stay on the device, and no per-loop timing events (those
# come from a separate, untimed pass)
TIMED = 1 | 4  # RUN_KEEP_DEVICE | RUN_NO_LOOP_TIMES


def our_arm(args, world, rank, local):
    import torch

    import paper_1806_01430_gb300 as gao
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    n, prec = args.n, args.prec
    if args.workload == "twelve_loop":
        prog = W.twelve_loop(args.m, args.k, W.SEED_TWELVE_LOOP + rank, outputs=("C", "r", "f", "q", "s"))
        wname = f"twelve_loop_m{args.m}_k{args.k}_all_gpu_{prec}"
    elif args.workload == "gemm":
        prog = W.gemm_only(n, W.six_loop_seed(n) + rank)
        wname = f"gemm_n{n}_all_gpu_{prec}"
    else:
        prog = W.six_loop(n, W.six_loop_seed(n) + rank, outputs=("C", "r", "f"))
        wname = f"six_loop_n{n}_all_gpu_{prec}"
    flops = prog.gemm_flops()
    # whether the GEMM runs with the chain in its epilogue (BF16 variants of programs that have one)
    chained = bool(args.fuse) and prec in ("bf16", "bf16x3", "bf16x6") and args.workload != "gemm"
    p = gao.prog_from_workload(prog, gemm_prec=PREC[prec], stream=stream, fuse_chains=args.fuse,
                               kchunk=args.kchunk, tile_cfg=args.tile_cfg)
    # the library's GA autotuner picks the GEMM's tile configuration (raster group, K chunk,
    # L2 prefetch) by measured kernel time on this GPU, unless one is given
    tune = None
    if args.autotune and prec != "fp32_simt" and args.kchunk == 0 and args.tile_cfg == 0:
        tune = gao.prog_autotune(p, pop=12, generations=12, seed=3)  # the paper's M = T = 12
    kc, tcfg = (tune["kchunk"], tune["tile_cfg"]) if tune else (args.kchunk, args.tile_cfg)
    mask = (1 << prog.n_loops) - 1
    gemm_loop = 1
    kern_ms, launches = [], 0
    loop_ms = [0.0] * prog.n_loops
    with Clocks(local) as clk:
        time.sleep(0.3)  # let the sampler start
        for _ in range(args.warmup):
            gao.prog_run(p, mask, TIMED)
        torch.cuda.synchronize()
        barrier(world)
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        t0 = clk.mark()
        ev0.record(stream)
        for _ in range(args.steps):
            gao.prog_run(p, mask, TIMED)
        ev1.record(stream)
        torch.cuda.synchronize()
        t1 = clk.mark()
        # per-loop CUDA-event times (kernel roofline, loop shares) from a second pass, so
        # that reading the statistics stays out of the timed region
        stat_steps = max(3, min(args.steps, 300))
        for _ in range(stat_steps):
            gao.prog_run(p, mask, gao.RUN_KEEP_DEVICE)
            st = gao.prog_stats(p)
            kern_ms.append(st[gemm_loop]["kernel_ms"])
            for i, s_ in enumerate(st):
                loop_ms[i] += s_["device_ms"]
        launches = sum(s_["launches"] for s_ in st) * args.steps  # the same kernels every step
        graph_replay = gao.prog_graphs(p)[0] > 0
        time.sleep(0.25)
    barrier(world)
    ms = ev0.elapsed_time(ev1) / args.steps
    ms = allmax(world, ms)
    total_flops = allsum(world, flops)
    value = total_flops / (ms / 1e3) / 1e12
    clocks = clk.summary(t0, t1)
    hbm = peaks().get("hbm_gbs", FALLBACK["hbm_gbs"])
    loop_gbs = pass_gbs(prog, st, loop_ms, stat_steps, hbm)
    loop_ms = {f"L{i}_{W.KIND_NAMES[lp.kind]}": round(v / stat_steps, 4) for i, (lp, v) in enumerate(zip(prog.loops, loop_ms))}

    # accuracy of this run's GEMM against the oracle on sampled entries (no timing)
    err = None
    if rank == 0 and args.check:
        import oracle
        gao.prog_run(p, mask)
        C = gao.prog_output(p, prog.index("C"))
        gm, gk = prog.buffers[prog.index("A")].rows, prog.buffers[prog.index("A")].cols
        gn = prog.buffers[prog.index("B")].cols
        rng = np.random.default_rng(1)
        ii, jj = rng.integers(0, gm, 128), rng.integers(0, gn, 128)
        want = oracle.gemm_init_entries(prog.seed, (0, 1, 2), False, gm, gn, gk, 1.5, 0.5, ii, jj)
        got = C[ii, jj].astype(np.float64)
        err = math.sqrt(float(((got - want) ** 2).mean()) / float((want ** 2).mean()))
    gao.prog_destroy(p)

    # the same program with the chain as separate kernels (GEMM kernel without the fused epilogue)
    unfused = None
    if chained:
        q = gao.prog_from_workload(prog, gemm_prec=PREC[prec], stream=stream, fuse_chains=False, kchunk=kc,
                                   tile_cfg=tcfg)
        for _ in range(3):
            gao.prog_run(q, mask, TIMED)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k = max(3, min(args.steps // 2, 500))
        e0.record(stream)
        for _ in range(k):
            gao.prog_run(q, mask, TIMED)
        e1.record(stream)
        torch.cuda.synchronize()
        ums = e0.elapsed_time(e1) / k
        ks = []
        for _ in range(max(3, min(k, 200))):
            gao.prog_run(q, mask, gao.RUN_KEEP_DEVICE)
            ks.append(gao.prog_stats(q)[gemm_loop]["kernel_ms"])
        bf16 = peaks().get("bf16_tflops_sustained", FALLBACK["bf16_tflops_sustained"])
        gk = flops / (statistics.mean(ks) / 1e3) / 1e12
        unfused = {"value": flops / (ums / 1e3) / 1e12, "unit": "TFLOP/s", "ms_per_step": ums,
                   "gemm_kernel_tflops": gk, "gemm_kernel_frac": gk / (bf16 / PRODUCTS[prec])}
        gao.prog_destroy(q)

    # FP32 SIMT comparison (same program, same n)
    simt = None
    if args.compare_simt and prec != "fp32_simt":
        q = gao.prog_from_workload(prog, gemm_prec=PREC["fp32_simt"], stream=stream)
        for _ in range(2):
            gao.prog_run(q, mask, gao.RUN_KEEP_DEVICE)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k = max(3, min(args.steps // 4, 200))
        ks = []
        e0.record(stream)
        for _ in range(k):
            gao.prog_run(q, mask, gao.RUN_KEEP_DEVICE)
            ks.append(gao.prog_stats(q)[gemm_loop]["kernel_ms"])
        e1.record(stream)
        torch.cuda.synchronize()
        sms = e0.elapsed_time(e1) / k
        simt = {"value": flops / (sms / 1e3) / 1e12, "unit": "TFLOP/s", "ms_per_step": sms,
                "gemm_kernel_tflops": flops / (statistics.mean(ks) / 1e3) / 1e12}
        gao.prog_destroy(q)

    # end to end: inputs from pinned host memory, results read back, every step
    e2e = None
    if args.e2e and args.workload == "six_loop":
        hp = W.host_input_program(n, prog.seed, outputs=("r", "f"))
        q = gao.prog_from_workload(hp, gemm_prec=PREC[prec], stream=stream, fuse_chains=args.fuse, kchunk=kc,
                                   tile_cfg=tcfg)
        import oracle  # input generation only (seeded counter hash); not on the timed path
        for nm, b in (("A", 0), ("B", 1), ("C0", 2)):
            gao.prog_set_input(q, hp.index(nm), oracle.init_matrix(prog.seed, b, n, n).astype(np.float32))
        m5 = (1 << hp.n_loops) - 1
        for _ in range(2):
            gao.prog_run(q, m5, gao.RUN_NO_LOOP_TIMES)
        k = max(3, min(args.steps // 2, 400))
        walls = []
        for _ in range(k):
            walls.append(gao.prog_run(q, m5, gao.RUN_NO_LOOP_TIMES))
        st = gao.prog_stats(q)
        h2d = sum(s["h2d_bytes"] for s in st)
        d2h = sum(s["d2h_bytes"] for s in st)
        ew = statistics.median(walls)
        e2e = {"value": allsum(world, flops) / allmax(world, ew) / 1e12, "unit": "TFLOP/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "ms_per_step": ew * 1e3}
        gao.prog_destroy(q)

    # the all-64-genes search of the n = 4096 FP32 SIMT program (the paper's experiment
    # shape): every gene measured once (CPU loops included), then the paper's GA
    # (M = T = 12, Pc 0.9, Pm 0.05) on the measured table; the paper's metric is the
    # all-CPU time over the best gene's time
    search = None
    if args.search and rank == 0 and args.workload == "six_loop":
        sp = W.six_loop(args.n, W.six_loop_seed(args.n), outputs=("C", "r", "f"))
        q = gao.prog_from_workload(sp, gemm_prec=PREC["fp32_simt"], stream=stream)
        gao.prog_run(q, 0b111111)
        t0 = time.perf_counter()
        fit, secs, hits = gao.ga_evaluate([q], list(range(64)))
        t_search = time.perf_counter() - t0
        ga = gao.ga_run([q], **W.PAPER_GA, seed=11)
        order = np.argsort(secs)
        search = {"workload": f"six_loop_n{args.n}_fp32_simt_all_64_genes", "evals": 64,
                  "wall_s": t_search, "evals_per_s": 64 / t_search,
                  "all_cpu_s": float(secs[0]), "all_gpu_s": float(secs[63]),
                  "best_gene": format(int(order[0]), "06b"), "best_s": float(secs[order[0]]),
                  "speedup_best_vs_all_cpu": float(secs[0] / secs[order[0]]),
                  "top5": [[format(int(m), "06b"), float(secs[m])] for m in order[:5]],
                  "paper_ga": {"best_gene": format(ga.best_mask, "06b"), "best_s": ga.best_s,
                               "found_exhaustive_best": bool(ga.best_mask == int(order[0])),
                               "measured": ga.evaluations, "served": ga.cache_hits,
                               "generation_wall_s": [h["wall_s"] for h in ga.history]}}
        gao.prog_destroy(q)

    # the twelve-loop program's search: the paper's GA (M = T = 12) over the 12-bit gene with
    # transfer-aware times (every host <-> device copy a gene implies is in its time; a gene
    # over 10x the all-GPU time is cut off at that budget), and the FP8 path on the same program
    if args.search and rank == 0 and args.workload == "twelve_loop":
        q = gao.prog_from_workload(prog, gemm_prec=PREC[prec], stream=stream)
        t0 = time.perf_counter()
        ga = gao.ga_run([q], **W.PAPER_GA, seed=11, timeout_s=-1.0)
        t_search = time.perf_counter() - t0
        all_gpu = gao.prog_run(q, (1 << 12) - 1)
        gao.prog_destroy(q)
        search = {"workload": wname.replace("all_gpu_", "") + "_paper_ga", "wall_s": t_search,
                  "measured": ga.evaluations, "served": ga.cache_hits,
                  "best_gene": format(ga.best_mask, "012b"), "best_s": ga.best_s, "all_gpu_s": all_gpu,
                  "history_best_s": [h["best_s"] for h in ga.history],
                  "history_wall_s": [h["wall_s"] for h in ga.history]}
        if prec != "fp8":
            q = gao.prog_from_workload(prog, gemm_prec=PREC["fp8"], stream=stream)
            for _ in range(3):
                gao.prog_run(q, mask, gao.RUN_KEEP_DEVICE)
            ks = []
            for _ in range(20):
                gao.prog_run(q, mask, gao.RUN_KEEP_DEVICE)
                ks.append(gao.prog_stats(q)[gemm_loop]["kernel_ms"])
            gao.prog_run(q, mask)
            C8 = gao.prog_output(q, prog.index("C"))
            gm, gk = prog.buffers[prog.index("A")].rows, prog.buffers[prog.index("A")].cols
            gn = prog.buffers[prog.index("B")].cols
            rng = np.random.default_rng(1)
            ii, jj = rng.integers(0, gm, 128), rng.integers(0, gn, 128)
            import oracle
            want = oracle.gemm_init_entries(prog.seed, (0, 1, 2), False, gm, gn, gk, 1.5, 0.5, ii, jj)
            got = C8[ii, jj].astype(np.float64)
            search["fp8"] = {"gemm_kernel_tflops": flops / (statistics.median(ks) / 1e3) / 1e12,
                             "gemm_rel_err_sampled": math.sqrt(float(((got - want) ** 2).mean()) /
                                                               float((want ** 2).mean()))}
            gao.prog_destroy(q)

    if rank != 0:
        return
    pk = peaks()
    gemm_ms = statistics.mean(kern_ms)
    tc = prec != "fp32_simt"
    if tc:
        bf16 = pk.get("bf16_tflops_sustained", FALLBACK["bf16_tflops_sustained"])
        # peak of the kernel's own arithmetic: FP8 at the nominal 2x of bf16; a split
        # variant spends PRODUCTS bf16 MMAs on every FP32-accurate multiply-add
        peak = bf16 * 2.0 if prec == "fp8" else bf16 / PRODUCTS[prec]
        achieved = flops / (gemm_ms / 1e3) / 1e12
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                # DRAM traffic depends on the tile configuration: only a capture of this one counts
                "traffic": profile_traffic("gemm_tc.cu", f"gemm_tc_{prec}_{wname.split('_all_gpu')[0]}"
                                                         f"{'_fused' if chained else ''}_k{kc}_t{tcfg}.md"),
                "kernel": f"gemm_tc ({prec})" + (" with the fused scale-add / transpose / row-sum / norm epilogue"
                                                  if chained else ""),
                "products": PRODUCTS[prec],
                "hw_tflops": achieved * PRODUCTS[prec], "hw_frac": achieved * PRODUCTS[prec] / bf16,
                "peak_source": f"{pk['source']} bf16 sustained" +
                               (" x2 (fp8 nominal ratio)" if prec == "fp8" else
                                f" / {PRODUCTS[prec]} (bf16 products per FP32-accurate product)"
                                if PRODUCTS[prec] > 1 else "")}
    else:
        mhz = pk.get("sm_max_mhz", 2070.0)
        peak = 152 * 128 * 2 * mhz * 1e6 / 1e12
        achieved = flops / (gemm_ms / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": profile_traffic("gemm_simt.cu", f"gemm_simt_n{n}.md"), "kernel": "gemm_simt",
                "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x max SM clock"}
    cpu = None
    if args.cpu_baseline:
        v, rows, secs, thr = oracle_sample(n, W.six_loop_seed(n), args.ref_target_s)
        cpu = {"value": v / 1e12, "unit": "TFLOP/s", "cores": thr, "kind": "oracle",
               "sample": f"rows 0..{rows - 1} of the n={n} program in FP64 ({secs:.1f} s)"}
    line = {"metric": "gemm_program_tflops", "value": value, "unit": "TFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16x6->f32" if prec == "bf16x6" else prec,
            "data": "synthetic (seeded counter hash, U[-1,1))",
            "config": {"workload": wname, "n": n if args.workload in ("six_loop", "gemm") else None,
                       "gene": format(mask, f"0{prog.n_loops}b"),
                       "gemm": prec, "fused_chain": chained, "graph_replay": graph_replay,
                       "kchunk": kc, "tile_cfg": tcfg,
                       "parallelism": f"replicas{world}" if world > 1 else "single",
                       "l2": "working set larger than the 129 MB L2 (no flush)"},
            "autotune": tune,
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clocks, "gemm_rel_err_sampled": err, "unfused_chain": unfused, "fp32_simt": simt,
            "loop_ms": loop_ms,
            "loop_gbs": loop_gbs, "ga_search": search}
    print(json.dumps(line), flush=True)


def image_arm(args, world, rank, local):
    """Edge-detection image program (the paper's motivating camera workload, Sec. 1):
    nine loops (init, blur, Sobel x/y, squares, magnitude, energy, column maxima) on an
    h x w binary32 image, all on the GPU; metric: image pixels processed per second."""
    import torch

    import paper_1806_01430_gb300 as gao
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    h, w = args.h, args.w
    prog = W.image_program(h, w, W.SEED_IMAGE + rank, outputs=("e", "q"))
    p = gao.prog_from_workload(prog, stream=stream, fuse_chains=args.fuse)
    mask = (1 << prog.n_loops) - 1
    loop_ms = [0.0] * prog.n_loops
    launches = 0
    with Clocks(local) as clk:
        time.sleep(0.3)
        for _ in range(args.warmup):
            gao.prog_run(p, mask, TIMED)
        torch.cuda.synchronize()
        barrier(world)
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        t0 = clk.mark()
        ev0.record(stream)
        for _ in range(args.steps):
            gao.prog_run(p, mask, TIMED)
        ev1.record(stream)
        torch.cuda.synchronize()
        t1 = clk.mark()
        stat_steps = max(3, min(args.steps, 300))  # per-loop event times, outside the timed region
        for _ in range(stat_steps):
            gao.prog_run(p, mask, gao.RUN_KEEP_DEVICE)
            st = gao.prog_stats(p)
            for i, s_ in enumerate(st):
                loop_ms[i] += s_["device_ms"]
        launches = sum(s_["launches"] for s_ in st) * args.steps
        graph_replay = gao.prog_graphs(p)[0] > 0
        time.sleep(0.25)
    barrier(world)
    ms = allmax(world, ev0.elapsed_time(ev1) / args.steps)
    pixels = float(h * w)
    value = allsum(world, pixels) / (ms / 1e3) / 1e9
    clocks = clk.summary(t0, t1)
    hbm = peaks().get("hbm_gbs", FALLBACK["hbm_gbs"])
    per_loop = {f"L{i}_{W.KIND_NAMES[lp.kind]}": round(v / stat_steps, 4)
                for i, (lp, v) in enumerate(zip(prog.loops, loop_ms))}
    loop_gbs = pass_gbs(prog, st, loop_ms, stat_steps, hbm)
    # dominant kernel: the stencil passes (the blur, and Sobel x / Sobel y or, fused, the
    # gradient chain that reads the blurred image once and writes only the magnitude),
    # 8 algorithmic bytes per pixel each
    st_idx = [i for i, lp in enumerate(prog.loops) if lp.kind == W.STENCIL3 and loop_ms[i] > 0]
    st_ms = sum(loop_ms[i] for i in st_idx) / (len(st_idx) * stat_steps)
    achieved = 8.0 * pixels / (st_ms / 1e3) / 1e9
    gao.prog_destroy(p)

    # the same frame with every loop a separate kernel
    unfused = None
    if args.fuse:
        q = gao.prog_from_workload(prog, stream=stream, fuse_chains=False)
        for _ in range(3):
            gao.prog_run(q, mask, TIMED)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k = max(3, min(args.steps // 2, 300))
        e0.record(stream)
        for _ in range(k):
            gao.prog_run(q, mask, TIMED)
        e1.record(stream)
        torch.cuda.synchronize()
        ums = e0.elapsed_time(e1) / k
        unfused = {"value": pixels / (ums / 1e3) / 1e9, "unit": "Gpixel/s", "ms_per_step": ums}
        gao.prog_destroy(q)

    # end to end: the image arrives from pinned host memory every step (a camera
    # frame, INPUT buffer), the energy and column maxima are read back
    e2e = None
    if args.e2e:
        hp = W.image_program(h, w, W.SEED_IMAGE + rank, outputs=("e", "q"), host_image=True)
        q = gao.prog_from_workload(hp, stream=stream, fuse_chains=args.fuse)
        import oracle  # input generation only (seeded counter hash); not on the timed path
        gao.prog_set_input(q, hp.index("X"), oracle.init_matrix(hp.seed, 0, h, w).astype(np.float32))
        m8 = (1 << hp.n_loops) - 1
        for _ in range(2):
            gao.prog_run(q, m8, gao.RUN_NO_LOOP_TIMES)
        k = max(3, min(args.steps // 2, 200))
        walls = [gao.prog_run(q, m8, gao.RUN_NO_LOOP_TIMES) for _ in range(k)]
        st = gao.prog_stats(q)
        ew = statistics.median(walls)
        e2e = {"value": allsum(world, pixels) / allmax(world, ew) / 1e9, "unit": "Gpixel/s",
               "h2d_bytes_per_step": int(sum(s_["h2d_bytes"] for s_ in st)),
               "d2h_bytes_per_step": int(sum(s_["d2h_bytes"] for s_ in st)), "ms_per_step": ew * 1e3}
        gao.prog_destroy(q)

    # the offload search on a 2048 x 2048 frame: all 512 genes measured (CPU loops
    # included), then the paper's GA (M = T = 12, Pc 0.9, Pm 0.05) on the same program
    search = None
    if args.search and rank == 0:
        sh = sw = 2048
        sp = W.image_program(sh, sw, W.SEED_IMAGE, outputs=("e", "q"))
        q = gao.prog_from_workload(sp, stream=stream)
        gao.prog_run(q, (1 << sp.n_loops) - 1)
        t0s = time.perf_counter()
        fit, secs, hits = gao.ga_evaluate([q], list(range(1 << sp.n_loops)))
        t_search = time.perf_counter() - t0s
        ga = gao.ga_run([q], **W.PAPER_GA, seed=11)
        order = np.argsort(secs)
        nb = sp.n_loops
        search = {"workload": f"image_{sh}x{sw}_all_{1 << nb}_genes", "evals": 1 << nb, "wall_s": t_search,
                  "all_cpu_s": float(secs[0]), "all_gpu_s": float(secs[-1]),
                  "best_gene": format(int(order[0]), f"0{nb}b"), "best_s": float(secs[order[0]]),
                  "speedup_best_vs_all_cpu": float(secs[0] / secs[order[0]]),
                  "top5": [[format(int(m), f"0{nb}b"), float(secs[m])] for m in order[:5]],
                  "paper_ga": {"best_gene": format(ga.best_mask, f"0{nb}b"), "best_s": ga.best_s,
                               "rank_in_exhaustive": int(np.where(order == ga.best_mask)[0][0]),
                               "measured": ga.evaluations, "served": ga.cache_hits}}
        gao.prog_destroy(q)

    if rank != 0:
        return
    cpu = None
    if args.cpu_baseline:
        import oracle
        rows = 16
        while True:
            sub = W.image_program(rows, w, W.SEED_IMAGE, outputs=("e", "q"))
            t0c = time.perf_counter()
            oracle.run_program(sub)
            dt = time.perf_counter() - t0c
            if dt >= args.ref_target_s or rows >= h:
                break
            rows = min(h, rows * max(2, int(args.ref_target_s / max(dt, 1e-3) * 0.7)))
        cpu = {"value": rows * w / dt / 1e9, "unit": "Gpixel/s", "cores": oracle.num_threads(), "kind": "oracle",
               "sample": f"a {rows} x {w} image through the nine loops in FP64 ({dt:.1f} s)"}
    line = {"metric": "image_program_gpixels", "value": value, "unit": "Gpixel/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded counter hash, U[-1,1))",
            "config": {"workload": f"image_{h}x{w}_all_gpu", "h": h, "w": w, "graph_replay": graph_replay,
                       "fused_chain": bool(args.fuse),
                       "gene": format(mask, f"0{prog.n_loops}b"),
                       "parallelism": f"replicas{world}" if world > 1 else "single",
                       "l2": "working set larger than the 129 MB L2 (no flush)"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                         "traffic": profile_traffic("kernels_ew.cu", f"stencil3_image_{h}x{w}.md"),
                         "kernel": "stencil3 passes" + (" (blur; fused Sobel x/y, squares, sum)" if args.fuse else "")
                                   + " (8 algorithmic bytes per pixel)",
                         "peak_source": f"{peaks()['source']} hbm_gbs"},
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
            "unfused_chain": unfused, "loop_ms": per_loop, "loop_gbs": loop_gbs, "ga_search": search}
    print(json.dumps(line), flush=True)


def batch_arm(args, world, rank, local):
    """Batched-population workload: a suite of programs of uneven sizes (n log-uniform
    in [128, 2048]), every gene evaluated over the whole suite with one graph launch
    per GPU loop and one grouped tensor-core GEMM launch; the Simple GA runs on top.
    value = GA fitness evaluations per second (individuals scored, measured or served
    from the cache, over the wall time of the GA)."""
    import torch

    import paper_1806_01430_gb300 as gao
    torch.cuda.set_device(local)
    sizes = W.batch_sizes(args.programs)
    progs = [W.six_loop(n, W.SEED_BATCH_BASE + p, outputs=("f",)) for p, n in enumerate(sizes)]
    handles = [gao.prog_from_workload(pr, gemm_prec=PREC[args.prec],
                                      fuse_chains=gao.FUSE_ON if args.fuse else gao.FUSE_OFF,
                                      kchunk=args.kchunk, tile_cfg=args.tile_cfg) for pr in progs]
    b = gao.batch_create(handles)
    # warm-up: the all-GPU gene once (not cached afterwards: fresh batch for the timed GA)
    gao.batch_evaluate(b, [(1 << 6) - 1])
    st_w = gao.batch_stats(b)
    gao.batch_destroy(b)
    b = gao.batch_create(handles)
    # the GA autotuner picks the grouped GEMM's configuration unless one is given
    tune = None
    if args.autotune and args.prec != "fp32_simt" and args.kchunk == 0 and args.tile_cfg == 0:
        tune = gao.batch_autotune(b, pop=12, generations=12, seed=3)
    kc, tcfg = (tune["kchunk"], tune["tile_cfg"]) if tune else (args.kchunk, args.tile_cfg)
    torch.cuda.synchronize()
    barrier(world)
    k_before = gao.batch_stats(b)["kernel_launches"]
    with Clocks(local) as clk:
        time.sleep(0.3)
        t0 = clk.mark()
        res = gao.batch_ga_run(b, pop=args.pop, generations=args.generations, pc=0.9, pm=0.05,
                               seed=7 + rank, timeout_s=-1.0)
        t1 = clk.mark()
        time.sleep(0.25)
    st = gao.batch_stats(b)
    launches = st["kernel_launches"] - k_before  # kernels of the genes the timed GA measured
    wall = allmax(world, t1 - t0)
    evals = allsum(world, args.pop * args.generations)
    gemm_tf = st["gemm_flops"] / (st["gemm_phase_ms"] / 1e3) / 1e12 if st["gemm_phase_ms"] > 0 else None
    if rank == 0:
        pk = peaks()
        peak = pk.get("bf16_tflops_sustained", FALLBACK["bf16_tflops_sustained"])
        roof = None
        if gemm_tf and args.prec != "fp32_simt":
            # the grouped GEMM phase (operand splits included, so a lower bound for the kernel)
            # against the kernel's own arithmetic peak, as in the single-program line
            gpk = peak * 2.0 if args.prec == "fp8" else peak / PRODUCTS[args.prec]
            roof = {"bound": "tensor", "achieved": gemm_tf, "peak": gpk, "unit": "TFLOP/s", "frac": gemm_tf / gpk,
                    "traffic": profile_traffic("gemm_tc.cu", f"gemm_tc_grouped_batch{args.programs}_{args.prec}"
                                                             f"{'_fused' if args.fuse else ''}_k{kc}_t{tcfg}.md"),
                    "kernel": "gemm_tc_grouped_kernel (one launch over all programs' tiles; phase time incl. splits)",
                    "peak_source": f"{pk['source']} bf16 sustained" +
                                   (" x2 (fp8 nominal ratio)" if args.prec == "fp8" else f" / {PRODUCTS[args.prec]}")}
        line = {"metric": "ga_evals_per_s", "value": evals / wall, "unit": "evals/s", "n_gpus": world,
                "steps": args.generations, "warmup": 1, "ms_per_step": wall / args.generations * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.prec,
                "data": "synthetic (seeded counter hash, U[-1,1))",
                "config": {"workload": f"batch_{args.programs}_programs_n128_2048_pop{args.pop}_gen{args.generations}",
                           "programs": args.programs, "sizes_min_max": [min(sizes), max(sizes)], "pop": args.pop,
                           "generations": args.generations, "gemm": args.prec, "fused_chain": bool(args.fuse),
                           "kchunk": kc, "tile_cfg": tcfg},
                "executed_genes": st["executed"], "served_genes": st["served"],
                "executed_program_evals_per_s": st["executed"] * args.programs / max(st["exec_seconds"], 1e-9),
                "best_gene": format(res.best_mask, "06b"), "best_s": res.best_s,
                "grouped_gemm": {"tiles": st["gemm_tiles"], "phase_ms": st["gemm_phase_ms"],
                                 "effective_tflops": gemm_tf,
                                 "hw_frac": (gemm_tf * PRODUCTS[args.prec] / peak) if gemm_tf else None},
                "launches_per_all_gpu_gene": st["launches_per_gene"], "graphs": st["graphs"],
                "fused_gemm_phases": st["fused_phases"], "gpu_launches": launches,
                "autotune": tune, "roofline": roof,
                "all_gpu_gene_warm_s": st_w["exec_seconds"],
                "history": [{"best_s": h["best_s"], "evaluated": h["evaluated"], "hits": h["cache_hits"],
                             "wall_s": h["wall_s"]} for h in res.history],
                "clocks": clk.summary(t0, t1)}
        print(json.dumps(line), flush=True)
    gao.batch_destroy(b)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1500)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--workload", default="six_loop", choices=["six_loop", "gemm", "twelve_loop", "batch", "image"])
    ap.add_argument("--h", type=int, default=8192)
    ap.add_argument("--w", type=int, default=8192)
    ap.add_argument("--programs", type=int, default=64)
    ap.add_argument("--pop", type=int, default=20)
    ap.add_argument("--generations", type=int, default=20)
    ap.add_argument("--no-autotune", dest="autotune", action="store_false")
    ap.add_argument("--kchunk", type=int, default=0, help="fixed GEMM K chunk (with --tile-cfg: skips the autotuner)")
    ap.add_argument("--tile-cfg", type=int, default=0, help="fixed GEMM tile configuration id (skips the autotuner)")
    ap.add_argument("--m", type=int, default=16384)
    ap.add_argument("--k", type=int, default=4096)
    ap.add_argument("--prec", default=None, choices=list(PREC),
                    help="GEMM arithmetic (default: bf16x6 for the six-loop program, bf16x3 for the "
                         "twelve-loop program and the batch, as their configurations state)")
    ap.add_argument("--no-check", dest="check", action="store_false")
    ap.add_argument("--no-e2e", dest="e2e", action="store_false")
    ap.add_argument("--no-simt", dest="compare_simt", action="store_false")
    ap.add_argument("--no-cpu", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-search", dest="search", action="store_false")
    ap.add_argument("--no-fuse", dest="fuse", action="store_false",
                    help="run GEMM, scale-add, transpose and norm as separate kernels (default: the chain "
                         "runs as one GEMM epilogue when all of it is on the GPU)")
    ap.add_argument("--ref-target-s", type=float, default=8.0)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.prec is None:
        args.prec = "bf16x3" if args.workload in ("twelve_loop", "batch") else "bf16x6"
    world, rank, local = dist_init()
    if args.impl == "reference":
        reference_arm(args, world, rank)
    elif args.workload == "batch":
        batch_arm(args, world, rank, local)
    elif args.workload == "image":
        image_arm(args, world, rank, local)
    else:
        our_arm(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
