"""Benchmark of the loop-program hot path on GB300.

Default workload: the precision study's GEMM program at n = 8192 -- INIT of A, B, C0
(counter hash, U[-1,1)) and C = 1.5 A B + 0.5 C0 -- under the all-GPU gene, through the
C ABI (prog_run), with the GEMM as the three-term split-bfloat16 product (BF16X6, the
path that meets 1e-6).  One step = one run of the program.  value = 2 n^3 / step time
(TFLOP/s).  Inputs never leave the device inside the timed region for `value`; `e2e`
repeats the measurement with A, B, C0 copied from the caller's pinned host arrays and C
copied back into one, every step.  The same JSON line carries, at the same n: plain
FP32 SIMT, BF16X3, plain BF16 and FP8 with their TFLOP/s and their errors against the
FP64 oracle on the uniform and the row-scaled input sets; the FP64 residual check of
every entry of C on the GPU; the FP64 oracle timed on the host cores; and, as
sub-results, the batched GA over 64 programs (GA evaluations/s), the twelve-loop
program at m = 16384, k = 4096, and the all-64-genes offload search.

Other workloads: --workload six_loop | twelve_loop | image | batch.

Launch: python bench.py [--gpus N --steps K --warmup W]; for N > 1 under
torch.distributed.run, each rank runs its own replica on its own GPU (replicas
only: the path has no exchange step); value sums the ranks' work over the max
time.  --impl reference times the FP64 CPU oracle on a bounded sample instead.
"""
from __future__ import annotations

import argparse
import ctypes
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
GATE = {"fp32_simt": 1e-6, "bf16x6": 1e-6, "bf16x3": 2e-5, "bf16": 5e-3, "fp8": 6e-2}
FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}
NOMINAL_DENSE_BF16 = 2250.0  # TFLOP/s, GB300 datasheet, dense (no 2:4 sparsity)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        d["source"] = "measured"
        return d
    d = dict(FALLBACK)
    d["source"] = "fallback"
    return d


def tensor_peak(prec: str, pk=None):
    """(peak TFLOP/s of the kernel's own arithmetic, how it was formed, sustained-peak
    equivalent): the measured burst bf16 peak (a kernel timed in a sub-second pass), / the
    products a split variant spends per FP32-accurate multiply-add, x2 for FP8 (nominal
    ratio)."""
    pk = pk or peaks()
    burst = pk.get("bf16_tflops", FALLBACK["bf16_tflops"])
    sus = pk.get("bf16_tflops_sustained", FALLBACK["bf16_tflops_sustained"])
    f = 2.0 if prec == "fp8" else 1.0 / PRODUCTS[prec]
    how = f"{pk['source']} bf16 burst" + (" x2 (fp8 nominal ratio)" if prec == "fp8" else
                                          f" / {PRODUCTS[prec]} (bf16 products per FP32-accurate product)"
                                          if PRODUCTS[prec] > 1 else "")
    return burst * f, how, sus * f


class Clocks:
    """Samples nvidia-smi every 200 ms while running (fallback when NVML is not loadable)."""

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


class NvmlClocks:
    """Reads the SM clock, its maximum and the active clock-event reasons through NVML (the
    driver's libnvidia-ml) every `period` seconds on a thread, so that even a timed region
    of a few tens of milliseconds holds samples.  Reads only: no setting is changed."""

    # public NVML clock-event reason bits
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
               0x80: "hw_power_brake_slowdown"}

    def __init__(self, local: int, period: float = 0.004):
        self.local, self.period = local, period
        self.samples = []  # (time, sm MHz, reasons bitmask)
        self.max_mhz = None
        self.ok = False
        self._stop = threading.Event()
        try:
            self.lib = ctypes.CDLL("libnvidia-ml.so.1")
            if self.lib.nvmlInit_v2() != 0:
                return
            self.h = ctypes.c_void_p()
            found = False
            try:  # the CUDA device's own GPU, whatever CUDA_VISIBLE_DEVICES maps it to
                import torch
                uid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
                found = self.lib.nvmlDeviceGetHandleByUUID(uid.encode(), ctypes.byref(self.h)) == 0
            except Exception:
                found = False
            if not found and self.lib.nvmlDeviceGetHandleByIndex_v2(local, ctypes.byref(self.h)) != 0:
                return
            mx = ctypes.c_uint(0)
            if self.lib.nvmlDeviceGetMaxClockInfo(self.h, 1, ctypes.byref(mx)) == 0:  # NVML_CLOCK_SM
                self.max_mhz = float(mx.value)
            self._reasons = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
            self.ok = True
        except (OSError, AttributeError):
            self.ok = False

    def _sample(self):
        c, r = ctypes.c_uint(0), ctypes.c_ulonglong(0)
        if self.lib.nvmlDeviceGetClockInfo(self.h, 1, ctypes.byref(c)) != 0:
            return
        self._reasons(self.h, ctypes.byref(r))
        self.samples.append((time.time(), float(c.value), int(r.value)))

    def _run(self):
        while not self._stop.is_set():
            self._sample()
            time.sleep(self.period)

    def __enter__(self):
        if self.ok:
            self.t = threading.Thread(target=self._run, daemon=True)
            self.t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        if self.ok:
            self.t.join(timeout=2)

    def mark(self):
        return time.time()

    def summary(self, t0=None, t1=None):
        sm, reasons = [], set()
        for ts, mhz, bits in self.samples:
            if t0 is not None and not (t0 <= ts <= t1):
                continue
            sm.append(mhz)
            for b, nm in self.REASONS.items():
                if bits & b:
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": self.max_mhz,
                "sm_mhz_min": min(sm) if sm else None, "reasons": sorted(reasons), "samples": len(sm),
                "source": "nvml", "period_ms": self.period * 1e3}


def clock_sampler(local: int):
    c = NvmlClocks(local)
    return c if c.ok else Clocks(local)


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


# ---- workload identity (the same config on both arms) -----------------------------------------

def workload_config(args) -> dict:
    """The `config` object of the JSON line: what the workload is, nothing about how it was
    launched, so that the reference arm prints the same one."""
    if args.workload == "gemm":
        return {"workload": f"precision_gemm_program_n{args.n}_{args.prec}", "n": args.n,
                "program": "INIT A, B, C0 (U[-1,1) counter hash); C = 1.5 A B + 0.5 C0",
                "gene": "11", "gemm": args.prec, "seed": W.six_loop_seed(args.n),
                "l2": "working set larger than the 129 MB L2 (no flush)"}
    if args.workload == "twelve_loop":
        return {"workload": f"twelve_loop_m{args.m}_k{args.k}_all_gpu_{args.prec}", "m": args.m, "k": args.k,
                "gene": "1" * 12, "gemm": args.prec, "seed": W.SEED_TWELVE_LOOP,
                "l2": "working set larger than the 129 MB L2 (no flush)"}
    return {"workload": f"six_loop_n{args.n}_all_gpu_{args.prec}", "n": args.n, "gene": "111111",
            "gemm": args.prec, "seed": W.six_loop_seed(args.n),
            "l2": "working set larger than the 129 MB L2 (no flush)"}


# ---- CPU oracle baseline -------------------------------------------------------------------

def oracle_rows(n: int, seed: int, r: int, B, workload: str = "six_loop") -> float:
    """Seconds the FP64 oracle takes for rows [0, r) of the program: INIT of those rows of
    A and C0, their GEMM rows (against the full B, initialised outside) and, for the
    six-loop program, scale-add, transpose, row sums and norm of those rows."""
    import oracle
    t0 = time.perf_counter()
    A = oracle.init_matrix(seed, 0, r, n)
    C0 = oracle.init_matrix(seed, 2, r, n)
    C = oracle.gemm(A, B, C0, 1.5, 0.5)
    if workload != "gemm":
        D = oracle.axpy(C, 2.0, A)
        E = oracle.transpose(D)
        oracle.rowsum(E)
        oracle.frobenius(E)
    return time.perf_counter() - t0


def oracle_calibrate(n: int, seed: int, target_s: float, workload: str = "six_loop"):
    """Rows r whose oracle time is about target_s (at most n); returns (r, B)."""
    import oracle
    B = oracle.init_matrix(seed, 1, n, n)
    r = 8
    while True:
        dt = oracle_rows(n, seed, r, B, workload)
        if dt >= 0.5 * target_s or r >= n:
            r = max(1, min(n, int(r * target_s / max(dt, 1e-4))))
            return r, B
        r = min(n, r * 4)


def oracle_sample(n: int, seed: int, target_s: float, workload: str = "six_loop"):
    """(flop-equivalent per s, rows, seconds, threads) of one bounded oracle sample."""
    import oracle
    r, B = oracle_calibrate(n, seed, target_s, workload)
    dt = oracle_rows(n, seed, r, B, workload)
    return 2.0 * r * n * n / dt, r, dt, oracle.num_threads()


def sample_text(n, r, workload):
    what = "INIT and GEMM rows" if workload == "gemm" else \
        "their init, GEMM rows, scale-add, transpose, row sums, norm"
    return (f"rows 0..{r - 1} of the n={n} {'GEMM' if workload == 'gemm' else 'six-loop'} program per step "
            f"({what}; GEMM rows against the full B) in FP64")


def reference_arm(args, world, rank):
    """The oracle, as it stands, on the host cores: each step is the same bounded
    sample (rows 0..r-1 of the program), r sized so that the whole run takes about
    two minutes whatever --steps/--warmup are."""
    if rank != 0:
        return
    import oracle
    n = args.n
    wl = "gemm" if args.workload == "gemm" else "six_loop"
    per_step = max(0.02, min(args.ref_target_s, 120.0 / (args.steps + args.warmup)))
    r, B = oracle_calibrate(n, W.six_loop_seed(n), per_step, wl)
    secs = []
    for i in range(args.warmup + args.steps):
        dt = oracle_rows(n, W.six_loop_seed(n), r, B, wl)
        if i >= args.warmup:
            secs.append(dt)
    ms = statistics.median(secs) * 1e3
    val = 2.0 * r * n * n / (ms / 1e3) / 1e12
    sample = sample_text(n, r, wl)
    line = {"impl": "reference", "metric": "gemm_program_tflops", "value": val, "unit": "TFLOP/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded counter hash)",
            "config": workload_config(args),
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


def group_bytes(prog, idx, planes=None) -> float:
    """Algorithmic bytes of loops run as one pass: the buffers it reads that it does not
    produce, read once, and the buffers it produces that are OUTPUTs or read after it,
    written once -- as bfloat16 planes (P x 2 bytes per element) for an INIT output the
    library formed straight into a GEMM's operand planes (planes: buffer -> P)."""
    planes = planes or {}

    def nbytes(b):
        B = prog.buffers[b]
        if b in planes:
            return B.rows * B.cols * 2 * planes[b]
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


def planes_of_run(gao, p, prog, prec):
    """Buffers the last run formed only as a GEMM's bfloat16 planes -> planes per element."""
    P = {"bf16": 1, "bf16x3": 2, "bf16x6": 3}.get(prec)
    if P is None:
        return {}
    return {b: P for b in range(len(prog.buffers)) if gao.prog_planes_for(p, b) >= 0}


def pass_gbs(prog, stats, loop_ms, steps, hbm, planes=None):
    """GB/s of every memory-bound pass (a loop, or loops fused into one pass) from the
    per-loop CUDA-event times; a fused pass is keyed by its first loop and its length."""
    out = {}
    for head, idx in fused_groups(prog, stats).items():
        lp = prog.loops[head]
        if lp.kind == W.GEMM or loop_ms[head] <= 0:
            continue
        g = group_bytes(prog, idx, planes) / (loop_ms[head] / steps / 1e3) / 1e9
        key = f"L{head}_{W.KIND_NAMES[lp.kind]}" + (f"+{len(idx) - 1}fused" if len(idx) > 1 else "")
        out[key] = {"gbs": round(g, 1), "hbm_frac": round(g / hbm, 3)}
    return out


# ---- shared measurement pieces -----------------------------------------------------------------

def timed_steps(gao, p, mask, steps, warmup, stream, gemm_loop, world, clk):
    """W untimed runs, then exactly K runs bracketed by a barrier and a synchronize on both
    sides, timed with CUDA events on the program's stream.  Every timed run also records the
    library's per-loop CUDA events on that stream: the GEMM kernel's duration (its roofline)
    and each loop's device time come from the timed runs themselves."""
    import torch
    for _ in range(warmup):
        gao.prog_run(p, mask, gao.RUN_KEEP_DEVICE)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kern, loop_ms, st = [], None, None
    t0 = clk.mark()
    ev0.record(stream)
    for _ in range(steps):
        gao.prog_run(p, mask, gao.RUN_KEEP_DEVICE)
        st = gao.prog_stats(p)  # events of the run just finished (prog_run waited for them)
        kern.append(st[gemm_loop]["kernel_ms"])
        if loop_ms is None:
            loop_ms = [0.0] * len(st)
        for i, s_ in enumerate(st):
            loop_ms[i] += s_["device_ms"]
    ev1.record(stream)
    torch.cuda.synchronize()
    t1 = clk.mark()
    barrier(world)
    ms = ev0.elapsed_time(ev1) / steps
    launches = sum(s_["launches"] for s_ in st) * steps  # the same kernels every step
    return {"ms": ms, "kern_ms": kern, "loop_ms": loop_ms, "stats": st, "launches": launches, "t0": t0, "t1": t1}


def quick_rate(gao, p, mask, k, stream, gemm_loop, flops):
    """(program TFLOP/s, GEMM kernel TFLOP/s, ms per step) over k runs (after 2 warm-ups)."""
    import torch
    for _ in range(2):
        gao.prog_run(p, mask, gao.RUN_KEEP_DEVICE)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ks = []
    e0.record(stream)
    for _ in range(k):
        gao.prog_run(p, mask, gao.RUN_KEEP_DEVICE)
        ks.append(gao.prog_stats(p)[gemm_loop]["kernel_ms"])
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / k
    return flops / (ms / 1e3) / 1e12, flops / (statistics.mean(ks) / 1e3) / 1e12, ms


def sampled_gemm_err(C, seed, rowscale, M, N, K, rng_seed, count=192):
    """Normwise relative error of sampled entries of C = 1.5 A B + 0.5 C0 against the
    oracle's binary64 entries (from the counter hash).  Row-scaled inputs: errors and the
    product term in units of each row's factor 2^e, so that every row counts (a plain
    normwise error over few samples measures only the largest rows)."""
    import oracle
    rng = np.random.default_rng(rng_seed)
    ii, jj = rng.integers(0, M, count), rng.integers(0, N, count)
    want = oracle.gemm_init_entries(seed, (0, 1, 2), rowscale, M, N, K, 1.5, 0.5, ii, jj)
    got = C[ii, jj].astype(np.float64)
    if not rowscale:
        return math.sqrt(float(((got - want) ** 2).mean()) / float((want ** 2).mean()))
    unit = np.array([2.0 ** oracle.row_exponent(seed, int(i)) for i in ii])
    c0 = np.array([oracle.init_value(seed, 2, int(i) * N + int(j)) for i, j in zip(ii, jj)])
    return math.sqrt(float((((got - want) / unit) ** 2).mean()) / float((((want - 0.5 * c0) / unit) ** 2).mean()))


def device_residual(gao, p, loop, n_rows, n_cols, seed):
    """FP64 Freivalds residuals of the program's GEMM on the GPU (random sign vectors)."""
    rng = np.random.default_rng(seed)
    x, y = rng.choice([-1.0, 1.0], n_cols), rng.choice([-1.0, 1.0], n_rows)
    t0 = time.perf_counter()
    r = gao.prog_gemm_residual(p, loop, x, y)
    r["wall_ms"] = (time.perf_counter() - t0) * 1e3
    return {k: (float(v) if isinstance(v, float) else v) for k, v in r.items()}


# ---- the default arm: the n = 8192 GEMM program ---------------------------------------------------

def gemm_arm(args, world, rank, local):
    import torch

    import paper_1806_01430_gb300 as gao
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    n, prec = args.n, args.prec
    seed = W.six_loop_seed(n) + rank
    prog = W.gemm_only(n, seed)
    flops = prog.gemm_flops()
    mask, gemm_loop = 0b11, 1
    tc = prec != "fp32_simt"
    p = gao.prog_from_workload(prog, gemm_prec=PREC[prec], stream=stream, kchunk=args.kchunk, tile_cfg=args.tile_cfg)
    # the library's GA autotuner picks the GEMM's tile configuration (raster group, K chunk,
    # L2 prefetch) by measured kernel time on this GPU, unless one is given
    tune = None
    if args.autotune and tc and args.kchunk == 0 and args.tile_cfg == 0:
        tune = gao.prog_autotune(p, pop=12, generations=12, seed=3)  # the paper's M = T = 12
    kc, tcfg = (tune["kchunk"], tune["tile_cfg"]) if tune else (args.kchunk, args.tile_cfg)
    clk = clock_sampler(local)
    with clk:
        time.sleep(0.05)
        T = timed_steps(gao, p, mask, args.steps, args.warmup, stream, gemm_loop, world, clk)
        time.sleep(0.02)
    ms = allmax(world, T["ms"])
    value = allsum(world, flops) / (ms / 1e3) / 1e12
    clocks = clk.summary(T["t0"], T["t1"])
    graph_replay = gao.prog_graphs(p)[0] > 0
    pk = peaks()
    hbm = pk.get("hbm_gbs", FALLBACK["hbm_gbs"])
    loop_gbs = pass_gbs(prog, T["stats"], T["loop_ms"], args.steps, hbm, planes_of_run(gao, p, prog, prec))
    loop_ms = {f"L{i}_{W.KIND_NAMES[lp.kind]}": round(v / args.steps, 4)
               for i, (lp, v) in enumerate(zip(prog.loops, T["loop_ms"]))}

    variants, residual, err, err_rows = {}, None, None, None
    if rank == 0 and args.check:
        gao.prog_run(p, mask)  # C to the host
        err = sampled_gemm_err(gao.prog_output(p, prog.index("C")), seed, False, n, n, n, 1)
        residual = device_residual(gao, p, gemm_loop, n, n, 8192)
    gao.prog_destroy(p)

    def rows_err(v):
        """The row-scaled input set (rows of A times 2^e, e in [-10, 10])."""
        rs = W.gemm_only(n, W.SEED_N8192_ROWS, rowscale_a=True)
        q = gao.prog_from_workload(rs, gemm_prec=PREC[v], stream=stream)
        gao.prog_run(q, mask)
        e = sampled_gemm_err(gao.prog_output(q, rs.index("C")), rs.seed, True, n, n, n, 2)
        res = device_residual(gao, q, gemm_loop, n, n, 8193)
        gao.prog_destroy(q)
        return e, res

    if rank == 0 and args.check:
        err_rows, res_rows = rows_err(prec)
    if rank == 0 and args.compare:
        # every other GEMM arithmetic on the same program, same n (the precision study)
        for v in ("fp32_simt", "bf16x3", "bf16", "fp8"):
            if v == prec:
                continue
            q = gao.prog_from_workload(prog, gemm_prec=PREC[v], stream=stream)
            k = max(3, min(args.steps, 20))
            prog_tf, kern_tf, vms = quick_rate(gao, q, mask, k, stream, gemm_loop, flops)
            gao.prog_run(q, mask)
            e = sampled_gemm_err(gao.prog_output(q, prog.index("C")), seed, False, n, n, n, 1)
            res = device_residual(gao, q, gemm_loop, n, n, 8192)
            gao.prog_destroy(q)
            e_rows, _ = rows_err(v)
            d = {"program_tflops": prog_tf, "gemm_kernel_tflops": kern_tf, "ms_per_step": vms,
                 "rel_err_sampled": e, "rel_err_sampled_row_scaled": e_rows, "gate": GATE[v],
                 "freivalds_residual": max(res["right"], res["left"])}
            if v != "fp32_simt":
                peak, _, _ = tensor_peak(v, pk)
                d["gemm_kernel_frac_of_peak"] = kern_tf / peak
            else:
                d["gemm_kernel_frac_of_ffma_peak"] = kern_tf / (152 * 128 * 2 * pk.get("sm_max_mhz", 2070.0) / 1e6)
            variants[v] = d

    # end to end through the public API: the caller's pinned host arrays bound to the
    # program's buffers; every step copies A, B, C0 to the device and C back
    e2e = None
    if args.e2e:
        e2e = gemm_e2e(gao, torch, n, seed, prec, kc, tcfg, stream, args.steps, world, flops)

    if rank != 0:
        return
    gemm_ms = statistics.mean(T["kern_ms"])
    achieved = flops / (gemm_ms / 1e3) / 1e12
    if tc:
        peak, how, sus = tensor_peak(prec, pk)
        bf16 = pk.get("bf16_tflops", FALLBACK["bf16_tflops"])
        # DRAM bytes per launch from the ncu summary of this configuration, else of the
        # library's default configuration of the same kernel (named, since the raster group
        # and prefetch change the traffic)
        traffic_src = f"gemm_tc_{prec}_gemm_n{n}_k{kc}_t{tcfg}.md"
        traffic = profile_traffic("gemm_tc.cu", traffic_src)
        if traffic is None:
            for alt in (f"gemm_tc_{prec}_gemm_n{n}_k256_t0.md", f"gemm_tc_{prec}_gemm_n{n}.md"):
                traffic = profile_traffic("gemm_tc.cu", alt)
                if traffic is not None:
                    traffic_src = alt
                    break
        if traffic is None:
            traffic_src = None
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic, "traffic_profile": traffic_src,
                "kernel": f"gemm_tc ({prec})", "products": PRODUCTS[prec],
                "hw_tflops": achieved * PRODUCTS[prec], "hw_frac": achieved * PRODUCTS[prec] / bf16,
                "frac_of_sustained": achieved / sus, "peak_source": how,
                # the datasheet's dense bf16 figure (2.25 PFLOP/s), for comparison with the measured peaks
                "frac_of_nominal_dense": achieved * PRODUCTS[prec] / (NOMINAL_DENSE_BF16 * (2.0 if prec == "fp8" else 1.0)),
                "kernel_ms": gemm_ms, "kernel_ms_source": "library CUDA events around the kernel, every timed step"}
    else:
        mhz = pk.get("sm_max_mhz", 2070.0)
        peak = 152 * 128 * 2 * mhz * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": profile_traffic("gemm_simt.cu", f"gemm_simt_n{n}.md"), "kernel": "gemm_simt",
                "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x max SM clock"}
    cpu = None
    if args.cpu_baseline:
        v, rows, secs, thr = oracle_sample(n, W.six_loop_seed(n), args.ref_target_s, "gemm")
        cpu = {"value": v / 1e12, "unit": "TFLOP/s", "cores": thr, "kind": "oracle",
               "sample": sample_text(n, rows, "gemm") + f" ({secs:.1f} s)"}
    simt = variants.get("fp32_simt")
    extra = sub_results(args, gao, torch, stream) if args.sub else None
    line = {"metric": "gemm_program_tflops", "value": value, "unit": "TFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16x6->f32" if prec == "bf16x6" else prec,
            "data": "synthetic (seeded counter hash, U[-1,1); row-scaled set for the error study)",
            "config": workload_config(args),
            "launch_config": {"kchunk": kc, "tile_cfg": tcfg, "graph_replay": graph_replay,
                              "parallelism": f"replicas{world}" if world > 1 else "single"},
            "autotune": tune, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": T["launches"],
            "clocks": clocks,
            "accuracy": {"rel_err_sampled": err, "rel_err_sampled_row_scaled": err_rows, "gate": GATE[prec],
                         "freivalds_residual_fp64_gpu": residual,
                         "freivalds_residual_row_scaled": (res_rows if args.check else None)},
            "vs_fp32_simt": ({"fp32_simt_program_tflops": simt["program_tflops"],
                              "speedup_program": value / simt["program_tflops"],
                              "fp32_simt_rel_err_sampled": simt["rel_err_sampled"]} if simt else None),
            "variants": variants, "loop_ms": loop_ms, "loop_gbs": loop_gbs, "sub_results": extra}
    print(json.dumps(line), flush=True)


def gemm_e2e(gao, torch, n, seed, prec, kc, tcfg, stream, steps, world, flops):
    """The GEMM program fed from the caller's memory: A, B, C0 formed once by the library's
    own INIT and read back into pinned torch CPU tensors, which are bound (prog_bind_host)
    as the INPUT buffers of a GEMM-only program, and C bound as its OUTPUT.  Each timed step
    is one prog_run: the three operands cross the link (A in row blocks overlapped with the
    GEMM), the GEMM runs, C comes back into the caller's array."""
    host = init_inputs(gao, torch, seed, [("A", n, n), ("B", n, n), ("C0", n, n)], stream)
    host["C"] = torch.empty((n, n), dtype=torch.float32, pin_memory=True)
    hp = W.host_input_gemm(n)
    q = gao.prog_from_workload(hp, gemm_prec=PREC[prec], stream=stream, kchunk=kc, tile_cfg=tcfg)
    for nm in ("A", "B", "C0", "C"):
        gao.prog_bind_host(q, hp.index(nm), host[nm])
    for _ in range(2):
        gao.prog_run(q, 1, gao.RUN_NO_LOOP_TIMES)
    k = max(3, min(steps, 20))
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(k):
        gao.prog_run(q, 1, gao.RUN_NO_LOOP_TIMES)
    wall = (time.perf_counter() - t0) / k
    st = gao.prog_stats(q)
    gao.prog_destroy(q)
    wall = allmax(world, wall)
    return {"value": allsum(world, flops) / wall / 1e12, "unit": "TFLOP/s",
            "h2d_bytes_per_step": int(sum(s_["h2d_bytes"] for s_ in st)),
            "d2h_bytes_per_step": int(sum(s_["d2h_bytes"] for s_ in st)), "ms_per_step": wall * 1e3,
            "steps": k, "api": "prog_bind_host (caller's pinned arrays) + prog_run, host wall clock",
            "inputs": "formed by the library's INIT loop, read back once"}


def init_inputs(gao, torch, seed, shapes, stream):
    """Host inputs formed by the library's own INIT loop (buffer ids 0, 1, ... in order, the
    hash streams of the programs' INIT loops) and read back into pinned torch CPU tensors."""
    bufs = [W.Buffer(nm, r, c, W.F32, W.OUTPUT) for nm, r, c in shapes]
    gen = W.Program("inputs", bufs, [W.Loop(W.INIT, [], list(range(len(bufs))))], seed)
    g = gao.prog_from_workload(gen, stream=stream)
    gao.prog_run(g, 1)
    host = {}
    for i, (nm, r, c) in enumerate(shapes):
        host[nm] = torch.empty((r, c), dtype=torch.float32, pin_memory=True)
        host[nm].numpy()[:] = gao.prog_output(g, i)
    gao.prog_destroy(g)
    return host


# ---- sub-results: the other configurations, in the default line -------------------------------

def sub_results(args, gao, torch, stream):
    out = {}
    t = time.perf_counter()
    try:
        out["batch_ga"] = batch_result(args, gao, torch)
    except Exception as e:  # reported, not hidden
        out["batch_ga"] = {"error": str(e)}
    try:
        out["twelve_loop"] = twelve_result(args, gao, torch, stream)
    except Exception as e:
        out["twelve_loop"] = {"error": str(e)}
    try:
        out["six_loop_fused"] = six_fused_result(args, gao, torch, stream)
    except Exception as e:
        out["six_loop_fused"] = {"error": str(e)}
    if args.search:
        try:
            out["six_loop_search"] = search_result(args, gao, stream, 4096)
        except Exception as e:
            out["six_loop_search"] = {"error": str(e)}
    out["wall_s"] = time.perf_counter() - t
    return out


def search_result(args, gao, stream, n):
    """The all-64-genes search of the n = 4096 FP32 SIMT six-loop program (the paper's
    experiment shape): every gene measured once (CPU loops included), then the paper's GA
    (M = T = 12, Pc 0.9, Pm 0.05) on the same program; the paper's metric is the all-CPU
    time over the best gene's time."""
    sp = W.six_loop(n, W.six_loop_seed(n), outputs=("C", "r", "f"))
    q = gao.prog_from_workload(sp, gemm_prec=PREC["fp32_simt"], stream=stream)
    gao.prog_run(q, 0b111111)
    t0 = time.perf_counter()
    fit, secs, hits = gao.ga_evaluate([q], list(range(64)))
    t_search = time.perf_counter() - t0
    ga = gao.ga_run([q], **W.PAPER_GA, seed=11)
    order = np.argsort(secs)
    gao.prog_destroy(q)
    return {"workload": f"six_loop_n{n}_fp32_simt_all_64_genes", "evals": 64, "wall_s": t_search,
            "evals_per_s": 64 / t_search, "all_cpu_s": float(secs[0]), "all_gpu_s": float(secs[63]),
            "best_gene": format(int(order[0]), "06b"), "best_s": float(secs[order[0]]),
            "speedup_best_vs_all_cpu": float(secs[0] / secs[order[0]]),
            "top5": [[format(int(m), "06b"), float(secs[m])] for m in order[:5]],
            "paper_ga": {"best_gene": format(ga.best_mask, "06b"), "best_s": ga.best_s,
                         "found_exhaustive_best": bool(ga.best_mask == int(order[0])),
                         "measured": ga.evaluations, "served": ga.cache_hits}}


def batch_result(args, gao, torch, programs=64, pop=20, generations=20, prec="bf16x3", replicas=None):
    """The batched-population configuration: 64 six-loop programs (n log-uniform in [128,
    2048]), the GA (20 individuals x 20 generations) scoring genes over the whole suite; each
    generation's new genes are measured together on copies of the suite (replicas = the
    population), their GEMMs in one grouped persistent launch; GA evaluations per second over
    the GA's wall time."""
    replicas = pop if replicas is None else replicas
    sizes = W.batch_sizes(programs)
    progs = [W.six_loop(n, W.SEED_BATCH_BASE + p, outputs=("f",)) for p, n in enumerate(sizes)]
    handles = [gao.prog_from_workload(pr, gemm_prec=PREC[prec], fuse_chains=gao.FUSE_ON) for pr in progs]
    b = gao.batch_create(handles)
    tune = gao.batch_autotune(b, pop=12, generations=12, seed=3)
    t0 = time.perf_counter()
    gao.batch_set_replicas(b, replicas)
    t_rep = time.perf_counter() - t0
    gao.batch_evaluate(b, [(1 << 6) - 1])  # warm
    gao.batch_set_replicas(b, replicas)     # clears the cache: the GA starts from nothing measured
    st0 = gao.batch_stats(b)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = gao.batch_ga_run(b, pop=pop, generations=generations, pc=0.9, pm=0.05, seed=7, timeout_s=-1.0)
    wall = time.perf_counter() - t0
    st = gao.batch_stats(b)
    # the grouped launch over the whole generation: every gene of a group that offloads the GEMM
    gl, gg = st["grouped_launches"] - st0["grouped_launches"], st["grouped_genes"] - st0["grouped_genes"]
    # one full-suite grouped launch timed alone (the all-GPU gene, cache cleared)
    gao.batch_set_replicas(b, 1)
    gao.batch_evaluate(b, [(1 << 6) - 1])
    one = gao.batch_stats(b)
    gao.batch_destroy(b)
    gemm_tf = one["gemm_flops"] / (one["gemm_phase_ms"] / 1e3) / 1e12 if one["gemm_phase_ms"] > 0 else None
    peak, how, _ = tensor_peak(prec)
    return {"metric": "ga_evals_per_s", "value": pop * generations / wall, "unit": "evals/s",
            "workload": f"batch_{programs}_programs_n128_2048_pop{pop}_gen{generations}_{prec}",
            "sizes_min_max": [min(sizes), max(sizes)], "ga_wall_s": wall, "replicas": replicas,
            "replica_setup_s": t_rep,
            "executed_genes": st["executed"] - st0["executed"], "served_genes": st["served"] - st0["served"],
            "grouped_launches": gl, "genes_in_grouped_launches": gg,
            "best_gene": format(res.best_mask, "06b"), "best_s": res.best_s,
            "grouped_gemm_one_suite": {"tiles": one["gemm_tiles"], "launch_ms": one["gemm_phase_ms"],
                                       "effective_tflops": gemm_tf,
                                       "frac_of_peak": gemm_tf / peak if gemm_tf else None, "peak_source": how},
            "autotune": tune}


def twelve_result(args, gao, torch, stream, m=16384, k=4096, prec="bf16x3"):
    """The large rectangular configuration: the twelve-loop program (GEMM M = N = 16384,
    K = 4096, BF16X3, the chain in the GEMM epilogue) under the all-GPU gene, and its GEMM
    on the FP8 path; the memory-bound loops' GB/s."""
    prog = W.twelve_loop(m, k, W.SEED_TWELVE_LOOP, outputs=("C", "r", "f", "q", "s"))
    flops = prog.gemm_flops()
    mask = (1 << 12) - 1
    p = gao.prog_from_workload(prog, gemm_prec=PREC[prec], stream=stream, fuse_chains=True)
    clk = Clocks(0)  # not sampled: the main line carries the clock record
    steps = 10
    T = timed_steps(gao, p, mask, steps, 3, stream, 1, 1, clk)
    hbm = peaks().get("hbm_gbs", FALLBACK["hbm_gbs"])
    gbs = pass_gbs(prog, T["stats"], T["loop_ms"], steps, hbm, planes_of_run(gao, p, prog, prec))
    gao.prog_run(p, mask)
    err = sampled_gemm_err(gao.prog_output(p, prog.index("C")), prog.seed, False, m, m, k, 1)
    gao.prog_destroy(p)
    peak, how, _ = tensor_peak(prec)
    kern = flops / (statistics.mean(T["kern_ms"]) / 1e3) / 1e12
    q = gao.prog_from_workload(prog, gemm_prec=PREC["fp8"], stream=stream)
    _, kern8, _ = quick_rate(gao, q, mask, 5, stream, 1, flops)
    gao.prog_run(q, mask)
    err8 = sampled_gemm_err(gao.prog_output(q, prog.index("C")), prog.seed, False, m, m, k, 1)
    gao.prog_destroy(q)
    peak8, how8, _ = tensor_peak("fp8")
    return {"workload": f"twelve_loop_m{m}_k{k}_all_gpu_{prec}_fused", "program_tflops": flops / (T["ms"] / 1e3) / 1e12,
            "ms_per_step": T["ms"], "gemm_kernel_tflops": kern, "gemm_kernel_frac_of_peak": kern / peak,
            "peak_source": how, "rel_err_sampled": err, "loop_gbs": gbs,
            "fp8": {"gemm_kernel_tflops": kern8, "frac_of_peak": kern8 / peak8, "peak_source": how8,
                    "rel_err_sampled": err8}}


def six_fused_result(args, gao, torch, stream, n=4096, prec="bf16x6"):
    """The six-loop program at n = 4096 under the all-GPU gene with its chain (scale-add,
    transpose, row sums, Frobenius norm) in the BF16x6 GEMM's epilogue, library default
    tile configuration: program and GEMM-kernel TFLOP/s, the kernel's fraction of the
    burst peak / 6, and the sampled error of C."""
    prog = W.six_loop(n, W.six_loop_seed(n), outputs=("C", "D", "E", "r", "f"))
    flops = prog.gemm_flops()
    mask = (1 << prog.n_loops) - 1
    p = gao.prog_from_workload(prog, gemm_prec=PREC[prec], stream=stream, fuse_chains=True)
    steps = 20
    T = timed_steps(gao, p, mask, steps, 3, stream, 1, 1, Clocks(0))
    gao.prog_run(p, mask)
    err = sampled_gemm_err(gao.prog_output(p, prog.index("C")), prog.seed, False, n, n, n, 1)
    gao.prog_destroy(p)
    peak, how, _ = tensor_peak(prec)
    kern = flops / (statistics.mean(T["kern_ms"]) / 1e3) / 1e12
    return {"workload": f"six_loop_n{n}_all_gpu_{prec}_fused", "program_tflops": flops / (T["ms"] / 1e3) / 1e12,
            "ms_per_step": T["ms"], "gemm_kernel_tflops": kern, "gemm_kernel_frac_of_peak": kern / peak,
            "peak_source": how, "rel_err_sampled": err}


# ---- six-loop and twelve-loop lines ------------------------------------------------------------------

def our_arm(args, world, rank, local):
    import torch

    import paper_1806_01430_gb300 as gao
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    n, prec = args.n, args.prec
    if args.workload == "twelve_loop":
        prog = W.twelve_loop(args.m, args.k, W.SEED_TWELVE_LOOP + rank, outputs=("C", "r", "f", "q", "s"))
        wname = f"twelve_loop_m{args.m}_k{args.k}"
    else:
        prog = W.six_loop(n, W.six_loop_seed(n) + rank, outputs=("C", "r", "f"))
        wname = f"six_loop_n{n}"
    flops = prog.gemm_flops()
    # whether the GEMM runs with the chain in its epilogue (BF16 variants of programs that have one)
    chained = bool(args.fuse) and prec in ("bf16", "bf16x3", "bf16x6")
    p = gao.prog_from_workload(prog, gemm_prec=PREC[prec], stream=stream, fuse_chains=args.fuse,
                               kchunk=args.kchunk, tile_cfg=args.tile_cfg)
    tune = None
    if args.autotune and prec != "fp32_simt" and args.kchunk == 0 and args.tile_cfg == 0:
        tune = gao.prog_autotune(p, pop=12, generations=12, seed=3)  # the paper's M = T = 12
    kc, tcfg = (tune["kchunk"], tune["tile_cfg"]) if tune else (args.kchunk, args.tile_cfg)
    mask = (1 << prog.n_loops) - 1
    gemm_loop = 1
    clk = clock_sampler(local)
    with clk:
        time.sleep(0.05)
        T = timed_steps(gao, p, mask, args.steps, args.warmup, stream, gemm_loop, world, clk)
        time.sleep(0.02)
    ms = allmax(world, T["ms"])
    value = allsum(world, flops) / (ms / 1e3) / 1e12
    clocks = clk.summary(T["t0"], T["t1"])
    graph_replay = gao.prog_graphs(p)[0] > 0
    pk = peaks()
    hbm = pk.get("hbm_gbs", FALLBACK["hbm_gbs"])
    loop_gbs = pass_gbs(prog, T["stats"], T["loop_ms"], args.steps, hbm, planes_of_run(gao, p, prog, prec))
    loop_ms = {f"L{i}_{W.KIND_NAMES[lp.kind]}": round(v / args.steps, 4)
               for i, (lp, v) in enumerate(zip(prog.loops, T["loop_ms"]))}
    err = None
    if rank == 0 and args.check:
        gao.prog_run(p, mask)
        gm, gk = prog.buffers[prog.index("A")].rows, prog.buffers[prog.index("A")].cols
        gn = prog.buffers[prog.index("B")].cols
        err = sampled_gemm_err(gao.prog_output(p, prog.index("C")), prog.seed, False, gm, gn, gk, 1, 128)
    gao.prog_destroy(p)

    unfused = None
    if chained:
        q = gao.prog_from_workload(prog, gemm_prec=PREC[prec], stream=stream, fuse_chains=False, kchunk=kc,
                                   tile_cfg=tcfg)
        ptf, ktf, ums = quick_rate(gao, q, mask, max(3, min(args.steps, 50)), stream, gemm_loop, flops)
        peak, _, _ = tensor_peak(prec, pk)
        unfused = {"value": ptf, "unit": "TFLOP/s", "ms_per_step": ums, "gemm_kernel_tflops": ktf,
                   "gemm_kernel_frac": ktf / peak}
        gao.prog_destroy(q)

    e2e = None
    if args.e2e and args.workload == "six_loop":
        hp = W.host_input_program(n, prog.seed, outputs=("r", "f"))
        host = init_inputs(gao, torch, prog.seed, [("A", n, n), ("B", n, n), ("C0", n, n)], stream)
        q = gao.prog_from_workload(hp, gemm_prec=PREC[prec], stream=stream, fuse_chains=args.fuse, kchunk=kc,
                                   tile_cfg=tcfg)
        for nm in ("A", "B", "C0"):
            gao.prog_bind_host(q, hp.index(nm), host[nm])
        m5 = (1 << hp.n_loops) - 1
        for _ in range(2):
            gao.prog_run(q, m5, gao.RUN_NO_LOOP_TIMES)
        k = max(3, min(args.steps, 50))
        t0 = time.perf_counter()
        for _ in range(k):
            gao.prog_run(q, m5, gao.RUN_NO_LOOP_TIMES)
        ew = (time.perf_counter() - t0) / k
        st = gao.prog_stats(q)
        e2e = {"value": allsum(world, flops) / allmax(world, ew) / 1e12, "unit": "TFLOP/s",
               "h2d_bytes_per_step": int(sum(s["h2d_bytes"] for s in st)),
               "d2h_bytes_per_step": int(sum(s["d2h_bytes"] for s in st)), "ms_per_step": ew * 1e3,
               "api": "prog_bind_host (caller's pinned arrays) + prog_run, host wall clock"}
        gao.prog_destroy(q)

    search = None
    if args.search and rank == 0 and args.workload == "six_loop":
        search = search_result(args, gao, stream, args.n)
    if args.search and rank == 0 and args.workload == "twelve_loop":
        q = gao.prog_from_workload(prog, gemm_prec=PREC[prec], stream=stream)
        t0 = time.perf_counter()
        ga = gao.ga_run([q], **W.PAPER_GA, seed=11, timeout_s=-1.0)
        t_search = time.perf_counter() - t0
        all_gpu = gao.prog_run(q, (1 << 12) - 1)
        gao.prog_destroy(q)
        search = {"workload": wname + f"_{prec}_paper_ga", "wall_s": t_search,
                  "measured": ga.evaluations, "served": ga.cache_hits,
                  "best_gene": format(ga.best_mask, "012b"), "best_s": ga.best_s, "all_gpu_s": all_gpu,
                  "history_best_s": [h["best_s"] for h in ga.history],
                  "history_wall_s": [h["wall_s"] for h in ga.history]}

    if rank != 0:
        return
    gemm_ms = statistics.mean(T["kern_ms"])
    achieved = flops / (gemm_ms / 1e3) / 1e12
    if prec != "fp32_simt":
        peak, how, sus = tensor_peak(prec, pk)
        bf16 = pk.get("bf16_tflops", FALLBACK["bf16_tflops"])
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": profile_traffic("gemm_tc.cu", f"gemm_tc_{prec}_{wname}"
                                                         f"{'_fused' if chained else ''}_k{kc}_t{tcfg}.md"),
                "kernel": f"gemm_tc ({prec})" + (" with the fused scale-add / transpose / row-sum / norm epilogue"
                                                  if chained else ""),
                "products": PRODUCTS[prec], "hw_tflops": achieved * PRODUCTS[prec],
                "hw_frac": achieved * PRODUCTS[prec] / bf16, "frac_of_sustained": achieved / sus,
                "peak_source": how}
    else:
        mhz = pk.get("sm_max_mhz", 2070.0)
        peak = 152 * 128 * 2 * mhz * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": profile_traffic("gemm_simt.cu", f"gemm_simt_n{n}.md"), "kernel": "gemm_simt",
                "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x max SM clock"}
    cpu = None
    if args.cpu_baseline and args.workload == "six_loop":
        v, rows, secs, thr = oracle_sample(n, W.six_loop_seed(n), args.ref_target_s)
        cpu = {"value": v / 1e12, "unit": "TFLOP/s", "cores": thr, "kind": "oracle",
               "sample": sample_text(n, rows, "six_loop") + f" ({secs:.1f} s)"}
    line = {"metric": "gemm_program_tflops", "value": value, "unit": "TFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16x6->f32" if prec == "bf16x6" else prec,
            "data": "synthetic (seeded counter hash, U[-1,1))", "config": workload_config(args),
            "launch_config": {"fused_chain": chained, "graph_replay": graph_replay, "kchunk": kc, "tile_cfg": tcfg,
                              "parallelism": f"replicas{world}" if world > 1 else "single"},
            "autotune": tune, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": T["launches"],
            "clocks": clocks, "gemm_rel_err_sampled": err, "unfused_chain": unfused,
            "loop_ms": loop_ms, "loop_gbs": loop_gbs, "ga_search": search}
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
    clk = clock_sampler(local)
    with clk:
        time.sleep(0.05)
        T = timed_steps(gao, p, mask, args.steps, args.warmup, stream, 1, world, clk)
        time.sleep(0.02)
    st, loop_ms = T["stats"], T["loop_ms"]
    graph_replay = gao.prog_graphs(p)[0] > 0
    ms = allmax(world, T["ms"])
    pixels = float(h * w)
    value = allsum(world, pixels) / (ms / 1e3) / 1e9
    clocks = clk.summary(T["t0"], T["t1"])
    hbm = peaks().get("hbm_gbs", FALLBACK["hbm_gbs"])
    per_loop = {f"L{i}_{W.KIND_NAMES[lp.kind]}": round(v / args.steps, 4)
                for i, (lp, v) in enumerate(zip(prog.loops, loop_ms))}
    loop_gbs = pass_gbs(prog, st, loop_ms, args.steps, hbm)
    # dominant kernels: the stencil passes -- the blur, Sobel x and Sobel y, or, fused, one
    # pass that reads the raw frame once and forms the blur, both gradients, the squares, the
    # magnitude and its sum and column maxima (writing none of the intermediates) -- with each
    # pass's algorithmic bytes (the same accounting as loop_gbs)
    groups = fused_groups(prog, st)
    st_idx = [i for i in groups if prog.loops[i].kind == W.STENCIL3 and loop_ms[i] > 0]
    st_bytes = sum(group_bytes(prog, groups[i]) for i in st_idx)
    st_ms = sum(loop_ms[i] for i in st_idx) / args.steps
    achieved = st_bytes / (st_ms / 1e3) / 1e9
    st_bpp = st_bytes / pixels
    # the same passes against the FP32 lanes: one operation per nonzero stencil weight
    # (a multiply-add), square, magnitude multiply-add and sum addition per pixel
    nonzero = {W.BLUR: 9, W.LAPLACIAN: 5, W.SOBEL_X: 6, W.SOBEL_Y: 6}
    kind_ops = {W.SQUARE: 1, W.AXPY: 1, W.SUM: 1}
    ops_px = sum(nonzero[prog.loops[j].flags] if prog.loops[j].kind == W.STENCIL3 else kind_ops.get(prog.loops[j].kind, 0)
                 for i in st_idx for j in groups[i])
    fp32_peak = 152 * 128 * 2.07e9 / 1e12  # lane operations per second: SMs x FP32 lanes x maximum SM clock
    alu_achieved = ops_px * pixels / (st_ms / 1e3) / 1e12
    gao.prog_destroy(p)

    unfused = None
    if args.fuse:
        q = gao.prog_from_workload(prog, stream=stream, fuse_chains=False)
        for _ in range(3):
            gao.prog_run(q, mask, gao.RUN_KEEP_DEVICE)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k = max(3, min(args.steps, 100))
        e0.record(stream)
        for _ in range(k):
            gao.prog_run(q, mask, gao.RUN_KEEP_DEVICE | gao.RUN_NO_LOOP_TIMES)
        e1.record(stream)
        torch.cuda.synchronize()
        ums = e0.elapsed_time(e1) / k
        unfused = {"value": pixels / (ums / 1e3) / 1e9, "unit": "Gpixel/s", "ms_per_step": ums}
        gao.prog_destroy(q)

    # end to end: the frame arrives from the caller's pinned host array every step (a camera
    # frame bound as the INPUT buffer), the energy and column maxima are read back
    e2e = None
    if args.e2e:
        hp = W.image_program(h, w, W.SEED_IMAGE + rank, outputs=("e", "q"), host_image=True)
        frame = init_inputs(gao, torch, W.SEED_IMAGE + rank, [("X", h, w)], stream)["X"]
        q = gao.prog_from_workload(hp, stream=stream, fuse_chains=args.fuse)
        gao.prog_bind_host(q, hp.index("X"), frame)
        m8 = (1 << hp.n_loops) - 1
        for _ in range(2):
            gao.prog_run(q, m8, gao.RUN_NO_LOOP_TIMES)
        k = max(3, min(args.steps, 100))
        t0 = time.perf_counter()
        for _ in range(k):
            gao.prog_run(q, m8, gao.RUN_NO_LOOP_TIMES)
        ew = (time.perf_counter() - t0) / k
        st2 = gao.prog_stats(q)
        e2e = {"value": allsum(world, pixels) / allmax(world, ew) / 1e9, "unit": "Gpixel/s",
               "h2d_bytes_per_step": int(sum(s_["h2d_bytes"] for s_ in st2)),
               "d2h_bytes_per_step": int(sum(s_["d2h_bytes"] for s_ in st2)), "ms_per_step": ew * 1e3,
               "api": "prog_bind_host (caller's pinned frame) + prog_run, host wall clock"}
        gao.prog_destroy(q)

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
            "config": {"workload": f"image_{h}x{w}_all_gpu", "h": h, "w": w,
                       "gene": format(mask, f"0{prog.n_loops}b"),
                       "l2": "working set larger than the 129 MB L2 (no flush)"},
            "launch_config": {"graph_replay": graph_replay, "fused_chain": bool(args.fuse),
                              "parallelism": f"replicas{world}" if world > 1 else "single"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                         "traffic": profile_traffic("kernels_ew.cu", f"edge_chain_image_{h}x{w}.md" if args.fuse
                                                    else f"stencil3_image_{h}x{w}.md"),
                         "kernel": ("edge_chain_kernel (the blur, Sobel x/y, squares, magnitude, its sum and column"
                                    " maxima in one pass over the raw frame)" if args.fuse else "stencil3 passes")
                                   + f" ({st_bpp:.1f} algorithmic bytes per pixel over the passes)",
                         "peak_source": f"{peaks()['source']} hbm_gbs",
                         "alu": {"ops_per_pixel": ops_px, "achieved": alu_achieved, "peak": fp32_peak,
                                 "unit": "T lane-op/s", "frac": alu_achieved / fp32_peak,
                                 "peak_source": "152 SMs x 128 FP32 lanes x 2070 MHz"}},
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": T["launches"], "clocks": clocks,
            "unfused_chain": unfused, "loop_ms": per_loop, "loop_gbs": loop_gbs, "ga_search": search}
    print(json.dumps(line), flush=True)


def batch_arm(args, world, rank, local):
    """Batched-population workload as its own line: value = GA fitness evaluations per
    second (individuals scored, measured or served from the cache, over the GA's wall time)."""
    import torch

    import paper_1806_01430_gb300 as gao
    torch.cuda.set_device(local)
    clk = clock_sampler(local)
    with clk:
        t0 = clk.mark()
        r = batch_result(args, gao, torch, args.programs, args.pop, args.generations, args.prec)
        t1 = clk.mark()
    wall = allmax(world, r["ga_wall_s"])
    evals = allsum(world, args.pop * args.generations)
    if rank == 0:
        line = {"metric": "ga_evals_per_s", "value": evals / wall, "unit": "evals/s", "n_gpus": world,
                "steps": args.generations, "warmup": 1, "ms_per_step": wall / args.generations * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.prec,
                "data": "synthetic (seeded counter hash, U[-1,1))",
                "config": {"workload": r["workload"], "programs": args.programs, "pop": args.pop,
                           "generations": args.generations, "gemm": args.prec},
                "batch": r, "clocks": clk.summary(t0, t1)}
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=8192)
    ap.add_argument("--workload", default="gemm", choices=["gemm", "six_loop", "twelve_loop", "batch", "image"])
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
                    help="GEMM arithmetic (default: bf16x6 for the GEMM and six-loop programs, bf16x3 for the "
                         "twelve-loop program and the batch, as their configurations state)")
    ap.add_argument("--no-check", dest="check", action="store_false")
    ap.add_argument("--no-e2e", dest="e2e", action="store_false")
    ap.add_argument("--no-compare", dest="compare", action="store_false",
                    help="skip the other GEMM arithmetics at the same n")
    ap.add_argument("--no-cpu", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-search", dest="search", action="store_false")
    ap.add_argument("--no-sub", dest="sub", action="store_false",
                    help="skip the batched-GA, twelve-loop and search sub-results of the default line")
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
    elif args.workload == "gemm":
        gemm_arm(args, world, rank, local)
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
