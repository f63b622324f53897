"""Seeded workload descriptions shared by the oracle, the tests and bench.py.

Plain data only: buffer shapes, loop lists, seeds and GA parameters.  None of
the method's arithmetic lives here; the FP64 oracle (``oracle/``) and the CUDA
library (``paper_1806_01430_gb300``) each compute from these descriptions on
their own.  Every matrix input is produced by the program's own INIT loop from
its seed (counter hash, implemented separately on each side), so nothing
random is generated in this module except the GA test tables at the bottom.

Programs follow the loop program of the paper's evaluation (Sec. 5.1.1: a
matrix-product benchmark whose loops the paper does not list).  The six-loop
program is init / GEMM / scale-add / transpose / row sums / Frobenius norm; the
twelve-loop program adds four element-wise and two reduction loops.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

# gao_loop_kind values (include/gao.h)
INIT, GEMM, AXPY, TRANSPOSE, ROWSUM, FROBENIUS, RELU, SQUARE, COLMAX, SUM, STENCIL3, RECURRENCE, FIND = range(13)
KIND_NAMES = ["init", "gemm", "axpy", "transpose", "rowsum", "frobenius", "relu", "square", "colmax", "sum",
              "stencil3", "recurrence", "find"]
EXTERNAL_CALL = 1 << 63  # loop flag: the body calls a host routine
# STENCIL3 presets (loop flags)
BLUR, LAPLACIAN, SOBEL_X, SOBEL_Y = range(4)
# gao_dtype
F32, F64 = 0, 1
# gao_buf_role
TEMP, INPUT, OUTPUT = 0, 1, 2
# gao_gemm_prec
FP32_SIMT, BF16, BF16X3, BF16X6, FP8 = range(5)
PREC_NAMES = ["fp32_simt", "bf16", "bf16x3", "bf16x6", "fp8"]


@dataclass
class Buffer:
    name: str
    rows: int
    cols: int
    dtype: int = F32
    role: int = TEMP


@dataclass
class Loop:
    kind: int
    ins: List[int]
    outs: List[int]
    alpha: float = 0.0
    beta: float = 0.0
    flags: int = 0


@dataclass
class Program:
    name: str
    buffers: List[Buffer]
    loops: List[Loop]
    seed: int
    meta: dict = field(default_factory=dict)

    def index(self, name: str) -> int:
        for i, b in enumerate(self.buffers):
            if b.name == name:
                return i
        raise KeyError(name)

    @property
    def n_loops(self) -> int:
        return len(self.loops)

    def gemm_flops(self) -> float:
        """2*M*N*K summed over the GEMM loops (algorithmic flop count)."""
        tot = 0.0
        for lp in self.loops:
            if lp.kind == GEMM:
                a, b = self.buffers[lp.ins[0]], self.buffers[lp.ins[1]]
                tot += 2.0 * a.rows * b.cols * a.cols
        return tot


def six_loop(n: int, seed: int, alpha: float = 1.5, beta: float = 0.5, rowscale_a: bool = False,
             outputs=("C", "r", "f")) -> Program:
    """Six-loop program on n x n matrices: L0 init A,B,C; L1 C = alpha*A@B + beta*C;
    L2 D = C + 2A; L3 E = D^T; L4 r = row sums of E; L5 f = ||E||_F."""
    names = ["A", "B", "C", "D", "E", "r", "f"]
    shapes = {"A": (n, n), "B": (n, n), "C": (n, n), "D": (n, n), "E": (n, n), "r": (n, 1), "f": (1, 1)}
    bufs = [Buffer(nm, *shapes[nm], dtype=F64 if nm == "f" else F32,
                   role=OUTPUT if nm in outputs else TEMP) for nm in names]
    A, B, C, D, E, r, f = range(7)
    loops = [
        Loop(INIT, [], [A, B, C], flags=1 if rowscale_a else 0),
        Loop(GEMM, [A, B, C], [C], alpha=alpha, beta=beta),
        Loop(AXPY, [C, A], [D], alpha=2.0),
        Loop(TRANSPOSE, [D], [E]),
        Loop(ROWSUM, [E], [r]),
        Loop(FROBENIUS, [E], [f]),
    ]
    return Program(f"six_loop_n{n}", bufs, loops, seed, {"n": n, "alpha": alpha, "beta": beta,
                                                          "rowscale_a": rowscale_a})


def gemm_only(n: int, seed: int, alpha: float = 1.5, beta: float = 0.5, rowscale_a: bool = False) -> Program:
    """The GEMM on its own, n x n: L0 init A, B, C0; L1 C = alpha*A@B + beta*C0 (the first
    two loops of the six-loop program, same hash streams: buffer ids 0, 1, 2).  C is a
    buffer of its own, so C0 is still there after a run for a residual check."""
    bufs = [Buffer("A", n, n, F32, TEMP), Buffer("B", n, n, F32, TEMP), Buffer("C0", n, n, F32, TEMP),
            Buffer("C", n, n, F32, OUTPUT)]
    loops = [Loop(INIT, [], [0, 1, 2], flags=1 if rowscale_a else 0),
             Loop(GEMM, [0, 1, 2], [3], alpha=alpha, beta=beta)]
    return Program(f"gemm_n{n}", bufs, loops, seed, {"n": n, "alpha": alpha, "beta": beta, "rowscale_a": rowscale_a})


def host_input_gemm(n: int, alpha: float = 1.5, beta: float = 0.5) -> Program:
    """The GEMM with its operands from host memory: A, B, C0 are INPUT buffers (copied to the
    device inside every run), C the OUTPUT (copied back): L0 C = alpha*A@B + beta*C0."""
    bufs = [Buffer("A", n, n, F32, INPUT), Buffer("B", n, n, F32, INPUT), Buffer("C0", n, n, F32, INPUT),
            Buffer("C", n, n, F32, OUTPUT)]
    return Program(f"host_input_gemm_n{n}", bufs, [Loop(GEMM, [0, 1, 2], [3], alpha=alpha, beta=beta)], 0,
                   {"n": n, "alpha": alpha, "beta": beta})


def host_input_program(n: int, seed: int, alpha: float = 1.5, beta: float = 0.5,
                       outputs=("r", "f")) -> Program:
    """The six-loop program without its INIT loop: A, B, C0 arrive from host memory
    (INPUT buffers) and are copied to the device inside every run.  Loops:
    L0 C = alpha*A@B + beta*C0; L1 D = C + 2A; L2 E = D^T; L3 r; L4 f."""
    names = ["A", "B", "C0", "C", "D", "E", "r", "f"]
    bufs = []
    for nm in names:
        rows, cols = (n, 1) if nm == "r" else ((1, 1) if nm == "f" else (n, n))
        role = INPUT if nm in ("A", "B", "C0") else (OUTPUT if nm in outputs else TEMP)
        bufs.append(Buffer(nm, rows, cols, F64 if nm == "f" else F32, role))
    A, B, C0, C, D, E, r, f = range(8)
    loops = [
        Loop(GEMM, [A, B, C0], [C], alpha=alpha, beta=beta),
        Loop(AXPY, [C, A], [D], alpha=2.0),
        Loop(TRANSPOSE, [D], [E]),
        Loop(ROWSUM, [E], [r]),
        Loop(FROBENIUS, [E], [f]),
    ]
    return Program(f"host_input_n{n}", bufs, loops, seed, {"n": n, "alpha": alpha, "beta": beta})


def twelve_loop(m: int, k: int, seed: int, alpha: float = 1.5, beta: float = 0.5,
                outputs=("C", "r", "f", "q", "s")) -> Program:
    """Twelve-loop program (M = N = m, inner dimension k): the six-loop program with
    the scale-add reading an m x m matrix S, plus L6 F = max(E,0); L7 G = E - 0.5F;
    L8 H = G(.)G; L9 P = H + 0.25D; L10 q = column maxima of P; L11 s = sum of P."""
    names = ["A", "B", "C", "S", "D", "E", "r", "f", "F", "G", "H", "P", "q", "s"]
    shapes = {"A": (m, k), "B": (k, m), "r": (m, 1), "f": (1, 1), "q": (1, m), "s": (1, 1)}
    bufs = []
    for nm in names:
        rows, cols = shapes.get(nm, (m, m))
        bufs.append(Buffer(nm, rows, cols, F64 if nm in ("f", "s") else F32,
                           OUTPUT if nm in outputs else TEMP))
    A, B, C, S, D, E, r, f, F, G, H, P, q, s = range(14)
    loops = [
        Loop(INIT, [], [A, B, C, S]),
        Loop(GEMM, [A, B, C], [C], alpha=alpha, beta=beta),
        Loop(AXPY, [C, S], [D], alpha=2.0),
        Loop(TRANSPOSE, [D], [E]),
        Loop(ROWSUM, [E], [r]),
        Loop(FROBENIUS, [E], [f]),
        Loop(RELU, [E], [F]),
        Loop(AXPY, [E, F], [G], alpha=-0.5),
        Loop(SQUARE, [G], [H]),
        Loop(AXPY, [H, D], [P], alpha=0.25),
        Loop(COLMAX, [P], [q]),
        Loop(SUM, [P], [s]),
    ]
    return Program(f"twelve_loop_m{m}_k{k}", bufs, loops, seed, {"m": m, "k": k, "alpha": alpha, "beta": beta})


def image_program(h: int, w: int, seed: int, outputs=("M2", "e", "q"), host_image: bool = False) -> Program:
    """Edge-detection program on an h x w image (the paper's motivating camera-analysis
    workload, Sec. 1): L0 init X; L1 B = binomial blur of X; L2 gx = Sobel-x of B;
    L3 gy = Sobel-y of B; L4 sx = gx(.)gx; L5 sy = gy(.)gy; L6 M2 = sx + sy (squared
    gradient magnitude); L7 e = sum of M2 (edge energy); L8 q = column maxima of M2.
    With ``host_image`` the image X is an INPUT buffer supplied from host memory (a
    camera frame) and the INIT loop is dropped (eight loops)."""
    names = ["X", "B", "gx", "gy", "sx", "sy", "M2", "e", "q"]
    shapes = {"e": (1, 1), "q": (1, w)}
    bufs = []
    for nm in names:
        rows, cols = shapes.get(nm, (h, w))
        role = INPUT if (nm == "X" and host_image) else (OUTPUT if nm in outputs else TEMP)
        bufs.append(Buffer(nm, rows, cols, F64 if nm == "e" else F32, role))
    X, B_, gx, gy, sx, sy, M2, e, q = range(9)
    loops = [] if host_image else [Loop(INIT, [], [X])]
    loops += [
        Loop(STENCIL3, [X], [B_], flags=BLUR),
        Loop(STENCIL3, [B_], [gx], flags=SOBEL_X),
        Loop(STENCIL3, [B_], [gy], flags=SOBEL_Y),
        Loop(SQUARE, [gx], [sx]),
        Loop(SQUARE, [gy], [sy]),
        Loop(AXPY, [sx, sy], [M2], alpha=1.0),
        Loop(SUM, [M2], [e]),
        Loop(COLMAX, [M2], [q]),
    ]
    return Program(f"image_{h}x{w}", bufs, loops, seed, {"h": h, "w": w})


ANALYSIS_ALPHA = 0.5       # decay of the recurrence loop
ANALYSIS_THRESHOLD = 0.75  # threshold of the find loop


def analysis_program(m: int, n: int, seed: int, outputs=("C", "k", "s")) -> Program:
    """Seven loops, three of which Sec. 4's parallelisability check excludes:
    L0 init X (m x n), B (n x n); L1 R = recurrence of X along rows (carried dependence);
    L2 C = R @ B; L3 T = C^T; L4 k = first column of each row of T above the threshold
    (early exit); L5 P = max(T, 0) in a loop that calls a host routine (external call);
    L6 s = sum of P.  Gene length 4 (loops 0, 2, 3, 6)."""
    names = ["X", "B", "R", "C", "T", "k", "P", "s"]
    shapes = {"X": (m, n), "B": (n, n), "R": (m, n), "C": (m, n), "T": (n, m), "k": (n, 1), "P": (n, m),
              "s": (1, 1)}
    bufs = [Buffer(nm, *shapes[nm], F64 if nm in ("k", "s") else F32, OUTPUT if nm in outputs else TEMP)
            for nm in names]
    X, B_, R, C, T, k, P, s = range(8)
    loops = [
        Loop(INIT, [], [X, B_]),
        Loop(RECURRENCE, [X], [R], alpha=ANALYSIS_ALPHA),
        Loop(GEMM, [R, B_, -1], [C], alpha=1.0, beta=0.0),
        Loop(TRANSPOSE, [C], [T]),
        Loop(FIND, [T], [k], alpha=ANALYSIS_THRESHOLD),
        Loop(RELU, [T], [P], flags=EXTERNAL_CALL),
        Loop(SUM, [P], [s]),
    ]
    return Program(f"analysis_{m}x{n}", bufs, loops, seed, {"m": m, "n": n})


# ---- seeds of the benchmark workloads -----------------------------------------
SEED_N256 = 1000         # six-loop n = 256, all-GPU gene
SEED_N4096 = 1001        # six-loop n = 4096, all 64 genes
SEED_N8192 = 1002        # n = 8192 precision study, U[-1,1)
SEED_N8192_ROWS = 1003   # n = 8192 precision study, rows of A scaled by 2^e
SEED_BATCH_BASE = 2000   # batch programs use 2000 + p
SEED_TWELVE_LOOP = 1005  # rectangular 16384 x 16384 x 4096, twelve loops
SEED_IMAGE = 1006        # edge-detection image program


def six_loop_seed(n: int) -> int:
    """Seed of the six-loop program at size n: the precision-study seed at n = 8192, the
    n = 256 seed there, the n = 4096 seed otherwise."""
    return {256: SEED_N256, 8192: SEED_N8192}.get(n, SEED_N4096)


# GA parameters of the paper's evaluation (Sec. 5.1.2)
PAPER_GA = dict(pop=12, generations=12, pc=0.9, pm=0.05, elite=1, mutation=0)


def batch_sizes(n_programs: int = 64, lo: int = 128, hi: int = 2048, base_seed: int = SEED_BATCH_BASE):
    """Square sizes log-uniform in [lo, hi] for the batched-population workload;
    program p draws from numpy's PCG64 seeded with base_seed + p."""
    out = []
    for p in range(n_programs):
        rng = np.random.default_rng(base_seed + p)
        out.append(int(round(float(np.exp(rng.uniform(np.log(lo), np.log(hi)))))))
    return out


def random_time_table(n_genes: int, seed: int, fail_frac: float = 0.0) -> np.ndarray:
    """A synthetic gene -> time table for GA tests: log-normal times, with an optional
    fraction of failed genes marked by -1."""
    rng = np.random.default_rng(seed)
    t = np.exp(rng.normal(0.0, 1.0, size=1 << n_genes))
    if fail_frac > 0:
        t[rng.random(1 << n_genes) < fail_frac] = -1.0
    return t


def loop_time_table(n_genes: int, seed: int, transfer: float = 0.3) -> np.ndarray:
    """A synthetic gene -> time table shaped like a loop program's: each loop has a
    CPU time and a GPU time (log-normal), and every change of side between
    consecutive loops, including the start and end on the host, costs `transfer`
    (the data the next loop reads has to move)."""
    rng = np.random.default_rng(seed)
    cpu = np.exp(rng.normal(0.0, 1.0, size=n_genes))
    gpu = np.exp(rng.normal(-1.0, 1.0, size=n_genes))
    out = np.empty(1 << n_genes)
    for m in range(1 << n_genes):
        t, side = 0.0, 0
        for i in range(n_genes):
            b = (m >> i) & 1
            t += gpu[i] if b else cpu[i]
            if b != side:
                t += transfer
            side = b
        if side:
            t += transfer
        out[m] = t
    return out
