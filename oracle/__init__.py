"""FP64 CPU oracle of the GA-offload loop program and of its Simple GA.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference leg of bench.py may import this package.  It shares no
code with the CUDA library and never imports it.

* ``oracle.c`` (compiled here with gcc into ``_build/liboracle.so``) holds each
  loop of the program as its plain definition in binary64, plus the
  SplitMix64 counter hash that generates the seeded inputs.
* ``run_program`` evaluates a ``workloads.Program`` loop by loop in program
  order.  A gene never changes the result (Sec. 4: the gene only decides where a
  loop runs), so the oracle has no gene argument.
* ``oracle.ga`` is the Simple GA of Sec. 3.3 / Sec. 4 / Sec. 5.1.2 in plain Python.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_d = ctypes.c_double
_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64
_P = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_PI = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_PU = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (IEEE arithmetic: no fast-math, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
               "-std=c11", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            L.orc_splitmix64.restype = _u64
            L.orc_splitmix64.argtypes = [_u64]
            L.orc_splitmix64_stream.argtypes = [_u64, _i64, _PU]
            L.orc_init_value.restype = _d
            L.orc_init_value.argtypes = [_u64, _i64, _i64]
            L.orc_row_exponent.restype = _i64
            L.orc_row_exponent.argtypes = [_u64, _i64]
            L.orc_init.argtypes = [_u64, _i64, _i64, _i64, ctypes.c_int, _P]
            L.orc_gemm.argtypes = [_i64, _i64, _i64, _d, _P, _P, _d, _P, _P]
            L.orc_axpy.argtypes = [_i64, _P, _d, _P, _P]
            L.orc_transpose.argtypes = [_i64, _i64, _P, _P]
            L.orc_rowsum.argtypes = [_i64, _i64, _P, _P]
            L.orc_frobenius.restype = _d
            L.orc_frobenius.argtypes = [_i64, _P]
            L.orc_relu.argtypes = [_i64, _P, _P]
            L.orc_square.argtypes = [_i64, _P, _P]
            L.orc_colmax.argtypes = [_i64, _i64, _P, _P]
            L.orc_sum.restype = _d
            L.orc_sum.argtypes = [_i64, _P]
            L.orc_gemm_init_entries.argtypes = [_u64, _i64, _i64, _i64, ctypes.c_int, _i64, _i64, _i64, _d, _d,
                                                _i64, _PI, _PI, _P]
            L.orc_gemm_column.argtypes = [_i64, _i64, _i64, _d, _P, _P, _d, _P, _i64, _P]
            L.orc_stencil3.restype = ctypes.c_int
            L.orc_stencil3.argtypes = [_i64, _i64, _P, ctypes.c_int, _P]
            L.orc_recurrence.argtypes = [_i64, _i64, _P, _d, _P]
            L.orc_find.argtypes = [_i64, _i64, _P, _d, _P]
            L.orc_num_threads.restype = ctypes.c_int
            L.orc_set_num_threads.argtypes = [ctypes.c_int]
            _lib = L
    return _lib


def _c(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ---- counter hash ------------------------------------------------------------

def splitmix64(state: int) -> int:
    return int(lib().orc_splitmix64(state & 0xFFFFFFFFFFFFFFFF))


def splitmix64_stream(seed: int, n: int) -> np.ndarray:
    out = np.zeros(n, dtype=np.uint64)
    lib().orc_splitmix64_stream(seed, n, out)
    return out


def init_value(seed: int, buf: int, idx: int) -> float:
    return float(lib().orc_init_value(seed, buf, idx))


def row_exponent(seed: int, row: int) -> int:
    return int(lib().orc_row_exponent(seed, row))


def init_matrix(seed: int, buf: int, rows: int, cols: int, rowscale: bool = False) -> np.ndarray:
    out = np.empty((rows, cols), dtype=np.float64)
    lib().orc_init(seed, buf, rows, cols, 1 if rowscale else 0, out)
    return out


# ---- loops -------------------------------------------------------------------

def gemm(A, B, C0, alpha: float, beta: float) -> np.ndarray:
    A, B, C0 = _c(A), _c(B), _c(C0)
    M, K = A.shape
    K2, N = B.shape
    assert K == K2 and C0.shape == (M, N)
    C = np.empty((M, N), dtype=np.float64)
    lib().orc_gemm(M, N, K, alpha, A, B, beta, C0, C)
    return C


def axpy(x, alpha: float, y) -> np.ndarray:
    x, y = _c(x), _c(y)
    assert x.shape == y.shape
    out = np.empty_like(x)
    lib().orc_axpy(x.size, x, alpha, y, out)
    return out


def transpose(X) -> np.ndarray:
    X = _c(X)
    r, c = X.shape
    out = np.empty((c, r), dtype=np.float64)
    lib().orc_transpose(r, c, X, out)
    return out


def rowsum(X) -> np.ndarray:
    X = _c(X)
    r, c = X.shape
    out = np.empty((r, 1), dtype=np.float64)
    lib().orc_rowsum(r, c, X, out)
    return out


def frobenius(X) -> float:
    X = _c(X)
    return float(lib().orc_frobenius(X.size, X))


def relu(X) -> np.ndarray:
    X = _c(X)
    out = np.empty_like(X)
    lib().orc_relu(X.size, X, out)
    return out


def square(X) -> np.ndarray:
    X = _c(X)
    out = np.empty_like(X)
    lib().orc_square(X.size, X, out)
    return out


def colmax(X) -> np.ndarray:
    X = _c(X)
    r, c = X.shape
    out = np.empty((1, c), dtype=np.float64)
    lib().orc_colmax(r, c, X, out)
    return out


def total(X) -> float:
    X = _c(X)
    return float(lib().orc_sum(X.size, X))


STENCIL_PRESETS = {"blur": 0, "laplacian": 1, "sobel_x": 2, "sobel_y": 3}


def stencil3(X, preset: int) -> np.ndarray:
    X = _c(X)
    r, c = X.shape
    out = np.empty_like(X)
    if lib().orc_stencil3(r, c, X, int(preset), out) != 0:
        raise ValueError("unknown stencil preset")
    return out


def recurrence(X, alpha: float) -> np.ndarray:
    X = _c(X)
    r, c = X.shape
    out = np.empty_like(X)
    lib().orc_recurrence(r, c, X, float(alpha), out)
    return out


def find_first(X, threshold: float) -> np.ndarray:
    X = _c(X)
    r, c = X.shape
    out = np.empty((r, 1), dtype=np.float64)
    lib().orc_find(r, c, X, float(threshold), out)
    return out


def gemm_init_entries(seed: int, bufs, rowscale_a: bool, M: int, N: int, K: int, alpha: float, beta: float,
                      ii, jj) -> np.ndarray:
    """C[i,j] of C = alpha*A@B + beta*C0 for freshly initialised A, B, C0 (buffer ids
    bufs = (a, b, c)), computed entry by entry without materialising the matrices."""
    ii = np.ascontiguousarray(ii, dtype=np.int64)
    jj = np.ascontiguousarray(jj, dtype=np.int64)
    out = np.empty(ii.size, dtype=np.float64)
    lib().orc_gemm_init_entries(seed, bufs[0], bufs[1], bufs[2], 1 if rowscale_a else 0, M, N, K, alpha, beta,
                                ii.size, ii, jj, out)
    return out


def gemm_column(A, B, C0, alpha: float, beta: float, j: int) -> np.ndarray:
    A, B, C0 = _c(A), _c(B), _c(C0)
    M, K = A.shape
    N = B.shape[1]
    out = np.empty(M, dtype=np.float64)
    lib().orc_gemm_column(M, N, K, alpha, A, B, beta, C0, j, out)
    return out


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_num_threads(n: int) -> None:
    lib().orc_set_num_threads(n)


# ---- whole program -------------------------------------------------------------

# loop kinds (gao_loop_kind); kept as literals so that the oracle does not depend
# on the product package.
_INIT, _GEMM, _AXPY, _TRANSPOSE, _ROWSUM, _FROB, _RELU, _SQUARE, _COLMAX, _SUM, _STENCIL3, _RECURRENCE, _FIND = range(13)
_EXTERNAL_CALL = 1 << 63  # loop flag that only decides placement


def run_program(prog, inputs: dict | None = None) -> dict:
    """Evaluate every loop of ``prog`` (a workloads.Program) in order, in binary64.

    ``inputs`` maps INPUT buffer names to arrays (host-supplied data).  Returns a
    dict buffer name -> ndarray (matrices, vectors) or float (scalar buffers)."""
    vals: dict = {}
    if inputs:
        for k, v in inputs.items():
            vals[prog.index(k)] = _c(v)
    for lp in prog.loops:
        ins = [vals[i] for i in lp.ins if i >= 0]
        o = lp.outs[0]
        if lp.kind == _INIT:
            for t, ob in enumerate(lp.outs):
                b = prog.buffers[ob]
                vals[ob] = init_matrix(prog.seed, ob, b.rows, b.cols, bool((lp.flags >> t) & 1))
        elif lp.kind == _GEMM:
            c0 = ins[2] if len(ins) > 2 else np.zeros((ins[0].shape[0], ins[1].shape[1]))  # no C0: beta = 0
            vals[o] = gemm(ins[0], ins[1], c0, lp.alpha, lp.beta if len(ins) > 2 else 0.0)
        elif lp.kind == _AXPY:
            vals[o] = axpy(ins[0], lp.alpha, ins[1])
        elif lp.kind == _TRANSPOSE:
            vals[o] = transpose(ins[0])
        elif lp.kind == _ROWSUM:
            vals[o] = rowsum(ins[0])
        elif lp.kind == _FROB:
            vals[o] = frobenius(ins[0])
        elif lp.kind == _RELU:
            vals[o] = relu(ins[0])
        elif lp.kind == _SQUARE:
            vals[o] = square(ins[0])
        elif lp.kind == _COLMAX:
            vals[o] = colmax(ins[0])
        elif lp.kind == _SUM:
            vals[o] = total(ins[0])
        elif lp.kind == _STENCIL3:
            vals[o] = stencil3(ins[0], lp.flags & ~_EXTERNAL_CALL)
        elif lp.kind == _RECURRENCE:
            vals[o] = recurrence(ins[0], lp.alpha)
        elif lp.kind == _FIND:
            vals[o] = find_first(ins[0], lp.alpha)
        else:
            raise ValueError(f"unknown loop kind {lp.kind}")
    return {prog.buffers[i].name: v for i, v in vals.items()}


def rel_err(x, ref) -> float:
    """Normwise relative error ||x - ref||_F / ||ref||_F (scalars: |x-ref|/|ref|)."""
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = float(np.linalg.norm(ref.ravel()))
    num = float(np.linalg.norm((x - ref).ravel()))
    if den == 0.0:
        return num
    return num / den
