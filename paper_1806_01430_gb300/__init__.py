"""Python binding of libgao.so (include/gao.h): argument marshalling only.

Every step of a program runs inside the C library (CUDA kernels for gene bits set
to 1, the library's own OpenMP loops for bits set to 0).  There is no Python or
CPU fallback: if the shared library is missing, importing the binding's entry
points raises.  PyTorch is optional plumbing: ``prog_create`` accepts a
``torch.cuda.Stream`` (or raw handle) and a device arena tensor.

Names follow the C ABI: prog_create, prog_run, prog_output, prog_stats,
ga_evaluate, ga_run, ga_run_table, prog_destroy, gao_last_error.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Dict, List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgao.so")

# enums (include/gao.h)
GAO_OK, GAO_EINVAL, GAO_ENOMEM, GAO_ECUDA, GAO_ETIMEOUT, GAO_EDEVICE, GAO_ENODEV, GAO_ECPU = range(8)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "ETIMEOUT", "EDEVICE", "ENODEV", "ECPU"]
INIT, GEMM, AXPY, TRANSPOSE, ROWSUM, FROBENIUS, RELU, SQUARE, COLMAX, SUM, STENCIL3, RECURRENCE, FIND = range(13)
LOOP_EXTERNAL_CALL = 1 << 63  # loop flag: the body calls a host routine (never offloaded)
OFFLOAD_OK, OFFLOAD_DEPENDENCE, OFFLOAD_EARLY_EXIT, OFFLOAD_EXTERNAL_CALL = range(4)
OFFLOAD_NAMES = ["ok", "dependence", "early_exit", "external_call"]
STENCIL_BLUR, STENCIL_LAPLACIAN, STENCIL_SOBEL_X, STENCIL_SOBEL_Y = range(4)  # STENCIL3 loop flags
F32, F64 = 0, 1
TEMP, INPUT, OUTPUT = 0, 1, 2
FP32_SIMT, BF16, BF16X3, BF16X6, FP8 = range(5)
PREC_NAMES = ["fp32_simt", "bf16", "bf16x3", "bf16x6", "fp8"]
RUN_KEEP_DEVICE = 1
RUN_NO_GRAPH = 2  # plain launches: no CUDA graph captured or replayed
RUN_NO_LOOP_TIMES = 4  # no per-loop CUDA events: prog_stats reports no loop times for the run
TRANSFER_RESIDENT, TRANSFER_PER_LOOP = 0, 1
FUSE_OFF, FUSE_ON, FUSE_GENE = 0, 1, 2
MAX_IO = 4


class gao_buffer(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int64), ("cols", ctypes.c_int64), ("dtype", ctypes.c_int32),
                ("role", ctypes.c_int32)]


class gao_loop(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("ins", ctypes.c_int32 * MAX_IO), ("outs", ctypes.c_int32 * MAX_IO),
                ("alpha", ctypes.c_double), ("beta", ctypes.c_double), ("flags", ctypes.c_uint64)]


class gao_opts(ctypes.Structure):
    _fields_ = [("gemm_prec", ctypes.c_int32), ("kchunk", ctypes.c_int32), ("tile_cfg", ctypes.c_int32),
                ("cpu_threads", ctypes.c_int32), ("seed", ctypes.c_uint64), ("timeout_s", ctypes.c_double),
                ("stream", ctypes.c_void_p), ("dev_arena", ctypes.c_void_p), ("dev_arena_bytes", ctypes.c_uint64),
                ("transfer_mode", ctypes.c_int32), ("fuse_chains", ctypes.c_int32)]


class gao_loop_stat(ctypes.Structure):
    _fields_ = [("placement", ctypes.c_int32), ("launches", ctypes.c_int32), ("device_ms", ctypes.c_double),
                ("kernel_ms", ctypes.c_double), ("cpu_ms", ctypes.c_double), ("copy_ms", ctypes.c_double),
                ("h2d_bytes", ctypes.c_uint64), ("d2h_bytes", ctypes.c_uint64)]


class gao_ga_params(ctypes.Structure):
    _fields_ = [("pop", ctypes.c_int32), ("generations", ctypes.c_int32), ("pc", ctypes.c_double),
                ("pm", ctypes.c_double), ("elite", ctypes.c_int32), ("mutation", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("timeout_s", ctypes.c_double)]


class gao_ga_gen(ctypes.Structure):
    _fields_ = [("best_mask", ctypes.c_uint64), ("best_s", ctypes.c_double), ("mean_s", ctypes.c_double),
                ("evaluated", ctypes.c_int32), ("cache_hits", ctypes.c_int32), ("wall_s", ctypes.c_double)]


class gao_ga_result(ctypes.Structure):
    _fields_ = [("best_mask", ctypes.c_uint64), ("best_s", ctypes.c_double), ("evaluations", ctypes.c_int32),
                ("cache_hits", ctypes.c_int32), ("history", ctypes.POINTER(gao_ga_gen)),
                ("populations", ctypes.POINTER(ctypes.c_uint64))]


class gao_autotune_result(ctypes.Structure):
    _fields_ = [("kchunk", ctypes.c_int32), ("tile_cfg", ctypes.c_int32), ("best_ms", ctypes.c_double),
                ("default_ms", ctypes.c_double), ("evaluations", ctypes.c_int32), ("_pad", ctypes.c_int32)]


class gao_batch_stat(ctypes.Structure):
    _fields_ = [("executed", ctypes.c_int64), ("served", ctypes.c_int64), ("exec_seconds", ctypes.c_double),
                ("gemm_phase_ms", ctypes.c_double), ("gemm_flops", ctypes.c_double), ("gemm_tiles", ctypes.c_int32),
                ("launches_per_gene", ctypes.c_int32), ("graphs", ctypes.c_int32), ("fused_phases", ctypes.c_int32),
                ("kernel_launches", ctypes.c_int64), ("grouped_launches", ctypes.c_int64),
                ("grouped_genes", ctypes.c_int64), ("replicas", ctypes.c_int32), ("_pad", ctypes.c_int32)]


class gao_residual(ctypes.Structure):
    _fields_ = [("right", ctypes.c_double), ("left", ctypes.c_double), ("right_inf", ctypes.c_double),
                ("left_inf", ctypes.c_double), ("right_argmax", ctypes.c_int64), ("left_argmax", ctypes.c_int64)]


# every entry point of include/gao.h: name -> (restype, argtypes)
_P = ctypes.c_void_p
SIGNATURES = {
    "prog_device_bytes": (ctypes.c_int, [ctypes.POINTER(gao_loop), ctypes.c_int, ctypes.POINTER(gao_buffer),
                                         ctypes.c_int, ctypes.POINTER(gao_opts), ctypes.POINTER(ctypes.c_uint64)]),
    "prog_create": (ctypes.c_int, [ctypes.POINTER(gao_loop), ctypes.c_int, ctypes.POINTER(gao_buffer), ctypes.c_int,
                                   ctypes.POINTER(gao_opts), ctypes.POINTER(_P)]),
    "prog_set_input": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_uint64]),
    "prog_bind_host": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_uint64]),
    "prog_run": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_uint32, ctypes.POINTER(ctypes.c_double)]),
    "prog_output": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(_P), ctypes.POINTER(gao_buffer)]),
    "prog_gene_length": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int)]),
    "prog_graphs": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "prog_cache_export": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_double),
                                         ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "prog_cache_import": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_double),
                                         ctypes.c_int]),
    "prog_loop_offload": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "prog_device_ptr": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(_P)]),
    "prog_planes_for": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "prog_stats": (ctypes.c_int, [_P, ctypes.POINTER(gao_loop_stat), ctypes.c_int]),
    "prog_cache_clear": (ctypes.c_int, [_P]),
    "prog_destroy": (None, [_P]),
    "ga_evaluate": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(ctypes.c_uint64), ctypes.c_int,
                                   ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_int)]),
    "ga_run": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(gao_ga_params),
                              ctypes.POINTER(gao_ga_result)]),
    "ga_run_table": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.POINTER(gao_ga_params),
                                    ctypes.POINTER(gao_ga_result)]),
    "gao_last_error": (ctypes.c_char_p, []),
    "gao_version": (ctypes.c_char_p, []),
    "gao_selftest_device_wait": (ctypes.c_int, [ctypes.c_double, _P]),
    "gao_colmax_noalloc": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int64, _P, _P]),
    "gao_gemm_residual_scratch": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                                 ctypes.POINTER(ctypes.c_uint64)]),
    "gao_gemm_residual": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                         ctypes.c_double, ctypes.c_double, _P, _P, _P, ctypes.c_uint64, _P, _P,
                                         ctypes.POINTER(gao_residual), _P]),
    "prog_gemm_residual": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_double), ctypes.POINTER(gao_residual)]),
    "batch_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(_P)]),
    "batch_set_replicas": (ctypes.c_int, [_P, ctypes.c_int]),
    "batch_replica_prog": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_P)]),
    "batch_evaluate": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint64), ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_int)]),
    "batch_ga_run": (ctypes.c_int, [_P, ctypes.POINTER(gao_ga_params), ctypes.POINTER(gao_ga_result)]),
    "batch_stats": (ctypes.c_int, [_P, ctypes.POINTER(gao_batch_stat)]),
    "batch_destroy": (None, [_P]),
    "ga_run_callback": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(gao_ga_params), ctypes.c_void_p, _P,
                                       ctypes.POINTER(gao_ga_result)]),
    "prog_autotune": (ctypes.c_int, [_P, ctypes.POINTER(gao_ga_params), ctypes.POINTER(gao_autotune_result)]),
    "batch_autotune": (ctypes.c_int, [_P, ctypes.POINTER(gao_ga_params), ctypes.POINTER(gao_autotune_result)]),
}

_lib = None


def lib() -> ctypes.CDLL:
    """Load libgao.so from the package directory (built by _build.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                               "(there is no fallback implementation)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class GaoError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = lib().gao_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")


def _check(st: int, where: str):
    if st != GAO_OK:
        raise GaoError(st, where)


def gao_last_error() -> str:
    return lib().gao_last_error().decode(errors="replace")


def gao_version() -> str:
    return lib().gao_version().decode()


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


def _marshal(buffers, loops):
    nb, nl = len(buffers), len(loops)
    cb = (gao_buffer * nb)()
    for i, b in enumerate(buffers):
        cb[i].rows, cb[i].cols, cb[i].dtype, cb[i].role = int(b.rows), int(b.cols), int(b.dtype), int(b.role)
    cl = (gao_loop * nl)()
    for i, lp in enumerate(loops):
        cl[i].kind = int(lp.kind)
        ins = list(lp.ins) + [-1] * (MAX_IO - len(lp.ins))
        outs = list(lp.outs) + [-1] * (MAX_IO - len(lp.outs))
        for t in range(MAX_IO):
            cl[i].ins[t] = ins[t]
            cl[i].outs[t] = outs[t]
        cl[i].alpha, cl[i].beta, cl[i].flags = float(lp.alpha), float(lp.beta), int(lp.flags)
    return cb, nb, cl, nl


def _opts(seed, gemm_prec, kchunk, tile_cfg, cpu_threads, timeout_s, stream, arena_ptr, arena_bytes,
          transfer_mode=TRANSFER_RESIDENT, fuse_chains=FUSE_OFF):
    o = gao_opts()
    o.transfer_mode = int(transfer_mode)
    o.fuse_chains = int(fuse_chains)  # False/True or FUSE_OFF/FUSE_ON/FUSE_GENE
    o.gemm_prec, o.kchunk, o.tile_cfg, o.cpu_threads = int(gemm_prec), int(kchunk), int(tile_cfg), int(cpu_threads)
    o.seed, o.timeout_s = int(seed), float(timeout_s)
    o.stream = _stream_handle(stream)
    o.dev_arena = arena_ptr
    o.dev_arena_bytes = int(arena_bytes)
    return o


class Prog:
    """Handle of a gao_prog (owning)."""

    def __init__(self, handle, buffers, loops, arena=None):
        self.handle = handle
        self.buffers = list(buffers)
        self.loops = list(loops)
        self._arena = arena  # keeps a caller/torch arena alive
        self.bound = {}  # host arrays bound with prog_bind_host, kept alive while bound
        self.owned = True  # False for a borrowed handle (a batch's copy of a program)

    @property
    def n_loops(self) -> int:
        return len(self.loops)

    def __del__(self):
        try:
            prog_destroy(self)
        except Exception:
            pass


def prog_device_bytes(buffers, loops, seed=0, gemm_prec=FP32_SIMT, kchunk=0, tile_cfg=0) -> int:
    cb, nb, cl, nl = _marshal(buffers, loops)
    o = _opts(seed, gemm_prec, kchunk, tile_cfg, 0, 0.0, None, None, 0)
    out = ctypes.c_uint64(0)
    _check(lib().prog_device_bytes(cl, nl, cb, nb, ctypes.byref(o), ctypes.byref(out)), "prog_device_bytes")
    return int(out.value)


def prog_create(buffers, loops, seed: int = 0, gemm_prec: int = FP32_SIMT, kchunk: int = 0, tile_cfg: int = 0,
                cpu_threads: int = 0, timeout_s: float = 0.0, stream=None, arena=None,
                transfer_mode: int = TRANSFER_RESIDENT, fuse_chains: int = FUSE_OFF) -> Prog:
    """Declare a program.  ``buffers``/``loops`` are sequences of objects with the
    gao_buffer / gao_loop fields (e.g. workloads.Buffer / workloads.Loop).  ``arena``:
    optional device memory (a torch uint8 CUDA tensor, or (ptr, bytes))."""
    cb, nb, cl, nl = _marshal(buffers, loops)
    ptr, nbytes, keep = None, 0, None
    if arena is not None:
        if isinstance(arena, tuple):
            ptr, nbytes = int(arena[0]), int(arena[1])
        else:
            ptr, nbytes, keep = int(arena.data_ptr()), int(arena.numel() * arena.element_size()), arena
    o = _opts(seed, gemm_prec, kchunk, tile_cfg, cpu_threads, timeout_s, stream, ptr, nbytes, transfer_mode,
              fuse_chains)
    h = ctypes.c_void_p(None)
    _check(lib().prog_create(cl, nl, cb, nb, ctypes.byref(o), ctypes.byref(h)), "prog_create")
    return Prog(h, buffers, loops, keep)


def prog_from_workload(program, **kw) -> Prog:
    """prog_create from a workloads.Program (uses its seed)."""
    return prog_create(program.buffers, program.loops, seed=program.seed, **kw)


def prog_set_input(p: Prog, buf: int, data: np.ndarray) -> None:
    a = np.ascontiguousarray(data, dtype=np.float64 if p.buffers[buf].dtype == F64 else np.float32)
    _check(lib().prog_set_input(p.handle, buf, a.ctypes.data_as(ctypes.c_void_p), a.nbytes), "prog_set_input")


def prog_bind_host(p: Prog, buf: int, arr) -> None:
    """Bind a caller array (numpy array or pinned torch CPU tensor; None unbinds) as buffer
    ``buf``'s host copy: runs copy inputs from it and outputs into it directly.  The caller
    keeps ``arr`` alive while it is bound (the Prog object holds a reference too)."""
    if arr is None:
        _check(lib().prog_bind_host(p.handle, buf, None, 0), "prog_bind_host")
        p.bound.pop(buf, None)
        return
    if hasattr(arr, "data_ptr"):  # torch tensor
        ptr, nbytes = arr.data_ptr(), arr.numel() * arr.element_size()
    else:
        if not (isinstance(arr, np.ndarray) and arr.flags["C_CONTIGUOUS"]):
            raise ValueError("prog_bind_host needs a C-contiguous numpy array or a torch tensor")
        ptr, nbytes = arr.ctypes.data, arr.nbytes
    _check(lib().prog_bind_host(p.handle, buf, ctypes.c_void_p(ptr), ctypes.c_uint64(nbytes)), "prog_bind_host")
    p.bound[buf] = arr


def prog_gene_length(p: Prog) -> int:
    """Gene length a: the number of offloadable loops."""
    a = ctypes.c_int(0)
    _check(lib().prog_gene_length(p.handle, ctypes.byref(a)), "prog_gene_length")
    return int(a.value)


def prog_loop_offload(p: Prog, loop: int):
    """(verdict, gene bit) of one loop; verdict is one of OFFLOAD_*, gene bit -1 when not offloadable."""
    v, g = ctypes.c_int(0), ctypes.c_int(0)
    _check(lib().prog_loop_offload(p.handle, loop, ctypes.byref(v), ctypes.byref(g)), "prog_loop_offload")
    return int(v.value), int(g.value)


def prog_graphs(p: Prog):
    """(genes replayed from a captured graph, genes whose capture failed)."""
    c, f = ctypes.c_int(0), ctypes.c_int(0)
    _check(lib().prog_graphs(p.handle, ctypes.byref(c), ctypes.byref(f)), "prog_graphs")
    return int(c.value), int(f.value)


def prog_cache_export(p: Prog):
    """(genes, seconds) of every measured gene, in gene order."""
    n = ctypes.c_int(0)
    _check(lib().prog_cache_export(p.handle, None, None, 0, ctypes.byref(n)), "prog_cache_export")
    g = (ctypes.c_uint64 * max(1, n.value))()
    t = (ctypes.c_double * max(1, n.value))()
    _check(lib().prog_cache_export(p.handle, g, t, n.value, ctypes.byref(n)), "prog_cache_export")
    return [int(g[i]) for i in range(n.value)], [float(t[i]) for i in range(n.value)]


def prog_cache_import(p: Prog, genes, seconds) -> None:
    k = len(genes)
    assert len(seconds) == k
    g = (ctypes.c_uint64 * max(1, k))(*[int(x) for x in genes])
    t = (ctypes.c_double * max(1, k))(*[float(x) for x in seconds])
    _check(lib().prog_cache_import(p.handle, g, t, k), "prog_cache_import")


def ga_checkpoint(progs: Sequence[Prog], path: str) -> None:
    """Write every program's measured gene times to a JSON file (a search checkpoint)."""
    import json
    data = {"programs": []}
    for p in progs:
        g, t = prog_cache_export(p)
        data["programs"].append({"genes": g, "seconds": t})
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f)
    os.replace(tmp, path)


def ga_resume(progs: Sequence[Prog], path: str) -> None:
    """Load a checkpoint written by ga_checkpoint into the programs' caches; a ga_run with
    the same parameters and seed then continues the search where it stopped."""
    import json
    with open(path) as f:
        data = json.load(f)
    if len(data["programs"]) != len(progs):
        raise ValueError("checkpoint holds a different number of programs")
    for p, e in zip(progs, data["programs"]):
        prog_cache_import(p, e["genes"], e["seconds"])


def prog_run(p: Prog, gene_mask: int, flags: int = 0) -> float:
    """Run under a gene; returns the wall seconds of the run."""
    s = ctypes.c_double(0.0)
    _check(lib().prog_run(p.handle, ctypes.c_uint64(gene_mask), flags, ctypes.byref(s)), "prog_run")
    return float(s.value)


def prog_run_status(p: Prog, gene_mask: int, flags: int = 0):
    """Like prog_run but returns (status, seconds) instead of raising."""
    s = ctypes.c_double(0.0)
    st = lib().prog_run(p.handle, ctypes.c_uint64(gene_mask), flags, ctypes.byref(s))
    return int(st), float(s.value)


def prog_output(p: Prog, buf: int) -> np.ndarray:
    """Copy of buffer ``buf``'s host data after a run (float32 matrix or float64 scalar)."""
    ptr = ctypes.c_void_p(None)
    shp = gao_buffer()
    _check(lib().prog_output(p.handle, buf, ctypes.byref(ptr), ctypes.byref(shp)), "prog_output")
    n = shp.rows * shp.cols
    ct = ctypes.c_double if shp.dtype == F64 else ctypes.c_float
    arr = np.ctypeslib.as_array(ctypes.cast(ptr, ctypes.POINTER(ct)), shape=(max(n, 1),))[:n]
    return arr.reshape(shp.rows, shp.cols).copy()


def prog_device_ptr(p: Prog, buf: int) -> int:
    ptr = ctypes.c_void_p(None)
    _check(lib().prog_device_ptr(p.handle, buf, ctypes.byref(ptr)), "prog_device_ptr")
    return int(ptr.value or 0)


def prog_planes_for(p: Prog, buf: int) -> int:
    """The GEMM loop whose bfloat16 planes the last run formed buffer `buf` into (the INIT
    loop skipped its binary32 array), or -1."""
    g = ctypes.c_int(-1)
    _check(lib().prog_planes_for(p.handle, buf, ctypes.byref(g)), "prog_planes_for")
    return g.value


def _residual_dict(r: "gao_residual") -> Dict:
    return {k: getattr(r, k) for k, _ in gao_residual._fields_}


def prog_gemm_residual(p: Prog, loop: int, x: np.ndarray, y: np.ndarray) -> Dict:
    """Freivalds' residual check of GEMM loop ``loop`` after a run, in binary64 on the GPU;
    x (N) and y (M) are host vectors.  Returns the gao_residual fields as a dict."""
    xa = np.ascontiguousarray(x, dtype=np.float64)
    ya = np.ascontiguousarray(y, dtype=np.float64)
    r = gao_residual()
    _check(lib().prog_gemm_residual(p.handle, int(loop), xa.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                    ya.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(r)),
           "prog_gemm_residual")
    return _residual_dict(r)


def gao_gemm_residual_scratch(M: int, N: int, K: int) -> int:
    b = ctypes.c_uint64(0)
    _check(lib().gao_gemm_residual_scratch(int(M), int(N), int(K), ctypes.byref(b)), "gao_gemm_residual_scratch")
    return int(b.value)


def gao_gemm_residual(A: int, B: int, C0: int, C: int, M: int, N: int, K: int, alpha: float, beta: float, x: int,
                      y: int, scratch: int, scratch_bytes: int, r_out: int = 0, s_out: int = 0, stream=None) -> Dict:
    """The same check on caller-owned device memory (integer device addresses, 0 for NULL)."""
    r = gao_residual()
    vp = lambda a: ctypes.c_void_p(int(a) or None)
    _check(lib().gao_gemm_residual(vp(A), vp(B), vp(C0), vp(C), int(M), int(N), int(K), float(alpha), float(beta),
                                   vp(x), vp(y), vp(scratch), ctypes.c_uint64(int(scratch_bytes)), vp(r_out),
                                   vp(s_out), ctypes.byref(r), _stream_handle(stream)), "gao_gemm_residual")
    return _residual_dict(r)


def prog_stats(p: Prog) -> List[Dict]:
    arr = (gao_loop_stat * p.n_loops)()
    _check(lib().prog_stats(p.handle, arr, p.n_loops), "prog_stats")
    return [{k: getattr(s, k) for k, _ in gao_loop_stat._fields_} for s in arr]


def prog_cache_clear(p: Prog) -> None:
    _check(lib().prog_cache_clear(p.handle), "prog_cache_clear")


def prog_destroy(p: Prog) -> None:
    if p.handle is not None and p.handle.value:
        if getattr(p, "owned", True):
            lib().prog_destroy(p.handle)
        p.handle = ctypes.c_void_p(None)


def _handles(progs: Sequence[Prog]):
    arr = (ctypes.c_void_p * len(progs))()
    for i, p in enumerate(progs):
        arr[i] = p.handle.value
    return arr


def ga_evaluate(progs: Sequence[Prog], population: Sequence[int]):
    """Returns (fitness[pop], seconds[pop], cache_hits)."""
    pop = len(population)
    pa = (ctypes.c_uint64 * pop)(*[int(m) for m in population])
    fit = (ctypes.c_double * pop)()
    sec = (ctypes.c_double * pop)()
    hits = ctypes.c_int(0)
    _check(lib().ga_evaluate(_handles(progs), len(progs), pa, pop, fit, sec, ctypes.byref(hits)), "ga_evaluate")
    return np.array(fit[:]), np.array(sec[:]), int(hits.value)


@dataclass
class GAResult:
    best_mask: int
    best_s: float
    evaluations: int
    cache_hits: int
    history: List[dict]
    populations: List[List[int]]


def _params(pop, generations, pc, pm, seed, elite=1, mutation=0, timeout_s=0.0):
    p = gao_ga_params()
    p.pop, p.generations, p.pc, p.pm = int(pop), int(generations), float(pc), float(pm)
    p.elite, p.mutation, p.seed, p.timeout_s = int(elite), int(mutation), int(seed), float(timeout_s)
    return p


def _result(params):
    hist = (gao_ga_gen * params.generations)()
    pops = (ctypes.c_uint64 * (params.generations * params.pop))()
    r = gao_ga_result()
    r.history = ctypes.cast(hist, ctypes.POINTER(gao_ga_gen))
    r.populations = ctypes.cast(pops, ctypes.POINTER(ctypes.c_uint64))
    return r, hist, pops


def _unpack(r, hist, pops, params) -> GAResult:
    h = [{k: getattr(g, k) for k, _ in gao_ga_gen._fields_} for g in hist]
    P = [list(pops[g * params.pop:(g + 1) * params.pop]) for g in range(params.generations)]
    return GAResult(int(r.best_mask), float(r.best_s), int(r.evaluations), int(r.cache_hits), h, P)


def ga_run(progs: Sequence[Prog], pop=12, generations=12, pc=0.9, pm=0.05, seed=0, elite=1, mutation=0,
           timeout_s=0.0) -> GAResult:
    params = _params(pop, generations, pc, pm, seed, elite, mutation, timeout_s)
    r, hist, pops = _result(params)
    _check(lib().ga_run(_handles(progs), len(progs), ctypes.byref(params), ctypes.byref(r)), "ga_run")
    return _unpack(r, hist, pops, params)


def ga_run_table(times: np.ndarray, n_genes: int, pop=12, generations=12, pc=0.9, pm=0.05, seed=0, elite=1,
                 mutation=0) -> GAResult:
    t = np.ascontiguousarray(times, dtype=np.float64)
    assert t.size >= (1 << n_genes)
    params = _params(pop, generations, pc, pm, seed, elite, mutation, 0.0)
    r, hist, pops = _result(params)
    _check(lib().ga_run_table(t.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n_genes, ctypes.byref(params),
                              ctypes.byref(r)), "ga_run_table")
    return _unpack(r, hist, pops, params)


def gao_selftest_device_wait(limit_s: float = 0.2, stream=None) -> int:
    """Returns the status (GAO_ETIMEOUT is the expected outcome)."""
    return int(lib().gao_selftest_device_wait(float(limit_s), _stream_handle(stream)))


COLMAX_NOALLOC_MAX_COLS = 65536


def gao_colmax_noalloc(dev_in: int, rows: int, cols: int, dev_out: int, stream=None) -> int:
    """Column maxima of a device matrix into caller device memory, with no allocation;
    returns the status (see include/gao.h for the shared-scratch rules)."""
    return int(lib().gao_colmax_noalloc(ctypes.c_void_p(dev_in), int(rows), int(cols), ctypes.c_void_p(dev_out),
                                        _stream_handle(stream)))


class Batch:
    """Handle of a gao_batch (owning); keeps its programs alive."""

    def __init__(self, handle, progs):
        self.handle = handle
        self.progs = list(progs)

    def __del__(self):
        try:
            batch_destroy(self)
        except Exception:
            pass


def batch_create(progs: Sequence[Prog], replicas: int = 1) -> Batch:
    """A batch over the suite `progs`; replicas > 1 measures a generation's new genes that
    many at a time, their GEMMs in one grouped launch (batch_set_replicas)."""
    h = ctypes.c_void_p(None)
    _check(lib().batch_create(_handles(progs), len(progs), ctypes.byref(h)), "batch_create")
    b = Batch(h, progs)
    if replicas != 1:
        batch_set_replicas(b, replicas)
    return b


def batch_set_replicas(b: Batch, replicas: int) -> None:
    _check(lib().batch_set_replicas(b.handle, int(replicas)), "batch_set_replicas")


def batch_replica_prog(b: Batch, replica: int, index: int) -> Prog:
    """Program `index` of copy `replica` of the suite (a borrowed handle: valid while the
    copy exists; never destroyed through this object)."""
    h = ctypes.c_void_p(None)
    _check(lib().batch_replica_prog(b.handle, int(replica), int(index), ctypes.byref(h)), "batch_replica_prog")
    src = b.progs[index]
    q = Prog(h, src.buffers, src.loops)
    q.owned = False
    return q


def batch_evaluate(b: Batch, population: Sequence[int]):
    """Returns (fitness[pop], seconds[pop], cache_hits)."""
    pop = len(population)
    pa = (ctypes.c_uint64 * pop)(*[int(m) for m in population])
    fit = (ctypes.c_double * pop)()
    sec = (ctypes.c_double * pop)()
    hits = ctypes.c_int(0)
    _check(lib().batch_evaluate(b.handle, pa, pop, fit, sec, ctypes.byref(hits)), "batch_evaluate")
    return np.array(fit[:]), np.array(sec[:]), int(hits.value)


def batch_ga_run(b: Batch, pop=12, generations=12, pc=0.9, pm=0.05, seed=0, elite=1, mutation=0,
                 timeout_s=0.0) -> GAResult:
    params = _params(pop, generations, pc, pm, seed, elite, mutation, timeout_s)
    r, hist, pops = _result(params)
    _check(lib().batch_ga_run(b.handle, ctypes.byref(params), ctypes.byref(r)), "batch_ga_run")
    return _unpack(r, hist, pops, params)


def batch_stats(b: Batch) -> Dict:
    st = gao_batch_stat()
    _check(lib().batch_stats(b.handle, ctypes.byref(st)), "batch_stats")
    return {k: getattr(st, k) for k, _ in gao_batch_stat._fields_ if k != "_pad"}


def batch_destroy(b: Batch) -> None:
    if b.handle is not None and b.handle.value:
        lib().batch_destroy(b.handle)
        b.handle = ctypes.c_void_p(None)


def _autotune_out(r) -> Dict:
    return {k: getattr(r, k) for k, _ in gao_autotune_result._fields_ if k != "_pad"}


def prog_autotune(p: Prog, pop=8, generations=6, pc=0.9, pm=0.05, seed=0) -> Dict:
    """GA over the GEMM's tile configuration (5-bit gene); applies and returns the best."""
    params = _params(pop, generations, pc, pm, seed)
    r = gao_autotune_result()
    _check(lib().prog_autotune(p.handle, ctypes.byref(params), ctypes.byref(r)), "prog_autotune")
    return _autotune_out(r)


def batch_autotune(b: Batch, pop=8, generations=6, pc=0.9, pm=0.05, seed=0) -> Dict:
    params = _params(pop, generations, pc, pm, seed)
    r = gao_autotune_result()
    _check(lib().batch_autotune(b.handle, ctypes.byref(params), ctypes.byref(r)), "batch_autotune")
    return _autotune_out(r)


GENE_EVAL_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.POINTER(ctypes.c_uint64), ctypes.c_int,
                                ctypes.POINTER(ctypes.c_double), ctypes.c_void_p)


def ga_run_callback(evaluate, n_genes: int, pop=12, generations=12, pc=0.9, pm=0.05, seed=0, elite=1,
                    mutation=0) -> GAResult:
    """Simple GA whose new genes of each generation are measured by ``evaluate(genes) ->
    seconds`` (lists).  An exception inside ``evaluate`` stops the GA (GaoError)."""
    errors = []

    def cb(genes_p, n, out_p, ctx):
        try:
            secs = evaluate([int(genes_p[i]) for i in range(n)])
            if len(secs) != n:
                raise ValueError("evaluate returned the wrong number of times")
            for i in range(n):
                out_p[i] = float(secs[i])
            return GAO_OK
        except BaseException as e:  # noqa: BLE001 - reported to the caller below
            errors.append(e)
            return GAO_ECPU

    c_cb = GENE_EVAL_FN(cb)
    params = _params(pop, generations, pc, pm, seed, elite, mutation, 0.0)
    r, hist, pops = _result(params)
    st = lib().ga_run_callback(n_genes, ctypes.byref(params), ctypes.cast(c_cb, ctypes.c_void_p), None,
                               ctypes.byref(r))
    if st != GAO_OK:
        err = GaoError(st, "ga_run_callback")
        if errors:
            raise err from errors[0]
        raise err
    return _unpack(r, hist, pops, params)
