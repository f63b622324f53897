"""Host-side checks of the C ABI (no GPU needed): the library builds and loads, every
entry point declared in include/gao.h is exported, struct layouts agree between the
header and the binding, argument validation rejects malformed programs, the
library fails loudly without a CUDA device or without its own shared library, and the C++ Simple GA
reproduces the oracle GA's trajectory draw for draw."""
import ctypes
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from oracle import ga as oga
import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gao.h")


@pytest.fixture(scope="module")
def gao():
    from paper_1806_01430_gb300 import _build
    _build.build()
    import paper_1806_01430_gb300 as g
    g.lib()
    return g


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:gao_status|void|const char\s*\*)\s*\**\s*(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(gao):
    names = _declared_functions()
    assert len(names) >= 14, names
    L = gao.lib()
    for n in names:
        assert hasattr(L, n), f"{n} declared in gao.h but not exported"
    assert set(names) == set(gao.SIGNATURES), "binding and header disagree on the entry points"
    out = subprocess.run(["nm", "-D", "--defined-only", gao.LIB_PATH], capture_output=True, text=True).stdout
    for n in names:
        assert re.search(rf"\bT {n}\b", out), n


def test_struct_layouts_match_header(gao, tmp_path):
    structs = ["gao_buffer", "gao_loop", "gao_opts", "gao_loop_stat", "gao_ga_params", "gao_ga_gen", "gao_ga_result",
               "gao_batch_stat", "gao_residual"]
    src = tmp_path / "sz.c"
    src.write_text('#include "gao.h"\n#include <stdio.h>\n#include <stddef.h>\nint main(void){\n' +
                   "".join(f'printf("%zu\\n", sizeof({s}));\n' for s in structs) +
                   'printf("%zu %zu %zu\\n", offsetof(gao_loop, alpha), offsetof(gao_opts, stream), '
                   'offsetof(gao_ga_result, history));\nreturn 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    lines = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    for s, l in zip(structs, lines):
        assert ctypes.sizeof(getattr(gao, s)) == int(l), s
    offs = [int(x) for x in lines[len(structs)].split()]
    assert offs == [gao.gao_loop.alpha.offset, gao.gao_opts.stream.offset, gao.gao_ga_result.history.offset]


def test_version_and_last_error(gao):
    assert "sm_103a" in gao.gao_version()
    assert isinstance(gao.gao_last_error(), str)


def _bad(gao, buffers, loops):
    with pytest.raises(gao.GaoError) as ei:
        gao.prog_create(buffers, loops)
    return ei.value


def test_validation_rejects_malformed_programs(gao):
    B, L = W.Buffer, W.Loop
    # shape mismatch in the GEMM
    e = _bad(gao, [B("A", 4, 5), B("B", 6, 4), B("C", 4, 4)],
             [L(W.INIT, [], [0, 1, 2]), L(W.GEMM, [0, 1, 2], [2], 1.0, 1.0)])
    assert e.status == gao.GAO_EINVAL and "inner dimensions" in str(e)
    # read before write
    e = _bad(gao, [B("X", 4, 4), B("Y", 4, 4)], [L(W.TRANSPOSE, [0], [1])])
    assert e.status == gao.GAO_EINVAL and "before any loop writes" in str(e)
    # wrong output shape of a transpose
    e = _bad(gao, [B("X", 4, 6), B("Y", 4, 6)], [L(W.INIT, [], [0]), L(W.TRANSPOSE, [0], [1])])
    assert e.status == gao.GAO_EINVAL
    # Frobenius must write a 1 x 1 binary64 scalar
    e = _bad(gao, [B("X", 4, 4), B("f", 1, 1, W.F32)], [L(W.INIT, [], [0]), L(W.FROBENIUS, [0], [1])])
    assert e.status == gao.GAO_EINVAL
    # too many loops for a 64-bit gene
    e = _bad(gao, [B("X", 2, 2)], [L(W.INIT, [], [0])] * 65)
    assert e.status == gao.GAO_EINVAL
    # unknown loop kind
    e = _bad(gao, [B("X", 2, 2)], [L(W.INIT, [], [0]), L(42, [0], [0])])
    assert e.status == gao.GAO_EINVAL
    # the loops kept on the CPU are validated like the others
    e = _bad(gao, [B("X", 3, 5), B("k", 3, 1, W.F32)], [L(W.INIT, [], [0]), L(W.FIND, [0], [1], 0.5)])
    assert e.status == gao.GAO_EINVAL and "expected 3x1" in str(e)
    e = _bad(gao, [B("X", 3, 5)], [L(W.INIT, [], [0]), L(W.RECURRENCE, [0], [0], 0.5)])
    assert e.status == gao.GAO_EINVAL and "in place" in str(e)
    e = _bad(gao, [B("X", 4, 4), B("Y", 4, 4)],
             [L(W.INIT, [], [0]), L(W.STENCIL3, [0], [1], flags=W.EXTERNAL_CALL | 5)])
    assert e.status == gao.GAO_EINVAL and "preset" in str(e)


@pytest.mark.skipif(os.path.exists("/dev/nvidia0"), reason="a GPU is present")
def test_valid_program_needs_the_gpu(gao):
    prog = W.six_loop(8, 1)
    with pytest.raises(gao.GaoError) as ei:
        gao.prog_from_workload(prog)
    assert ei.value.status in (gao.GAO_ENODEV, gao.GAO_ECUDA)


def test_missing_library_fails_loudly(gao, monkeypatch, tmp_path):
    """Without libgao.so the first call raises and names the missing file: the binding has no
    other implementation to fall back on."""
    monkeypatch.setattr(gao, "LIB_PATH", str(tmp_path / "libgao.so"))
    monkeypatch.setattr(gao, "_lib", None)
    with pytest.raises(RuntimeError) as ei:
        gao.prog_from_workload(W.six_loop(8, 1))
    assert "libgao.so is missing" in str(ei.value) and "no fallback" in str(ei.value)
    with pytest.raises(RuntimeError):
        gao.lib()


def _table_fn(t):
    return lambda m: float(t[m])


@pytest.mark.parametrize("case", [
    dict(n=6, pop=12, gens=12, pc=0.9, pm=0.05, seed=1, table="loop", mutation=0),
    dict(n=12, pop=12, gens=12, pc=0.9, pm=0.05, seed=7, table="rand", mutation=0),
    dict(n=12, pop=20, gens=20, pc=0.9, pm=0.05, seed=3, table="fail", mutation=0),
    dict(n=9, pop=7, gens=15, pc=0.6, pm=0.2, seed=11, table="rand", mutation=1),
    dict(n=1, pop=3, gens=4, pc=0.9, pm=0.5, seed=5, table="rand", mutation=0),
    dict(n=16, pop=13, gens=9, pc=1.0, pm=0.01, seed=99, table="rand", mutation=0),
])
def test_c_ga_matches_oracle_ga(gao, case):
    n = case["n"]
    if case["table"] == "loop":
        t = W.loop_time_table(n, seed=case["seed"])
    elif case["table"] == "fail":
        t = W.random_time_table(n, seed=case["seed"], fail_frac=0.3)
    else:
        t = W.random_time_table(n, seed=case["seed"])
    ref = oga.run(_table_fn(t), n, case["pop"], case["gens"], case["pc"], case["pm"], case["seed"],
                  mutation=case["mutation"])
    got = gao.ga_run_table(t, n, pop=case["pop"], generations=case["gens"], pc=case["pc"], pm=case["pm"],
                           seed=case["seed"], mutation=case["mutation"])
    assert got.populations == ref.populations
    assert got.best_mask == ref.best_mask and got.best_s == ref.best_s
    assert got.evaluations == ref.evaluations and got.cache_hits == ref.cache_hits
    for h, r in zip(got.history, ref.history):
        assert h["best_mask"] == r.best_mask and h["best_s"] == r.best_s
        assert h["evaluated"] == r.evaluated and h["cache_hits"] == r.cache_hits
        assert (h["mean_s"] == r.mean_s) or (np.isinf(h["mean_s"]) and np.isinf(r.mean_s))
        assert 0.0 <= h["wall_s"] < 60.0


def test_c_ga_rejects_bad_params(gao):
    t = np.ones(8)
    for kw in (dict(pop=0), dict(generations=0), dict(pc=1.5), dict(pm=-0.1)):
        with pytest.raises(gao.GaoError):
            gao.ga_run_table(t, 3, **kw)
