"""INIT outputs that only a split-precision GEMM reads are formed straight into the GEMM's
bfloat16 operand planes (the binary32 arrays are never written, the GEMM's split kernels
do not run).

Checked on the GPU against the same program with A and B made OUTPUT buffers (which keeps
them as binary32 and takes the INIT -> split -> MMA path): C must carry the same bits in
every precision and tile shape, with row-scaled A, and with ragged shapes; the launches show
which path ran; the FP64 residual check (which needs A and B as binary32) forms them on
demand and agrees with the reference program's; programs where A has a second reader or the
GEMM runs on the CPU keep the plain path.
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

PREC = {"bf16": 1, "bf16x3": 2, "bf16x6": 3}


@pytest.fixture(scope="module")
def gao():
    from paper_1806_01430_gb300 import _build
    _build.build()
    import paper_1806_01430_gb300 as g
    return g


def gemm_prog(M, N, K, seed, keep_ab=False, rowscale=False):
    role = W.OUTPUT if keep_ab else W.TEMP
    bufs = [W.Buffer("A", M, K, W.F32, role), W.Buffer("B", K, N, W.F32, role), W.Buffer("C0", M, N, W.F32, W.TEMP),
            W.Buffer("C", M, N, W.F32, W.OUTPUT)]
    loops = [W.Loop(W.INIT, [], [0, 1, 2], flags=1 if rowscale else 0), W.Loop(W.GEMM, [0, 1, 2], [3], 1.5, 0.5)]
    return W.Program(f"gemm_{M}x{N}x{K}", bufs, loops, seed)


def run(gao, prog, prec, mask=0b11, **kw):
    p = gao.prog_from_workload(prog, gemm_prec=PREC[prec], **kw)
    gao.prog_run(p, mask)
    C = gao.prog_output(p, prog.index("C")).copy()
    st = gao.prog_stats(p)
    return p, C, st


@pytest.mark.parametrize("prec,kchunk,cfg", [("bf16x6", 0, 0), ("bf16x6", 256, 0), ("bf16x6", 0, 8), ("bf16x3", 0, 0),
                                            ("bf16", 0, 0), ("bf16", 0, 1), ("bf16", 0, 2)])
@pytest.mark.parametrize("shape", [(300, 520, 1000), (129, 200, 77), (513, 130, 261), (256, 256, 64), (1, 1, 1)])
def test_init_planes_match_split_path(gao, prec, kchunk, cfg, shape):
    M, N, K = shape
    seed = 9000 + M + N + K
    p, C, st = run(gao, gemm_prog(M, N, K, seed), prec, kchunk=kchunk, tile_cfg=cfg)
    q, C_ref, st_ref = run(gao, gemm_prog(M, N, K, seed, keep_ab=True), prec, kchunk=kchunk, tile_cfg=cfg)
    assert np.array_equal(C.view(np.uint32), C_ref.view(np.uint32))
    # INIT: C0 as binary32, A and B as planes (3 launches); GEMM: the MMA alone
    assert st[0]["launches"] == 3 and st[1]["launches"] == 1
    assert st_ref[0]["launches"] == 1 and st_ref[1]["launches"] == 3
    assert [gao.prog_planes_for(p, b) for b in range(4)] == [1, 1, -1, -1]
    assert [gao.prog_planes_for(q, b) for b in range(4)] == [-1, -1, -1, -1]
    # a second run (graph replay) gives the same bits
    gao.prog_run(p, 0b11)
    assert np.array_equal(gao.prog_output(p, 3).view(np.uint32), C_ref.view(np.uint32))
    gao.prog_destroy(p)
    gao.prog_destroy(q)


@pytest.mark.parametrize("prec", ["bf16x6", "bf16x3"])
def test_init_planes_row_scaled(gao, prec):
    """Rows of A times 2^e (e from the row's hash): the planes take the same exponents."""
    M, N, K = 700, 300, 900
    p, C, st = run(gao, gemm_prog(M, N, K, 77, rowscale=True), prec)
    q, C_ref, _ = run(gao, gemm_prog(M, N, K, 77, keep_ab=True, rowscale=True), prec)
    assert np.array_equal(C.view(np.uint32), C_ref.view(np.uint32))
    assert st[0]["launches"] == 4  # row exponents, C0, A's planes, B's planes
    gao.prog_destroy(p)
    gao.prog_destroy(q)


def test_init_planes_residual_forms_operands_on_demand(gao):
    """The FP64 residual check reads A and B as binary32: after a run that formed them only as
    planes it forms them from the INIT loop first, and agrees with the reference program."""
    n = 1024
    p, C, st = run(gao, gemm_prog(n, n, n, 5), "bf16x6")
    q, C_ref, _ = run(gao, gemm_prog(n, n, n, 5, keep_ab=True), "bf16x6")
    assert st[1]["launches"] == 1
    rng = np.random.default_rng(3)
    x, y = rng.choice([-1.0, 1.0], n), rng.choice([-1.0, 1.0], n)
    assert gao.prog_planes_for(p, 0) == 1
    r = gao.prog_gemm_residual(p, 1, x, y)
    assert gao.prog_planes_for(p, 0) == -1  # formed as binary32 for the check
    r_ref = gao.prog_gemm_residual(q, 1, x, y)
    assert r["right"] == r_ref["right"] and r["left"] == r_ref["left"]
    assert max(r["right"], r["left"]) <= 1e-6
    # the next run forms the planes again (the operands formed on demand are dropped)
    gao.prog_run(p, 0b11)
    assert gao.prog_stats(p)[1]["launches"] == 1
    assert np.array_equal(gao.prog_output(p, 3).view(np.uint32), C_ref.view(np.uint32))
    gao.prog_destroy(p)
    gao.prog_destroy(q)


def test_init_planes_only_where_the_gemm_is_the_sole_reader(gao):
    """Six-loop program without fusion: A is also read by the scale-add, so it stays binary32
    (split by the GEMM); B is read by the GEMM alone and goes straight into its planes.  With
    the GEMM on the CPU nothing is deferred.  Results match the oracle."""
    n = 384
    prog = W.six_loop(n, 4321, outputs=("C", "D", "E", "r", "f"))
    ref = oracle.run_program(prog)
    for mask, fuse, init_l, gemm_l in ((0b111111, False, 2, 2), (0b111101, False, 1, None), (0b111111, True, 1, None)):
        p = gao.prog_from_workload(prog, gemm_prec=PREC["bf16x6"], fuse_chains=gao.FUSE_ON if fuse else gao.FUSE_OFF)
        gao.prog_run(p, mask)
        st = gao.prog_stats(p)
        assert st[0]["launches"] == init_l, (mask, fuse, st[0])
        if gemm_l is not None:
            assert st[1]["launches"] == gemm_l  # A's split and the MMA
        for nm in ("C", "D", "E", "r"):
            assert oracle.rel_err(gao.prog_output(p, prog.index(nm)), ref[nm]) <= 1e-6, (mask, nm)
        gao.prog_destroy(p)
