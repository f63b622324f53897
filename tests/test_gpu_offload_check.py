"""The parallelisability check of Sec. 4 at prog_create, through the C ABI on the GPU.

Loops with a loop-carried dependence (RECURRENCE), an early exit (FIND) or a call of a
host routine (GAO_LOOP_EXTERNAL_CALL) are excluded from the gene: they run on the CPU
under every gene, and gene bit k places the k-th offloadable loop.

Tolerances: the recurrence runs in binary32 with one fused multiply-add per step, so
|y_j - y_ref| <= gamma_{2(j+1)} * sum_k |alpha|^(j-k) |x_k| with u = 2^-24; FIND is a
decision on binary32 data and must match exactly on the same data; the FP32 GEMM and
what follows it are held to the 1e-6 normwise bound of the other program tests.
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def gao():
    from paper_1806_01430_gb300 import _build
    _build.build()
    import paper_1806_01430_gb300 as g
    return g


def rec_bound(X, alpha):
    X = np.abs(np.asarray(X, dtype=np.float64))
    scale = np.zeros_like(X)
    for j in range(X.shape[1]):
        scale[:, j] = X[:, j] if j == 0 else abs(alpha) * scale[:, j - 1] + X[:, j]
    g = 2 * (np.arange(X.shape[1]) + 1) * U32
    return g / (1 - g) * scale + 1e-300


def test_classification_and_gene_length(gao):
    prog = W.analysis_program(40, 24, 3)
    p = gao.prog_from_workload(prog)
    assert gao.prog_gene_length(p) == 4
    got = [gao.prog_loop_offload(p, i) for i in range(prog.n_loops)]
    assert got == [(gao.OFFLOAD_OK, 0), (gao.OFFLOAD_DEPENDENCE, -1), (gao.OFFLOAD_OK, 1), (gao.OFFLOAD_OK, 2),
                   (gao.OFFLOAD_EARLY_EXIT, -1), (gao.OFFLOAD_EXTERNAL_CALL, -1), (gao.OFFLOAD_OK, 3)]
    with pytest.raises(gao.GaoError):
        gao.prog_run(p, 1 << 4)  # bit at the gene length
    with pytest.raises(gao.GaoError):
        gao.prog_loop_offload(p, prog.n_loops)
    gao.prog_destroy(p)


def test_every_gene_matches_oracle_and_places_only_offloadable_loops(gao):
    m, n = 96, 80
    prog = W.analysis_program(m, n, 17, outputs=("R", "C", "T", "k", "s"))
    ref = oracle.run_program(prog)
    p = gao.prog_from_workload(prog)
    gene_loops = [0, 2, 3, 6]
    X = oracle.init_matrix(17, 0, m, n)
    for gene in range(16):
        gao.prog_run(p, gene)
        st = gao.prog_stats(p)
        for li in range(prog.n_loops):
            want = 1 if li in gene_loops and (gene >> gene_loops.index(li)) & 1 else 0
            assert st[li]["placement"] == want, (gene, li)
        R = gao.prog_output(p, prog.index("R")).astype(np.float64)
        assert np.all(np.abs(R - ref["R"]) <= rec_bound(X, W.ANALYSIS_ALPHA))
        C = gao.prog_output(p, prog.index("C"))
        assert oracle.rel_err(C, ref["C"]) <= 1e-6
        T = gao.prog_output(p, prog.index("T"))
        assert np.array_equal(T, C.T)
        k = gao.prog_output(p, prog.index("k")).ravel()
        thr = np.float32(W.ANALYSIS_THRESHOLD)
        want_k = [next((j for j in range(m) if T[i, j] > thr), m) for i in range(n)]
        assert np.array_equal(k, np.array(want_k, dtype=np.float64)), gene
        s = float(gao.prog_output(p, prog.index("s"))[0, 0])
        s_own = float(np.maximum(T.astype(np.float64), 0).sum())
        assert abs(s - s_own) <= 2e-7 * s_own
        assert abs(s - ref["s"]) <= 1e-6 * ref["s"]
    gao.prog_destroy(p)


@pytest.mark.parametrize("shape", [(1, 1), (5, 1), (3, 1000), (64, 4097), (0, 7), (7, 0)])
@pytest.mark.parametrize("alpha", [1.0, 0.5, -0.75])
def test_recurrence_loop(gao, shape, alpha):
    rows, cols = shape
    X = oracle.init_matrix(8, 0, rows, cols).astype(np.float32)
    bufs = [W.Buffer("X", rows, cols, W.F32, W.INPUT), W.Buffer("Y", rows, cols, W.F32, W.OUTPUT)]
    prog = W.Program("rec", bufs, [W.Loop(W.RECURRENCE, [0], [1], alpha=alpha)], 1)
    p = gao.prog_from_workload(prog)
    assert gao.prog_gene_length(p) == 0
    gao.prog_set_input(p, 0, X)
    gao.prog_run(p, 0)
    Y = gao.prog_output(p, 1).astype(np.float64)
    assert np.all(np.abs(Y - oracle.recurrence(X, alpha)) <= rec_bound(X, alpha))
    with pytest.raises(gao.GaoError):
        gao.ga_run([p], pop=4, generations=2)  # nothing to search
    gao.prog_destroy(p)


@pytest.mark.parametrize("shape", [(1, 1), (9, 33), (200, 1500), (3, 0)])
def test_find_loop_exact(gao, shape):
    rows, cols = shape
    X = oracle.init_matrix(9, 0, rows, cols).astype(np.float32)
    if rows and cols:
        X[0, :] = np.float32(0.1)  # equal to the binary32 threshold: never "greater"
    bufs = [W.Buffer("X", rows, cols, W.F32, W.INPUT), W.Buffer("k", rows, 1, W.F64, W.OUTPUT)]
    for t in (0.1, 0.5, 0.999, 2.0, -2.0):
        prog = W.Program("find", bufs, [W.Loop(W.FIND, [0], [1], alpha=t)], 1)
        p = gao.prog_from_workload(prog)
        gao.prog_set_input(p, 0, X)
        gao.prog_run(p, 0)
        k = gao.prog_output(p, 1)
        gao.prog_destroy(p)
        assert np.array_equal(k, oracle.find_first(X, t)), t


def test_ga_and_batch_over_offloadable_loops(gao):
    progs = [W.analysis_program(m, n, 30 + i) for i, (m, n) in enumerate([(64, 48), (128, 96), (200, 136)])]
    handles = [gao.prog_from_workload(pr) for pr in progs]
    r = gao.ga_run(handles, pop=6, generations=4, seed=5)
    assert 0 <= r.best_mask < 16 and r.evaluations <= 16
    fit, secs, hits = gao.ga_evaluate(handles, list(range(16)))
    assert np.all(np.asarray(secs) > 0)
    b = gao.batch_create(handles)
    fb, sb, hb = gao.batch_evaluate(b, list(range(16)))
    assert np.all(np.asarray(sb) > 0)
    rb = gao.batch_ga_run(b, pop=6, generations=4, seed=5)
    assert 0 <= rb.best_mask < 16
    with pytest.raises(gao.GaoError):
        gao.batch_evaluate(b, [16])
    # every program's outputs after the batch's last gene match a plain run of that gene
    gene = 0b1011
    gao.batch_evaluate(b, [gene])  # cached: runs nothing new
    gao.batch_destroy(b)
    for pr, h in zip(progs, handles):
        gao.prog_run(h, gene)
        ref = oracle.run_program(pr)
        assert abs(float(gao.prog_output(h, pr.index("s"))[0, 0]) - ref["s"]) <= 1e-6 * ref["s"]
        gao.prog_destroy(h)
