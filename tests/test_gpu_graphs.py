"""CUDA-graph replay of all-GPU genes: the second run of such a gene is captured, later
runs replay it.  Outputs must carry the same bits as plain launches, per-loop statistics
must still be measured, and new host inputs must flow through a replayed graph."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gao():
    from paper_1806_01430_gb300 import _build
    _build.build()
    import paper_1806_01430_gb300 as g
    return g


def outs(gao, p, prog):
    return {b.name: gao.prog_output(p, i).copy() for i, b in enumerate(prog.buffers) if b.role == W.OUTPUT}


@pytest.mark.parametrize("prec,fuse", [(3, 0), (3, 1), (0, 0), (2, 2)])
def test_replay_is_bit_identical_and_timed(gao, prec, fuse):
    prog = W.six_loop(320, 44, outputs=("C", "D", "E", "r", "f"))
    p = gao.prog_from_workload(prog, gemm_prec=prec, fuse_chains=fuse)
    gene = (1 << gao.prog_gene_length(p)) - 1
    plain = None
    for it in range(5):
        gao.prog_run(p, gene, gao.RUN_NO_GRAPH if it == 0 else 0)
        o = outs(gao, p, prog)
        st = gao.prog_stats(p)
        if plain is None:
            plain = o
            continue
        for nm in plain:
            assert np.array_equal(o[nm], plain[nm]), (it, nm)
        assert all(s["device_ms"] > 0 or s["placement"] == 2 for s in st), st
        assert st[1]["kernel_ms"] > 0 and st[1]["launches"] >= 1
    assert gao.prog_graphs(p) == (1, 0)  # captured on the second run, replayed since
    gao.prog_destroy(p)


def test_replay_with_new_host_inputs_and_overlap(gao):
    n, seed = 2048, 5
    hp = W.host_input_program(n, seed, outputs=("C", "r", "f"))
    p = gao.prog_from_workload(hp, gemm_prec=3)
    ins = {nm: oracle.init_matrix(seed, b, n, n).astype(np.float32) for nm, b in (("A", 0), ("B", 1), ("C0", 2))}
    for nm, v in ins.items():
        gao.prog_set_input(p, hp.index(nm), v)
    gene = (1 << hp.n_loops) - 1
    for _ in range(3):  # plain, capture, replay
        gao.prog_run(p, gene)
    assert gao.prog_graphs(p) == (1, 0)  # the copy-overlapped GEMM joins back into the capture
    C1 = gao.prog_output(p, hp.index("C")).copy()
    gao.prog_run(p, gene, gao.RUN_NO_GRAPH)
    assert np.array_equal(gao.prog_output(p, hp.index("C")), C1)
    assert gao.prog_stats(p)[0]["h2d_bytes"] == 3 * n * n * 4
    # new data through the replayed graph (same pinned mirrors, new contents)
    ins2 = {nm: (2.0 * v).astype(np.float32) for nm, v in ins.items()}
    for nm, v in ins2.items():
        gao.prog_set_input(p, hp.index(nm), v)
    gao.prog_run(p, gene)
    C2 = gao.prog_output(p, hp.index("C"))
    gao.prog_run(p, gene, gao.RUN_NO_GRAPH)
    assert np.array_equal(gao.prog_output(p, hp.index("C")), C2)
    # C = 1.5 AB + 0.5 C0 with every input doubled: 4x the product term, 2x the C0 term
    ref = 1.5 * 4 * (ins["A"].astype(np.float64)[:64] @ ins["B"].astype(np.float64)) + 0.5 * 2 * ins["C0"][:64]
    assert oracle.rel_err(C2[:64], ref) <= 1e-6
    gao.prog_destroy(p)


def test_graph_dropped_after_autotune_and_cache_clear(gao):
    prog = W.six_loop(512, 9, outputs=("C", "r", "f"))
    p = gao.prog_from_workload(prog, gemm_prec=2)
    for _ in range(3):
        gao.prog_run(p, 0b111111)
    C0 = gao.prog_output(p, prog.index("C")).copy()
    r = gao.prog_autotune(p, pop=4, generations=2, seed=1)
    for _ in range(3):  # recaptured with the tuned configuration
        gao.prog_run(p, 0b111111)
    C1 = gao.prog_output(p, prog.index("C"))
    assert oracle.rel_err(C1, C0) <= 2e-5
    gao.prog_cache_clear(p)
    gao.prog_run(p, 0b111111)
    assert np.array_equal(gao.prog_output(p, prog.index("C")), C1)
    gao.prog_destroy(p)


def test_mixed_genes_never_captured(gao):
    prog = W.six_loop(256, 10, outputs=("C", "r", "f"))
    p = gao.prog_from_workload(prog, gemm_prec=3)
    ref = None
    for _ in range(4):
        gao.prog_run(p, 0b110111)  # loop 3 on the CPU: plain launches every time
        C = gao.prog_output(p, prog.index("C"))
        if ref is None:
            ref = C.copy()
        assert np.array_equal(C, ref)
        assert gao.prog_stats(p)[3]["placement"] == 0
    assert gao.prog_graphs(p) == (0, 0)
    gao.prog_destroy(p)


def test_runs_without_loop_times(gao):
    """GAO_RUN_NO_LOOP_TIMES records no per-loop events (a captured graph without event
    nodes, kept apart from the timed one): the same outputs, the run's own time, and no loop
    times in the statistics; a later timed run reports them again."""
    prog = W.six_loop(320, 46, outputs=("C", "D", "E", "r", "f"))
    p = gao.prog_from_workload(prog, gemm_prec=3, fuse_chains=1)
    gene = (1 << gao.prog_gene_length(p)) - 1
    gao.prog_run(p, gene)
    want = outs(gao, p, prog)
    for it in range(3):  # the second run is captured, the third replayed
        secs = gao.prog_run(p, gene, gao.RUN_NO_LOOP_TIMES)
        assert secs > 0
        o = outs(gao, p, prog)
        for nm in want:
            assert np.array_equal(o[nm], want[nm]), (it, nm)
        st = gao.prog_stats(p)
        assert all(s["device_ms"] == 0 and s["kernel_ms"] == 0 and s["copy_ms"] == 0 for s in st), st
        assert [s["placement"] for s in st] == [1, 1, 2, 2, 2, 2]
    assert gao.prog_graphs(p)[0] == 1
    for _ in range(3):
        gao.prog_run(p, gene)
    st = gao.prog_stats(p)
    assert st[1]["kernel_ms"] > 0 and st[0]["device_ms"] > 0
    assert gao.prog_graphs(p)[0] == 2  # the timed variant has its own graph
    gao.prog_destroy(p)
