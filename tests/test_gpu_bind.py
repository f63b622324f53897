"""Caller host memory bound as a program's host copy (prog_bind_host) through the C ABI.

A run copies a bound INPUT straight from the caller's array and a bound OUTPUT straight
back into the caller's array.  The results must carry the same bits as the same program
fed through prog_set_input; rewriting the bound input between runs (also when the all-GPU
gene replays a captured graph) must show in the next run's output; pageable numpy memory
(registered by the library) and pinned torch memory both work; unbinding returns the
buffer to the library's mirror, after which an INPUT needs prog_set_input again.
"""
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


def _inputs(n, seed):
    return {nm: oracle.init_matrix(seed, b, n, n).astype(np.float32) for b, nm in enumerate(("A", "B", "C0"))}


@pytest.mark.parametrize("prec", ["bf16x6", "fp32_simt"])
def test_bound_inputs_and_output_match_set_input(gao, prec):
    n, seed = 1000, 61
    pr = {"bf16x6": gao.BF16X6, "fp32_simt": gao.FP32_SIMT}[prec]
    hp = W.host_input_gemm(n)
    ins = _inputs(n, seed)
    ref = gao.prog_from_workload(hp, gemm_prec=pr)
    for nm, v in ins.items():
        gao.prog_set_input(ref, hp.index(nm), v)
    gao.prog_run(ref, 1)
    C_ref = gao.prog_output(ref, hp.index("C"))
    gao.prog_destroy(ref)

    p = gao.prog_from_workload(hp, gemm_prec=pr)
    bound = {nm: v.copy() for nm, v in ins.items()}  # pageable numpy: the library registers it
    C_out = np.zeros((n, n), dtype=np.float32)
    for nm, v in bound.items():
        gao.prog_bind_host(p, hp.index(nm), v)
    gao.prog_bind_host(p, hp.index("C"), C_out)
    for run in range(4):  # plain runs, then the captured graph's replays
        C_out[:] = 0.0
        gao.prog_run(p, 1)
        assert np.array_equal(C_out.view(np.uint32), C_ref.view(np.uint32)), run
        assert np.array_equal(gao.prog_output(p, hp.index("C")), C_ref)
    assert gao.prog_graphs(p)[0] >= 1
    st = gao.prog_stats(p)
    assert sum(s["h2d_bytes"] for s in st) == 3 * n * n * 4
    assert sum(s["d2h_bytes"] for s in st) == n * n * 4
    # new data in the caller's array: the next run (a graph replay) reads it
    bound["C0"][:] = np.float32(0.0)
    gao.prog_run(p, 1)
    A, B = ins["A"].astype(np.float64), ins["B"].astype(np.float64)
    rng = np.random.default_rng(0)
    ii, jj = rng.integers(0, n, 64), rng.integers(0, n, 64)
    want = np.array([1.5 * (A[i] @ B[:, j]) for i, j in zip(ii, jj)])
    got = C_out[ii, jj].astype(np.float64)
    assert np.sqrt(((got - want) ** 2).mean() / (want ** 2).mean()) <= 1e-6
    # unbinding an INPUT: it needs prog_set_input again
    gao.prog_bind_host(p, hp.index("C0"), None)
    with pytest.raises(gao.GaoError):
        gao.prog_run(p, 1)
    gao.prog_set_input(p, hp.index("C0"), ins["C0"])
    gao.prog_run(p, 1)
    assert np.array_equal(C_out.view(np.uint32), C_ref.view(np.uint32))
    gao.prog_destroy(p)


def test_bound_pinned_torch_tensors(gao):
    torch = pytest.importorskip("torch")
    n, seed = 777, 62
    hp = W.host_input_gemm(n)
    ins = _inputs(n, seed)
    ref = oracle.run_program(hp, {k: v.astype(np.float64) for k, v in ins.items()})["C"]
    p = gao.prog_from_workload(hp, gemm_prec=gao.BF16X6)
    tens = {}
    for nm, v in ins.items():
        tens[nm] = torch.from_numpy(v).pin_memory()
        gao.prog_bind_host(p, hp.index(nm), tens[nm])
    tens["C"] = torch.zeros((n, n), dtype=torch.float32).pin_memory()
    gao.prog_bind_host(p, hp.index("C"), tens["C"])
    gao.prog_run(p, 1)
    assert oracle.rel_err(tens["C"].numpy(), ref) <= 1e-6
    gao.prog_destroy(p)


def test_bind_rejects_wrong_size(gao):
    hp = W.host_input_gemm(64)
    p = gao.prog_from_workload(hp)
    with pytest.raises(gao.GaoError):
        gao.prog_bind_host(p, 0, np.zeros((64, 63), dtype=np.float32))
    with pytest.raises(gao.GaoError):
        gao.prog_bind_host(p, 9, np.zeros((64, 64), dtype=np.float32))
    gao.prog_destroy(p)


@pytest.mark.parametrize("prec,n", [("bf16x6", 2304), ("bf16x3", 2500), ("bf16x6", 4096), ("bf16", 4352)])
def test_overlapped_gemm_copies_c_back_by_row_block(gao, prec, n):
    """A GEMM whose A comes from the host runs in row blocks overlapped with the copy in; with C
    an OUTPUT bound to the caller's array, each block's rows of C go back as soon as the block is
    done (the link's other direction).  C must carry the bits of the device-resident run, be
    copied back exactly once per run (plain runs and graph replays), and a run that keeps the
    device buffers must not copy it."""
    pr = {"bf16x6": gao.BF16X6, "bf16x3": gao.BF16X3, "bf16": gao.BF16}[prec]
    seed = 71
    hp = W.host_input_gemm(n)
    ins = _inputs(n, seed)
    # the same GEMM on operands formed on the device by the INIT loop (same hash streams):
    # one launch, no row blocks
    dev = W.gemm_only(n, seed)
    ref = gao.prog_from_workload(dev, gemm_prec=pr)
    gao.prog_run(ref, 0b11)
    assert sum(s["h2d_bytes"] for s in gao.prog_stats(ref)) == 0
    C_ref = gao.prog_output(ref, dev.index("C")).copy()
    gao.prog_destroy(ref)

    p = gao.prog_from_workload(hp, gemm_prec=pr)
    C_out = np.zeros((n, n), dtype=np.float32)
    for nm, v in ins.items():
        gao.prog_bind_host(p, hp.index(nm), v.copy())
    gao.prog_bind_host(p, hp.index("C"), C_out)
    for run in range(4):
        C_out[:] = np.float32(-1.0)
        gao.prog_run(p, 1)
        assert np.array_equal(C_out.view(np.uint32), C_ref.view(np.uint32)), run
        st = gao.prog_stats(p)
        assert sum(s["h2d_bytes"] for s in st) == 3 * n * n * 4
        assert sum(s["d2h_bytes"] for s in st) == n * n * 4, run
    C_out[:] = np.float32(-1.0)
    gao.prog_run(p, 1, gao.RUN_KEEP_DEVICE)
    assert sum(s["d2h_bytes"] for s in gao.prog_stats(p)) == 0
    assert np.all(C_out == np.float32(-1.0))
    gao.prog_destroy(p)


@pytest.mark.parametrize("prec,m,k,n", [("bf16x6", 4100, 1100, 1800), ("bf16", 4352, 1024, 2700),
                                         ("bf16x3", 5000, 900, 513)])
def test_overlapped_rectangular_gemm_bit_identical(gao, prec, m, k, n):
    """A rectangular GEMM whose operands come from the host (A's rows in blocks, the first
    block's columns of C in two ranges, beta C0 after each block): the bits of the same GEMM
    on operands the INIT loop formed on the device, one launch."""
    pr = {"bf16x6": gao.BF16X6, "bf16x3": gao.BF16X3, "bf16": gao.BF16}[prec]
    seed = 73
    shapes = {"A": (m, k), "B": (k, n), "C0": (m, n), "C": (m, n)}
    dev = W.Program("rect_dev", [W.Buffer(nm, *shapes[nm], W.F32, W.OUTPUT if nm == "C" else W.TEMP)
                                 for nm in ("A", "B", "C0", "C")],
                    [W.Loop(W.INIT, [], [0, 1, 2]), W.Loop(W.GEMM, [0, 1, 2], [3], alpha=1.5, beta=0.5)], seed)
    host = W.Program("rect_host", [W.Buffer(nm, *shapes[nm], W.F32, W.OUTPUT if nm == "C" else W.INPUT)
                                   for nm in ("A", "B", "C0", "C")],
                     [W.Loop(W.GEMM, [0, 1, 2], [3], alpha=1.5, beta=0.5)], seed)
    p = gao.prog_from_workload(dev, gemm_prec=pr)
    gao.prog_run(p, 0b11)
    C_ref = gao.prog_output(p, 3).copy()
    gao.prog_destroy(p)
    q = gao.prog_from_workload(host, gemm_prec=pr)
    for b, nm in enumerate(("A", "B", "C0")):
        gao.prog_set_input(q, b, oracle.init_matrix(seed, b, *shapes[nm]).astype(np.float32))
    for _ in range(2):  # a plain run, then the captured graph
        gao.prog_run(q, 0b1)
        assert np.array_equal(gao.prog_output(q, 3).view(np.uint32), C_ref.view(np.uint32))
    assert gao.prog_stats(q)[0]["launches"] > 3  # row blocks (and column ranges) ran
    gao.prog_destroy(q)
