"""Row sums in their fixed order (blocks of 32 elements, a quadruple tree per block, four
interleaved block accumulators): the GPU kernel and the host loop give exactly the bits of a
float32 emulation of that order, on ragged row lengths (vector and scalar paths), and stay
within the oracle's tolerance."""
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


def rowsum_fixed_order(X):
    """The order restated with float32 numpy operations (every + rounds to binary32)."""
    X = np.asarray(X, dtype=np.float32)
    rows, L = X.shape
    nblk = (L + 31) // 32
    pad = np.zeros((rows, max(nblk, 1) * 32), dtype=np.float32)
    pad[:, :L] = X
    x = pad.reshape(rows, -1, 8, 4)
    q = (x[..., 0] + x[..., 1]) + (x[..., 2] + x[..., 3])
    s = ((q[..., 0] + q[..., 4]) + (q[..., 2] + q[..., 6])) + ((q[..., 1] + q[..., 5]) + (q[..., 3] + q[..., 7]))
    u = np.zeros((rows, 4), dtype=np.float32)
    for p in range(nblk):
        u[:, p % 4] += s[:, p]
    return ((u[:, 0] + u[:, 2]) + (u[:, 1] + u[:, 3])).reshape(rows, 1)


def rowsum_program(rows, cols, seed):
    B_, L_ = W.Buffer, W.Loop
    bufs = [B_("X", rows, cols, role=W.OUTPUT), B_("r", rows, 1, role=W.OUTPUT)]
    loops = [L_(W.INIT, [], [0]), L_(W.ROWSUM, [0], [1])]
    return W.Program(f"rowsum_{rows}x{cols}", bufs, loops, seed)


@pytest.mark.parametrize("rows,cols", [(5, 1), (7, 3), (9, 31), (4, 33), (6, 100), (3, 127), (5, 129),
                                       (40, 1000), (33, 1001), (130, 4096), (17, 5000)])
def test_rowsum_bits_match_the_fixed_order(gao, rows, cols):
    prog = rowsum_program(rows, cols, 500 + cols)
    ref = oracle.run_program(prog)
    p = gao.prog_from_workload(prog)
    got = {}
    for gene in (0b11, 0b01):  # row sums on the GPU, then on the host
        gao.prog_run(p, gene)
        X = gao.prog_output(p, 0)
        got[gene] = gao.prog_output(p, 1).copy()
        want = rowsum_fixed_order(X)
        assert np.array_equal(got[gene], want), gene
    assert oracle.rel_err(got[0b11], ref["r"]) <= 1e-6
    gao.prog_destroy(p)


def test_rowsum_signed_zeros_and_cancellation(gao):
    """Given rows (an INPUT buffer): all -0 (the +0 starts of the accumulators give +0),
    exact cancellation of huge terms, and a ragged length with +0 padding -- GPU and host
    give the emulation's bits, signs of zero included."""
    X = np.zeros((4, 70), dtype=np.float32)
    X[0, :] = -0.0
    X[1, :35] = 1.5
    X[1, 35:] = -1.5
    X[2, ::2] = 3.0e38
    X[2, 1::2] = -3.0e38
    X[3, :] = np.arange(70, dtype=np.float32) * np.float32(1e-3)
    bufs = [W.Buffer("X", 4, 70, role=W.INPUT), W.Buffer("r", 4, 1, role=W.OUTPUT)]
    q = gao.prog_create(bufs, [W.Loop(W.ROWSUM, [0], [1])])
    gao.prog_set_input(q, 0, X)
    want = rowsum_fixed_order(X)
    for gene in (1, 0):
        gao.prog_run(q, gene)
        r = gao.prog_output(q, 1)
        assert np.array_equal(r.view(np.uint32), want.view(np.uint32)), gene
    gao.prog_destroy(q)
