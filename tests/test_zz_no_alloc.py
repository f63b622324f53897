"""Allocation-free column maxima (gao_colmax_noalloc) through the C ABI.

For callers that cannot allocate device memory when they need the result (a host
framework whose pool owns the GPU's memory, or a latency-critical loop that cannot
afford cudaMalloc/cudaFree): the entry point keeps its scratch in a fixed array
inside the library.  This test compares it with the existing COLMAX loop of a
program (prog_run), bit for bit since a maximum is exact, on two calls in a row
whose second input has smaller maxima than the first -- stale keys left by the
first call would show up as wrong maxima in the second.  Collected last so that a
run stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gao():
    from paper_1806_01430_gb300 import _build
    _build.build()
    import paper_1806_01430_gb300 as g
    return g


def colmax_via_program(gao, X):
    rows, cols = X.shape
    bufs = [W.Buffer("P", rows, cols, role=W.INPUT), W.Buffer("q", 1, cols, role=W.OUTPUT)]
    p = gao.prog_create(bufs, [W.Loop(W.COLMAX, [0], [1])])
    gao.prog_set_input(p, 0, X)
    gao.prog_run(p, 1)
    q = gao.prog_output(p, 1).ravel()
    gao.prog_destroy(p)
    return q


def test_colmax_noalloc_matches_program_twice(gao):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(17)
    rows, cols = 1000, 4099  # ragged: not a multiple of 4
    X1 = rng.standard_normal((rows, cols)).astype(np.float32)
    X2 = (X1 - 100.0).astype(np.float32)  # every maximum below the first call's
    s = torch.cuda.Stream()
    out = torch.empty(cols, dtype=torch.float32, device="cuda")
    for X in (X1, X2):
        d_in = torch.from_numpy(X).cuda()
        torch.cuda.synchronize()
        st = gao.gao_colmax_noalloc(d_in.data_ptr(), rows, cols, out.data_ptr(), s)
        assert st == gao.GAO_OK, gao.gao_last_error()
        s.synchronize()
        got = out.cpu().numpy()
        ref = colmax_via_program(gao, X)
        assert np.array_equal(got, ref)
        assert np.array_equal(got, X.max(axis=0))


def test_colmax_noalloc_limits(gao):
    torch = pytest.importorskip("torch")
    big = gao.COLMAX_NOALLOC_MAX_COLS + 1
    d = torch.zeros(big, dtype=torch.float32, device="cuda")
    assert gao.gao_colmax_noalloc(d.data_ptr(), 1, big, d.data_ptr()) == gao.GAO_EINVAL
    assert "65536" in gao.gao_last_error()
    # the maximum itself is accepted
    n = gao.COLMAX_NOALLOC_MAX_COLS
    x = torch.arange(2 * n, dtype=torch.float32, device="cuda").reshape(2, n)
    o = torch.empty(n, dtype=torch.float32, device="cuda")
    assert gao.gao_colmax_noalloc(x.data_ptr(), 2, n, o.data_ptr()) == gao.GAO_OK
    torch.cuda.synchronize()
    assert torch.equal(o, x[1])
