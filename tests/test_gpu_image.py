"""GPU parity of the 3x3 stencil loop and of the edge-detection image program
(the paper's motivating camera-analysis workload, Sec. 1) against the FP64 oracle.

Tolerances:
  * a stencil output is nine binary32 fused multiply-adds of exact products, so
    |y - y_ref| <= 9 * 2^-24 * sum |w| |x| (componentwise, gamma_9 bound);
  * the CPU loop (gene bit 0) and the GPU kernel add the terms in the same order
    with fused multiply-adds: bit-identical, for every loop of the program but the
    SUM, whose GPU form adds groups of four binary32 values before its binary64
    accumulation (at most 3 roundings of 2^-24 per group on non-negative data:
    2e-7 relative) -- in its own pass, or inside the fused gradient chain's pass
    (another partition of the same groups, so the two agree within the same bound);
  * squared gradient magnitude: |M2 - M2_ref| <= 64 * 2^-24 * (Gx^2 + Gy^2), with
    Gx, Gy the Sobel responses of the blur computed with |w| and |x| (the first-order
    propagation of the per-stage gamma_9 bounds through the square, with slack).
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
SUM_REL = 2e-7
KERNELS = {
    0: np.array([[1, 2, 1], [2, 4, 2], [1, 2, 1]], dtype=np.float64) / 16,
    1: np.array([[0, 1, 0], [1, -4, 1], [0, 1, 0]], dtype=np.float64),
    2: np.array([[-1, 0, 1], [-2, 0, 2], [-1, 0, 1]], dtype=np.float64),
    3: np.array([[-1, -2, -1], [0, 0, 0], [1, 2, 1]], dtype=np.float64),
}


@pytest.fixture(scope="module")
def gao():
    from paper_1806_01430_gb300 import _build
    _build.build()
    import paper_1806_01430_gb300 as g
    return g


def abs_stencil(X, preset):
    """sum |w_ab| |x_{i+a,j+b}| with zero padding (the scale of the rounding bound)."""
    Xp = np.pad(np.abs(np.asarray(X, dtype=np.float64)), 1)
    r, c = X.shape
    out = np.zeros((r, c))
    K = np.abs(KERNELS[preset])
    for a in range(3):
        for b in range(3):
            out += K[a, b] * Xp[a:a + r, b:b + c]
    return out


def one_stencil(rows, cols, preset):
    bufs = [W.Buffer("X", rows, cols, W.F32, W.INPUT), W.Buffer("Y", rows, cols, W.F32, W.OUTPUT)]
    return W.Program(f"stencil_{rows}x{cols}", bufs, [W.Loop(W.STENCIL3, [0], [1], flags=preset)], 5)


@pytest.mark.parametrize("shape", [(1, 1), (1, 7), (5, 1), (2, 2), (3, 4), (17, 513), (129, 260), (300, 1001),
                                   (64, 2048), (41, 2052)])
def test_stencil_loop_parity(gao, shape):
    rows, cols = shape
    X = oracle.init_matrix(31, 0, rows, cols, rowscale=True).astype(np.float32)
    for preset in range(4):
        prog = one_stencil(rows, cols, preset)
        ref = oracle.stencil3(X, preset)
        bound = 9 * U32 * abs_stencil(X, preset) + 1e-300
        p = gao.prog_from_workload(prog)
        gao.prog_set_input(p, 0, X)
        gao.prog_run(p, 0b1)
        Yg = gao.prog_output(p, 1)
        gao.prog_run(p, 0b0)
        Yc = gao.prog_output(p, 1)
        gao.prog_destroy(p)
        assert np.all(np.abs(Yg.astype(np.float64) - ref) <= bound), f"preset {preset}"
        assert np.array_equal(Yg.view(np.uint32), Yc.view(np.uint32)), f"preset {preset}: CPU and GPU bits differ"


def test_stencil_invalid_preset_and_in_place(gao):
    bufs = [W.Buffer("X", 8, 8, W.F32, W.INPUT), W.Buffer("Y", 8, 8, W.F32, W.OUTPUT)]
    with pytest.raises(gao.GaoError):
        gao.prog_from_workload(W.Program("bad", bufs, [W.Loop(W.STENCIL3, [0], [1], flags=4)], 1))
    bufs = [W.Buffer("X", 8, 8, W.F32, W.OUTPUT)]
    with pytest.raises(gao.GaoError):
        gao.prog_from_workload(W.Program("bad", bufs, [W.Loop(W.INIT, [], [0]), W.Loop(W.STENCIL3, [0], [0])], 1))


def m2_bound(X):
    """64 u (Gx^2 + Gy^2) with Gx, Gy the absolute-value Sobel responses of the absolute blur."""
    Babs = abs_stencil(X, 0)
    return 64 * U32 * (abs_stencil(Babs, 2) ** 2 + abs_stencil(Babs, 3) ** 2) + 1e-300


@pytest.mark.parametrize("hw", [(1, 1), (3, 5), (64, 64), (127, 257), (256, 383)])
def test_image_program_all_gpu(gao, hw):
    h, w = hw
    prog = W.image_program(h, w, W.SEED_IMAGE, outputs=("B", "gx", "M2", "e", "q"))
    ref = oracle.run_program(prog)
    p = gao.prog_from_workload(prog)
    gao.prog_run(p, (1 << prog.n_loops) - 1)
    out = {nm: gao.prog_output(p, prog.index(nm)) for nm in ("B", "gx", "M2", "e", "q")}
    gao.prog_destroy(p)
    X = oracle.init_matrix(W.SEED_IMAGE, 0, h, w)
    assert np.all(np.abs(out["B"] - ref["B"]) <= 9 * U32 * abs_stencil(X, 0) + 1e-300)
    M2 = out["M2"].astype(np.float64)
    assert np.all(np.abs(M2 - ref["M2"]) <= m2_bound(X))
    # reductions over the run's own M2: SUM in binary64, COLMAX exact
    e = float(out["e"][0, 0])
    assert abs(e - M2.sum()) <= SUM_REL * M2.sum() + 1e-300
    assert np.array_equal(out["q"].ravel(), out["M2"].max(axis=0))
    assert abs(e - ref["e"]) <= float(m2_bound(X).sum()) + SUM_REL * abs(ref["e"])


def test_image_genes_bit_identical(gao):
    h, w = 200, 300
    prog = W.image_program(h, w, W.SEED_IMAGE + 1, outputs=("M2", "e", "q"))
    p = gao.prog_from_workload(prog)
    rng = np.random.default_rng(3)
    masks = [0, (1 << prog.n_loops) - 1] + [int(m) for m in rng.integers(0, 1 << prog.n_loops, 14)]
    first = None
    for m in masks:
        gao.prog_run(p, m)
        got = (gao.prog_output(p, prog.index("M2")), float(gao.prog_output(p, prog.index("e"))[0, 0]),
               gao.prog_output(p, prog.index("q")))
        if first is None:
            first = got
            continue
        assert np.array_equal(got[0].view(np.uint32), first[0].view(np.uint32)), f"gene {m:09b}"
        assert np.array_equal(got[2].view(np.uint32), first[2].view(np.uint32)), f"gene {m:09b}"
        assert abs(got[1] - first[1]) <= SUM_REL * abs(first[1])
    gao.prog_destroy(p)


def test_host_image_program(gao):
    h, w = 96, 130
    prog = W.image_program(h, w, 44, outputs=("M2", "q"), host_image=True)
    X = oracle.init_matrix(44, 0, h, w).astype(np.float32)
    ref = oracle.run_program(prog, {"X": X})
    p = gao.prog_from_workload(prog)
    gao.prog_set_input(p, prog.index("X"), X)
    for mask in ((1 << prog.n_loops) - 1, 0, 0b10110101):
        gao.prog_run(p, mask)
        M2 = gao.prog_output(p, prog.index("M2")).astype(np.float64)
        assert np.all(np.abs(M2 - ref["M2"]) <= m2_bound(X))
        if mask & 1:
            assert gao.prog_stats(p)[0]["h2d_bytes"] == h * w * 4
    gao.prog_destroy(p)


def sample_m2(seed, h, w, i, j):
    """M2[i, j] of the full-size program from the 5 x 5 neighbourhood of X (oracle values)."""
    P = np.zeros((5, 5))
    for a in range(5):
        for b in range(5):
            y, x = i + a - 2, j + b - 2
            if 0 <= y < h and 0 <= x < w:
                P[a, b] = oracle.init_value(seed, 0, y * w + x)
    Bp = oracle.stencil3(P, 0)[1:4, 1:4]  # blur at rows i-1..i+1, cols j-1..j+1 (exact neighbourhood)
    for a in range(3):
        for b in range(3):
            if not (0 <= i + a - 1 < h and 0 <= j + b - 1 < w):
                Bp[a, b] = 0.0  # the blurred image is zero-padded too
    gx = float((KERNELS[2] * Bp).sum())
    gy = float((KERNELS[3] * Bp).sum())
    return gx * gx + gy * gy, P


def test_full_size_8192(gao):
    """The bench's frame, 8192 x 8192, every loop on the GPU: M2 on sampled pixels from their
    5 x 5 neighbourhoods (corners and edges included), then on every pixel against the oracle's
    binary64 program; the energy within its bound; the column maxima exact on the run's M2."""
    h = w = 8192
    prog = W.image_program(h, w, W.SEED_IMAGE, outputs=("M2", "e", "q"))
    p = gao.prog_from_workload(prog)
    gao.prog_run(p, (1 << prog.n_loops) - 1)
    M2 = gao.prog_output(p, prog.index("M2"))
    e = float(gao.prog_output(p, prog.index("e"))[0, 0])
    q = gao.prog_output(p, prog.index("q"))
    gao.prog_destroy(p)
    rng = np.random.default_rng(8)
    pts = [(0, 0), (h - 1, w - 1), (0, w - 1), (h - 1, 0), (1, 4095), (4096, 1)]
    pts += [(int(a), int(b)) for a, b in zip(rng.integers(0, h, 40), rng.integers(0, w, 40))]
    for i, j in pts:
        want, P = sample_m2(W.SEED_IMAGE, h, w, i, j)
        bnd = m2_bound(P)[2, 2]
        assert abs(float(M2[i, j]) - want) <= bnd, (i, j)
    M2d = M2.astype(np.float64)
    assert abs(e - M2d.sum()) <= SUM_REL * M2d.sum()
    assert np.array_equal(q.ravel(), M2.max(axis=0))
    # every pixel against the oracle's binary64 program, within the propagated gamma_9 bound
    ref = oracle.run_program(prog)
    X = oracle.init_matrix(W.SEED_IMAGE, 0, h, w)
    bound = m2_bound(X)
    del X
    assert np.all(np.abs(M2d - ref["M2"]) <= bound)
    assert abs(e - ref["e"]) <= float(bound.sum()) + SUM_REL * abs(ref["e"])


@pytest.mark.parametrize("outputs", [("M2", "e", "q"), ("gx", "sy", "M2", "e", "q"), ("e", "q"), ("B", "e", "q")])
@pytest.mark.parametrize("hw", [(64, 64), (127, 257), (300, 1001), (5, 481)])
def test_fused_gradient_chain_bit_identical(gao, hw, outputs):
    """The blur, Sobel x, Sobel y, the two squares and their sum in one pass over the raw
    image, with the edge energy (SUM) and the column maxima (COLMAX) of M2 formed in the same
    pass: the same bits as the eight separate loops (the edge energy within its rounding
    bound: the pass partitions the sum differently); the blurred image and the dead
    intermediates are not written (M2 too, when only the reductions read it) unless they are
    outputs.  Widths around a warp's 120 output columns and a block's 480 included."""
    h, w = hw
    prog = W.image_program(h, w, W.SEED_IMAGE + 3, outputs=outputs)
    res = {}
    for fuse in (gao.FUSE_OFF, gao.FUSE_ON):
        p = gao.prog_from_workload(prog, fuse_chains=fuse)
        gao.prog_run(p, (1 << prog.n_loops) - 1)
        res[fuse] = ({nm: gao.prog_output(p, prog.index(nm)) for nm in outputs}, gao.prog_stats(p))
        gao.prog_destroy(p)
    (a, _), (b, st) = res[gao.FUSE_OFF], res[gao.FUSE_ON]
    for nm in outputs:
        if nm == "e":
            ea, eb = float(a[nm][0, 0]), float(b[nm][0, 0])
            assert abs(ea - eb) <= 2 * SUM_REL * abs(ea), (ea, eb)
        else:
            assert np.array_equal(np.asarray(a[nm]).view(np.uint32), np.asarray(b[nm]).view(np.uint32)), nm
    assert [s["placement"] for s in st] == [1, 1, 2, 2, 2, 2, 2, 2, 2]
    assert st[1]["launches"] == 3  # the pass, the sum of its block partials, the column maxima's decode


@pytest.mark.parametrize("hw", [(1, 1), (2, 3), (3, 7), (9, 240), (17, 241), (33, 8), (4, 964)])
def test_fused_pass_degenerate_shapes(gao, hw):
    """The one-pass blur and gradient chain on frames of one to a few rows or columns and on
    widths around a warp's 240 output columns (a lane's eight columns straddling the right
    edge): the same bits as the separate loops for M2 and the column maxima, the edge energy
    within its rounding bound."""
    h, w = hw
    prog = W.image_program(h, w, W.SEED_IMAGE + 5, outputs=("M2", "e", "q"))
    res = {}
    for fuse in (gao.FUSE_OFF, gao.FUSE_ON):
        p = gao.prog_from_workload(prog, fuse_chains=fuse)
        gao.prog_run(p, (1 << prog.n_loops) - 1)
        res[fuse] = ({nm: gao.prog_output(p, prog.index(nm)) for nm in ("M2", "e", "q")}, gao.prog_stats(p))
        gao.prog_destroy(p)
    (a, _), (b, st) = res[gao.FUSE_OFF], res[gao.FUSE_ON]
    assert np.array_equal(a["M2"].view(np.uint32), b["M2"].view(np.uint32))
    assert np.array_equal(a["q"].view(np.uint32), b["q"].view(np.uint32))
    ea, eb = float(a["e"][0, 0]), float(b["e"][0, 0])
    assert abs(ea - eb) <= 2 * SUM_REL * abs(ea) + 1e-30, (ea, eb)
    assert st[1]["placement"] == 1 and all(s["placement"] == 2 for s in st[2:])


@pytest.mark.parametrize("hw", [(0, 64), (64, 0), (0, 0)])
def test_empty_frames(gao, hw):
    """Frames with no rows or no columns, separate loops and one fused pass: nothing is
    launched over the empty image, the edge energy is 0 and each column maximum of no rows is
    -inf, as in the oracle."""
    h, w = hw
    prog = W.image_program(h, w, W.SEED_IMAGE, outputs=("M2", "e", "q"))
    ref = oracle.run_program(prog)
    for fuse in (gao.FUSE_OFF, gao.FUSE_ON):
        p = gao.prog_from_workload(prog, fuse_chains=fuse)
        gao.prog_run(p, (1 << prog.n_loops) - 1)
        assert gao.prog_output(p, prog.index("M2")).shape == (h, w)
        assert float(gao.prog_output(p, prog.index("e"))[0, 0]) == 0.0 == float(ref["e"])
        q = gao.prog_output(p, prog.index("q"))
        assert q.shape == (1, w) and np.all(q == -np.inf) and np.all(np.asarray(ref["q"]) == -np.inf)
        gao.prog_destroy(p)


@pytest.mark.parametrize("h,w", [(64, 250), (2048, 2048)])
def test_fused_pass_special_values(gao, h, w):
    """A frame holding NaNs of either sign (quiet, signalling, with payloads), infinities,
    -0 and values whose squares overflow: the one-pass blur and gradient chain gives M2's and
    the column maxima's bits of the separate loops (the column maxima rank every value the
    same way whether taken in the pass or by the COLMAX loop), and an edge energy that is NaN
    exactly when theirs is.  The larger frame comes in row strips from the host."""
    seed = 61
    prog = W.image_program(h, w, seed, outputs=("M2", "e", "q"), host_image=True)
    X = oracle.init_matrix(seed, 0, h, w).astype(np.float32)
    bits = X.view(np.uint32)
    rng = np.random.default_rng(h + w)
    specials = np.array([0x7FC00000, 0xFFC00000, 0x7F800001, 0xFF800001, 0x7FFFFFFF, 0xFFFFFFFF,
                         0x7F800000, 0xFF800000, 0x80000000, 0x7149F2CA, 0xF149F2CA], dtype=np.uint32)
    for v in specials:  # a few of each, at random places (some columns clean)
        rr = rng.integers(0, h, 3)
        cc = rng.integers(0, w // 2, 3)
        bits[rr, cc] = v
    outs = {}
    for fuse in (gao.FUSE_OFF, gao.FUSE_ON):
        p = gao.prog_from_workload(prog, fuse_chains=fuse)
        gao.prog_set_input(p, prog.index("X"), X)
        gao.prog_run(p, (1 << prog.n_loops) - 1)
        outs[fuse] = {nm: gao.prog_output(p, prog.index(nm)).copy() for nm in ("M2", "e", "q")}
        gao.prog_destroy(p)
    a, b = outs[gao.FUSE_OFF], outs[gao.FUSE_ON]
    assert np.array_equal(a["M2"].view(np.uint32), b["M2"].view(np.uint32))
    assert np.array_equal(a["q"].view(np.uint32), b["q"].view(np.uint32))
    assert np.isnan(a["q"]).any()  # the special values reached the maxima
    ea, eb = float(a["e"][0, 0]), float(b["e"][0, 0])
    assert np.isnan(ea) == np.isnan(eb) and (np.isnan(ea) or ea == eb or abs(ea - eb) <= 2 * SUM_REL * abs(ea))


@pytest.mark.parametrize("hw", [(64, 64), (300, 1001)])
def test_gradient_chain_alone_when_blur_on_cpu(gao, hw):
    """With the blur on the CPU the gradient chain and its reductions still run as one pass,
    over the blurred image copied in: the same bits as the separate loops."""
    h, w = hw
    prog = W.image_program(h, w, W.SEED_IMAGE + 4, outputs=("M2", "e", "q"))
    gene = ((1 << prog.n_loops) - 1) & ~0b10
    res = {}
    for fuse in (gao.FUSE_OFF, gao.FUSE_ON):
        p = gao.prog_from_workload(prog, fuse_chains=fuse)
        gao.prog_run(p, gene)
        res[fuse] = ({nm: gao.prog_output(p, prog.index(nm)) for nm in ("M2", "e", "q")}, gao.prog_stats(p))
        gao.prog_destroy(p)
    (a, _), (b, st) = res[gao.FUSE_OFF], res[gao.FUSE_ON]
    assert np.array_equal(a["M2"].view(np.uint32), b["M2"].view(np.uint32))
    assert np.array_equal(a["q"].view(np.uint32), b["q"].view(np.uint32))
    assert abs(float(a["e"][0, 0]) - float(b["e"][0, 0])) <= 2 * SUM_REL * abs(float(a["e"][0, 0]))
    assert [s["placement"] for s in st] == [1, 0, 1, 2, 2, 2, 2, 2, 2]
    assert st[2]["launches"] == 3


def test_gradient_chain_only_when_all_on_gpu(gao):
    prog = W.image_program(96, 130, 45, outputs=("M2",))
    ref = oracle.run_program(prog)
    X = oracle.init_matrix(45, 0, 96, 130)
    p = gao.prog_from_workload(prog, fuse_chains=gao.FUSE_GENE)
    assert gao.prog_gene_length(p) == 10
    for gene, fused in ((0b1111111111, True), (0b1111111101, True), (0b0111111111, False), (0b1111101111, False),
                        (0b1000000000, False)):
        gao.prog_run(p, gene)
        st = gao.prog_stats(p)
        assert (st[3]["placement"] == 2) == fused, bin(gene)
        M2 = gao.prog_output(p, prog.index("M2")).astype(np.float64)
        assert np.all(np.abs(M2 - ref["M2"]) <= m2_bound(X))
    gao.prog_destroy(p)


@pytest.mark.parametrize("h,w", [(2048, 2048), (2051, 2049)])
@pytest.mark.parametrize("fuse,outputs", [(0, ("M2", "e", "q")), (1, ("M2", "e", "q")), (1, ("e", "q"))])
def test_host_frame_strips_bit_identical(gao, h, w, fuse, outputs):
    """A frame of 16 MiB or more from the host is copied in row strips, and the blur -- fused,
    in one pass with the gradient chain on its output and the edge energy and the column
    maxima of M2 -- runs on each strip's ready rows while the next strips are on the link.  M2 and the
    column maxima equal those of the same frame made on the device (one launch per pass) bit
    for bit, and so does the edge energy unfused; fused, the strips partition its sum
    differently from one launch (within the rounding bound), and the same in every run."""
    seed = 45
    hp = W.image_program(h, w, seed, outputs=outputs, host_image=True)
    dp = W.image_program(h, w, seed, outputs=outputs)
    X = oracle.init_matrix(seed, 0, h, w).astype(np.float32)
    p = gao.prog_from_workload(hp, fuse_chains=fuse)
    gao.prog_set_input(p, hp.index("X"), X)
    outs = []
    for _ in range(2):  # the second run of the all-GPU gene is captured as a graph
        gao.prog_run(p, (1 << hp.n_loops) - 1)
        outs.append({nm: gao.prog_output(p, hp.index(nm)).copy() for nm in outputs})
    st = gao.prog_stats(p)
    gao.prog_destroy(p)
    q = gao.prog_from_workload(dp, fuse_chains=fuse)
    gao.prog_run(q, (1 << dp.n_loops) - 1)
    want = {nm: gao.prog_output(q, dp.index(nm)) for nm in outputs}
    gao.prog_destroy(q)
    for o in outs:
        for nm in outputs:
            if nm == "e" and fuse:
                assert abs(float(o["e"][0, 0]) - float(want["e"][0, 0])) <= 2 * SUM_REL * abs(float(want["e"][0, 0]))
            else:
                assert np.array_equal(o[nm], want[nm]), nm
    assert np.array_equal(outs[0]["e"].view(np.uint64), outs[1]["e"].view(np.uint64))
    assert st[0]["h2d_bytes"] == h * w * 4
    # a stencil launch per strip (fused: the blur and the chain in one), then, fused, the
    # partials' sum and the keys' decode
    assert st[0]["launches"] == (6 if fuse else 4)
    assert [s["placement"] for s in st[1:8]] == ([2] * 7 if fuse else [1] * 7)
