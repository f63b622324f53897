"""Fused loop chain (GEMM -> scale-add -> transpose [-> row sums] [-> Frobenius] in one GEMM epilogue):
bit-identical C, D, E and row sums to the unfused run, the norm within the reduction's
rounding bound, the oracle's tolerance, and fusion only when the gene puts the whole
chain on the GPU."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

TOL = {1: 5e-3, 2: 2e-5, 3: 1e-6}


@pytest.fixture(scope="module")
def gao():
    from paper_1806_01430_gb300 import _build
    _build.build()
    import paper_1806_01430_gb300 as g
    return g


def outputs(gao, p, prog):
    out = {b.name: gao.prog_output(p, i) for i, b in enumerate(prog.buffers) if b.role == W.OUTPUT}
    for nm in ("f", "s"):
        if nm in out:
            out[nm] = float(out[nm][0, 0])
    return out


@pytest.mark.parametrize("prec", [3, 2, 1])
@pytest.mark.parametrize("n", [256, 129, 300, 1000])
def test_fused_six_loop_matches_unfused(gao, prec, n):
    prog = W.six_loop(n, 600 + n, outputs=("C", "D", "E", "r", "f"))
    ref = oracle.run_program(prog)
    res = {}
    for fuse in (False, True):
        p = gao.prog_from_workload(prog, gemm_prec=prec, fuse_chains=fuse)
        gao.prog_run(p, 0b111111)
        res[fuse] = (outputs(gao, p, prog), gao.prog_stats(p))
        gao.prog_destroy(p)
    (a, _), (b, st) = res[False], res[True]
    for nm in ("C", "D", "E", "r"):
        assert np.array_equal(a[nm], b[nm]), nm
    assert abs(a["f"] - b["f"]) <= 2e-7 * a["f"]
    assert [s["placement"] for s in st] == [1, 1, 2, 2, 2, 2]
    assert st[1]["launches"] == 5  # split A, split B, fused GEMM, norm partials, row-sum blocks
    for nm in ("C", "D", "E", "r"):
        assert oracle.rel_err(b[nm], ref[nm]) <= TOL[prec]
    assert abs(b["f"] - ref["f"]) <= TOL[prec] * ref["f"]


def test_fused_chain_only_when_all_on_gpu(gao):
    prog = W.six_loop(200, 71, outputs=("C", "E", "r", "f"))
    ref = oracle.run_program(prog)
    p = gao.prog_from_workload(prog, gemm_prec=3, fuse_chains=True)
    for mask, fused in ((0b111111, True), (0b111011, False), (0b110111, False), (0b011111, True),
                        (0b101111, True), (0b000111, False)):
        gao.prog_run(p, mask)
        st = gao.prog_stats(p)
        assert (st[2]["placement"] == 2) == fused, mask
        if fused:
            assert st[5]["placement"] == (2 if (mask >> 5) & 1 else 0)
            assert st[4]["placement"] == (2 if (mask >> 4) & 1 else 0)
        out = outputs(gao, p, prog)
        for nm in ("C", "E", "r"):
            assert oracle.rel_err(out[nm], ref[nm]) <= 1e-6
        assert abs(out["f"] - ref["f"]) <= 1e-6 * ref["f"]
    gao.prog_destroy(p)


def test_fused_twelve_loop(gao):
    prog = W.twelve_loop(200, 72, W.SEED_TWELVE_LOOP, outputs=("C", "D", "E", "r", "f", "P", "q", "s"))
    ref = oracle.run_program(prog)
    p = gao.prog_from_workload(prog, gemm_prec=3, fuse_chains=True)
    gao.prog_run(p, (1 << 12) - 1)
    st = gao.prog_stats(p)
    assert [s["placement"] for s in st[:6]] == [1, 1, 2, 2, 2, 2]
    out = outputs(gao, p, prog)
    for nm in ("C", "D", "E", "P", "r", "q"):
        assert oracle.rel_err(out[nm], ref[nm]) <= 1e-6, nm
    for nm in ("f", "s"):
        assert abs(out[nm] - ref[nm]) <= 1e-6 * abs(ref[nm])
    gao.prog_destroy(p)


def test_fused_full_size_n4096(gao):
    n, seed = 4096, W.SEED_N4096
    prog = W.six_loop(n, seed, outputs=("C", "D", "E", "r", "f"))
    res = {}
    for fuse in (False, True):
        p = gao.prog_from_workload(prog, gemm_prec=3, fuse_chains=fuse)
        gao.prog_run(p, 0b111111)
        res[fuse] = outputs(gao, p, prog)
        gao.prog_destroy(p)
    for nm in ("C", "D", "E", "r"):
        assert np.array_equal(res[False][nm], res[True][nm]), nm
    assert abs(res[False]["f"] - res[True]["f"]) <= 2e-7 * res[False]["f"]


def test_fusion_as_a_gene_bit(gao):
    """GAO_FUSE_GENE: one extra gene bit after the loop bits decides fusion; the GA searches
    placements and fusion together, and every gene gives the same C, E and row sums."""
    prog = W.six_loop(384, 73, outputs=("C", "E", "r", "f"))
    p = gao.prog_from_workload(prog, gemm_prec=3, fuse_chains=gao.FUSE_GENE)
    assert gao.prog_gene_length(p) == 7
    first = None
    for gene, fused in ((0b0111111, False), (0b1111111, True), (0b1111011, False), (0b1110111, False)):
        gao.prog_run(p, gene)
        st = gao.prog_stats(p)
        assert (st[2]["placement"] == 2) == fused, bin(gene)
        out = outputs(gao, p, prog)
        if first is None:
            first = out
        for nm in ("C", "E", "r"):
            assert np.array_equal(out[nm], first[nm]), (bin(gene), nm)
    gao.prog_run(p, 0b1000000)  # fusion bit alone: every loop on the CPU
    ref = oracle.run_program(prog)
    assert oracle.rel_err(outputs(gao, p, prog)["C"], ref["C"]) <= 1e-6
    with pytest.raises(gao.GaoError):
        gao.prog_run(p, 1 << 7)
    r = gao.ga_run([p], pop=8, generations=3, seed=2)
    assert 0 <= r.best_mask < (1 << 7)
    with pytest.raises(gao.GaoError):
        gao.batch_create([p])  # batches run loop by loop
    gao.prog_destroy(p)


@pytest.mark.parametrize("n,prec", [(2048, 3), (2500, 2), (2304, 1)])
def test_fused_chain_in_copy_overlapped_gemm(gao, n, prec):
    """Host inputs: the GEMM runs in row blocks overlapped with the copy, and with fusion
    each block's epilogue also writes its rows of D, its columns of E and its norm
    partials.  Same C, D, E, r as the unfused run; the norm within the reduction bound."""
    seed = 14
    hp = W.host_input_program(n, seed, outputs=("C", "D", "E", "r", "f"))
    ins = {nm: oracle.init_matrix(seed, b, n, n).astype(np.float32) for nm, b in (("A", 0), ("B", 1), ("C0", 2))}
    res = {}
    for fuse in (False, True):
        p = gao.prog_from_workload(hp, gemm_prec=prec, fuse_chains=fuse)
        for nm, v in ins.items():
            gao.prog_set_input(p, hp.index(nm), v)
        gao.prog_run(p, (1 << hp.n_loops) - 1)
        res[fuse] = (outputs(gao, p, hp), gao.prog_stats(p))
        gao.prog_destroy(p)
    (a, _), (b, st) = res[False], res[True]
    for nm in ("C", "D", "E", "r"):
        assert np.array_equal(a[nm], b[nm]), nm
    assert abs(a["f"] - b["f"]) <= 2e-7 * a["f"]
    assert [s["placement"] for s in st] == [1, 2, 2, 2, 2]
    assert st[0]["h2d_bytes"] == 3 * n * n * 4


@pytest.mark.parametrize("n,prec", [(640, 3), (2048, 3), (2304, 1)])
def test_special_values_fused_and_overlapped(gao, n, prec):
    """Host inputs with NaNs of either sign, infinities, -0 and huge values in A, B and C0
    (n = 640: one launch; n >= 2048: copy-overlapped row blocks, the first in column ranges):
    the chain in the GEMM's epilogue gives the same bits of C, D, E and r as the separate
    loops, and a norm that is NaN exactly when theirs is."""
    seed = 15
    hp = W.host_input_program(n, seed, outputs=("C", "D", "E", "r", "f"))
    ins = {nm: oracle.init_matrix(seed, b, n, n).astype(np.float32) for nm, b in (("A", 0), ("B", 1), ("C0", 2))}
    rng = np.random.default_rng(n)
    specials = np.array([0x7FC00000, 0xFFC00000, 0x7F800001, 0x7F800000, 0xFF800000, 0x80000000, 0x7E967699],
                        dtype=np.uint32)
    for nm in ("A", "B", "C0"):
        bits = ins[nm].view(np.uint32)
        for v in specials:
            bits[rng.integers(0, n // 2, 2), rng.integers(0, n // 2, 2)] = v
    res = {}
    for fuse in (False, True):
        p = gao.prog_from_workload(hp, gemm_prec=prec, fuse_chains=fuse)
        for nm, v in ins.items():
            gao.prog_set_input(p, hp.index(nm), v)
        gao.prog_run(p, (1 << hp.n_loops) - 1)
        res[fuse] = outputs(gao, p, hp)
        gao.prog_destroy(p)
    a, b = res[False], res[True]
    for nm in ("C", "D", "E", "r"):
        assert np.array_equal(a[nm].view(np.uint32), b[nm].view(np.uint32)), nm
    assert np.isnan(a["C"]).any() and np.isfinite(a["C"]).any()
    assert np.isnan(a["f"]) == np.isnan(b["f"])


def test_twelve_loop_elementwise_chain_bit_identical(gao):
    """ReLU, E - 0.5F, its square and P = H + 0.25D run as one element-wise pass (F, G, H
    never written): the same P, column maxima and sum as the separate loops."""
    prog = W.twelve_loop(300, 96, W.SEED_TWELVE_LOOP, outputs=("C", "D", "E", "r", "P", "q", "s"))
    res = {}
    for fuse in (False, True):
        p = gao.prog_from_workload(prog, gemm_prec=2, fuse_chains=fuse)
        gao.prog_run(p, (1 << 12) - 1)
        res[fuse] = (outputs(gao, p, prog), gao.prog_stats(p))
        gao.prog_destroy(p)
    (a, _), (b, st) = res[False], res[True]
    for nm in ("C", "D", "E", "r", "P", "q"):
        assert np.array_equal(a[nm], b[nm]), nm
    assert a["s"] == b["s"]
    assert [s_["placement"] for s_ in st] == [1, 1, 2, 2, 2, 2, 1, 2, 2, 2, 1, 1]
    assert st[6]["launches"] == 1


def _ew_program(rng, n_loops, rows, cols):
    """Random element-wise loops over a few initialised buffers (in place, both operands the
    same, references to older buffers), all buffers OUTPUT."""
    nb = 6
    bufs = [W.Buffer(f"b{i}", rows, cols, W.F32, W.OUTPUT) for i in range(nb)]
    loops = [W.Loop(W.INIT, [], [0, 1, 2])]
    defined = [0, 1, 2]
    for _ in range(n_loops):
        kind = int(rng.choice([W.RELU, W.SQUARE, W.AXPY]))
        out = int(rng.integers(0, nb))
        x = int(rng.choice(defined))
        if kind == W.AXPY:
            y = int(rng.choice(defined))
            loops.append(W.Loop(W.AXPY, [x, y], [out], alpha=float(rng.choice([2.0, -0.5, 0.25, 1.0]))))
        else:
            loops.append(W.Loop(kind, [x], [out]))
        if out not in defined:
            defined.append(out)
    for i in range(nb):
        if i not in defined:
            bufs[i].role = W.TEMP
    return W.Program("ew_random", bufs, loops, 61)


@pytest.mark.parametrize("seed", range(6))
def test_random_elementwise_chains_bit_identical(gao, seed):
    rng = np.random.default_rng(seed)
    rows, cols = [(64, 64), (37, 45), (128, 3)][seed % 3]
    prog = _ew_program(rng, 10, rows, cols)
    full = (1 << prog.n_loops) - 1
    genes = [full, full & ~(1 << int(rng.integers(1, prog.n_loops)))]
    for gene in genes:
        res = {}
        for fuse in (False, True):
            p = gao.prog_from_workload(prog, fuse_chains=fuse)
            gao.prog_run(p, gene)
            res[fuse] = {b.name: gao.prog_output(p, i).copy() for i, b in enumerate(prog.buffers)
                         if b.role == W.OUTPUT}
            gao.prog_destroy(p)
        for nm in res[False]:
            assert np.array_equal(res[False][nm].view(np.uint32), res[True][nm].view(np.uint32)), (seed, gene, nm)


def test_full_size_twelve_loop_sampled(gao):
    """The twelve-loop program at the size bench.py runs it: m = 16384, k = 4096, BF16x3, all twelve loops on
    the GPU with the fused chains.  C on sampled entries against the oracle (entry by entry
    from the counter hash) and on every entry through Freivalds' identities; D = C + 2S,
    E = D^T and P from E and D (the element-wise operations restated in binary32) exactly
    everywhere; the row sums in their fixed order on every row; column maxima exact; norm and
    sum within their reduction bounds."""
    import math
    from test_gpu_rowsum import rowsum_fixed_order
    m, k, seed = 16384, 4096, W.SEED_TWELVE_LOOP
    prog = W.twelve_loop(m, k, seed, outputs=("C", "D", "E", "r", "f", "P", "q", "s"))
    p = gao.prog_from_workload(prog, gemm_prec=2, fuse_chains=gao.FUSE_ON)
    gao.prog_run(p, (1 << 12) - 1)
    st = gao.prog_stats(p)
    assert [s_["placement"] for s_ in st] == [1, 1, 2, 2, 2, 2, 1, 2, 2, 2, 1, 1]
    out = outputs(gao, p, prog)
    gao.prog_destroy(p)
    rng = np.random.default_rng(5)
    ii, jj = rng.integers(0, m, 512), rng.integers(0, m, 512)
    want = oracle.gemm_init_entries(seed, (0, 1, 2), False, m, m, k, 1.5, 0.5, ii, jj)
    C, D, E, P = out["C"], out["D"], out["E"], out["P"]
    got = C[ii, jj].astype(np.float64)
    err = math.sqrt(float(((got - want) ** 2).mean()) / float((want ** 2).mean()))
    assert err <= TOL[2], err
    # every entry of C: C x = 1.5 A (B x) + 0.5 C0 x and y^T C = 1.5 (y^T A) B + 0.5 y^T C0
    # for random sign vectors (Freivalds 1977), operands in binary64 from the hash
    A, B = oracle.init_matrix(seed, 0, m, k), oracle.init_matrix(seed, 1, k, m)
    C0 = oracle.init_matrix(seed, 2, m, m)
    x, y = rng.choice([-1.0, 1.0], size=m), rng.choice([-1.0, 1.0], size=m)
    right, left = 1.5 * (A @ (B @ x)) + 0.5 * (C0 @ x), 1.5 * ((y @ A) @ B) + 0.5 * (y @ C0)
    del A, B, C0
    C64 = C.astype(np.float64)
    res = max(float(np.linalg.norm(C64 @ x - right) / np.linalg.norm(right)),
              float(np.linalg.norm(y @ C64 - left) / np.linalg.norm(left)))
    del C64
    print(f"twelve-loop m={m} k={k} Freivalds residual {res:.3e}")
    assert res <= TOL[2], res
    S = oracle.init_matrix(seed, 3, m, m).astype(np.float32)
    assert np.array_equal(D, C + np.float32(2.0) * S)
    del S
    assert np.array_equal(E, D.T)
    F = np.where(E > 0, E, np.float32(0))
    G = E + np.float32(-0.5) * F
    del F
    H = G * G
    del G
    assert np.array_equal(P, H + np.float32(0.25) * D)
    del H
    assert np.array_equal(out["r"], rowsum_fixed_order(E))
    assert np.array_equal(out["q"].ravel(), P.max(axis=0))
    E64 = E.astype(np.float64)
    fn = math.sqrt(float(np.einsum("ij,ij->", E64, E64)))
    assert abs(out["f"] - fn) <= 2e-7 * fn
    del E64
    P64 = P.astype(np.float64)
    assert abs(out["s"] - float(P64.sum())) <= 4 * 2.0 ** -24 * float(np.abs(P64).sum())
