"""GPU parity of the loop program through the C ABI against the FP64 oracle.

Tolerances (normwise relative error ||x - ref||_F / ||ref||_F):
  * bit-exact: INIT (counter hash), TRANSPOSE, AXPY/RELU/SQUARE given equal
    inputs, COLMAX given equal inputs;
  * 1e-6: FP32 SIMT GEMM and everything downstream of it (the stated bound for the
    FP32 and split-BF16 paths);
  * Frobenius / SUM over the device's own input: 2e-7 relative (binary32 partial
    sums of 4 squares: each group carries at most ~4 units of 2^-24 relative error,
    the binary64 accumulation adds nothing visible).
"""
import math

import numpy as np
import pytest

import oracle
from oracle import ga as oga
import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-6


@pytest.fixture(scope="module")
def gao():
    from paper_1806_01430_gb300 import _build
    _build.build()
    import paper_1806_01430_gb300 as g
    return g


def run_prog(gao, prog, mask, **kw):
    p = gao.prog_from_workload(prog, **kw)
    secs = gao.prog_run(p, mask)
    out = {}
    for i, b in enumerate(prog.buffers):
        if b.role == W.OUTPUT:
            v = gao.prog_output(p, i)
            out[b.name] = float(v[0, 0]) if (b.rows, b.cols) == (1, 1) and b.dtype == W.F64 else v
    stats = gao.prog_stats(p)
    gao.prog_destroy(p)
    return out, secs, stats


def all_outputs(prog):
    for b in prog.buffers:
        b.role = W.OUTPUT
    return prog


def check_six(out, ref, tol=TOL):
    for nm in ("C", "D", "E", "r"):
        err = oracle.rel_err(out[nm], ref[nm])
        assert err <= tol, f"{nm}: rel err {err:.3e} > {tol}"
    if ref["f"] > 0:
        assert abs(out["f"] - ref["f"]) / ref["f"] <= tol
    else:
        assert out["f"] == 0.0


def check_internal_consistency(out):
    """Relations that hold exactly (or within the reduction bound) among the run's own outputs."""
    C, A, D, E = out["C"], out["A"], out["D"], out["E"]
    Dx = (C.astype(np.float64) + 2.0 * A.astype(np.float64)).astype(np.float32)  # exact 2a, one rounding
    assert np.array_equal(D, Dx), "scale-add is not c + 2a rounded once"
    assert np.array_equal(E, D.T), "transpose is not exact"
    E64 = E.astype(np.float64)
    r_ref = E64.sum(axis=1, keepdims=True)
    scale = np.abs(E64).sum(axis=1, keepdims=True) + 1e-300
    assert np.all(np.abs(out["r"] - r_ref) <= 1e-6 * scale + 1e-30)
    f_ref = math.sqrt(float((E64 * E64).sum()))
    if f_ref > 0:
        assert abs(out["f"] - f_ref) / f_ref <= 2e-7


def test_config0_n256_all_gpu(gao):
    prog = all_outputs(W.six_loop(256, W.SEED_N256))
    ref = oracle.run_program(prog)
    out, secs, stats = run_prog(gao, prog, 0b111111)
    check_six(out, ref)
    check_internal_consistency(out)
    for nm in ("A", "B"):
        assert np.array_equal(out[nm], ref[nm].astype(np.float32)), f"init {nm} not bit-exact"
    assert all(s["placement"] == 1 for s in stats)
    assert stats[1]["kernel_ms"] > 0


@pytest.mark.parametrize("n", [0, 1, 3, 8, 64, 127, 129, 132, 300])
def test_six_loop_ragged_sizes(gao, n):
    prog = all_outputs(W.six_loop(n, 4242 + n))
    ref = oracle.run_program(prog)
    out, _, _ = run_prog(gao, prog, 0b111111)
    if n == 0:
        assert out["f"] == 0.0
        return
    check_six(out, ref)
    check_internal_consistency(out)


def test_all_64_masks_invariance(gao):
    """Every gene gives the oracle's result within tolerance; loops with bitwise-equal
    inputs give bitwise-equal outputs whichever side runs them."""
    n = 96
    prog = all_outputs(W.six_loop(n, 31))
    ref = oracle.run_program(prog)
    p = gao.prog_from_workload(prog)
    by_gemm_side = {}
    init0 = None
    for mask in range(64):
        gao.prog_run(p, mask)
        out = {b.name: gao.prog_output(p, i) for i, b in enumerate(prog.buffers)}
        out["f"] = float(out["f"][0, 0])
        check_six(out, ref)
        check_internal_consistency(out)
        init = (out["A"], out["B"])
        if init0 is None:
            init0 = init
            assert np.array_equal(init[0], ref["A"].astype(np.float32))
        assert np.array_equal(init[0], init0[0]) and np.array_equal(init[1], init0[1])
        key = (mask >> 1) & 1
        if key in by_gemm_side:
            C0, D0, E0, r0 = by_gemm_side[key]
            assert np.array_equal(out["C"], C0)
            assert np.array_equal(out["D"], D0) and np.array_equal(out["E"], E0)
            assert np.array_equal(out["r"], r0)  # one row-sum order on both sides
        else:
            by_gemm_side[key] = (out["C"], out["D"], out["E"], out["r"])
        st = gao.prog_stats(p)
        for i, s in enumerate(st):
            assert s["placement"] == ((mask >> i) & 1)
        # data moves only at CPU/GPU boundaries
        if mask == 0:
            assert all(s["h2d_bytes"] == 0 and s["d2h_bytes"] == 0 for s in st[:-1])
        if mask == 0b000011:  # init+GEMM on GPU, D = C + 2A on CPU: C and A come back
            assert st[2]["d2h_bytes"] == 2 * n * n * 4
    gao.prog_destroy(p)


@pytest.mark.parametrize("shapes", [[(7, 13), (1, 3), (1000, 1001)], [(4096, 4096)], [(1, 1), (3, 5), (2, 2)]])
def test_init_outputs_bit_exact(gao, shapes):
    """One INIT loop with several outputs of ragged sizes (a tail of 1-3 elements after the
    whole quadruples, grids that cover a buffer in several trips): every element is the
    counter hash's value, bit for bit against the oracle's."""
    seed = 4242
    bufs = [W.Buffer(f"X{k}", r, c, W.F32, W.OUTPUT) for k, (r, c) in enumerate(shapes)]
    prog = W.Program("init_only", bufs, [W.Loop(W.INIT, [], list(range(len(shapes))))], seed)
    out, _, _ = run_prog(gao, prog, 0b1)
    for k, (r, c) in enumerate(shapes):
        assert np.array_equal(out[f"X{k}"], oracle.init_matrix(seed, k, r, c).astype(np.float32)), (k, r, c)


@pytest.mark.parametrize("prec", ["FP32_SIMT", "BF16X6", "BF16", "FP8"])
@pytest.mark.parametrize("fuse", [0, 1])
def test_empty_six_loop_program(gao, prec, fuse):
    """n = 0: every buffer empty, every gene runs, nothing is launched over an empty shape and
    the norm is 0, as in the oracle."""
    prog = W.six_loop(0, 5, outputs=("C", "D", "E", "r", "f"))
    p = gao.prog_from_workload(prog, gemm_prec=getattr(gao, prec), fuse_chains=fuse)
    for mask in (0b111111, 0b000000, 0b101010):
        gao.prog_run(p, mask)
        for nm in ("C", "D", "E"):
            assert gao.prog_output(p, prog.index(nm)).shape == (0, 0)
        assert gao.prog_output(p, prog.index("r")).shape == (0, 1)
        assert float(gao.prog_output(p, prog.index("f"))[0, 0]) == 0.0
    gao.prog_destroy(p)


def test_row_scaled_init_bit_exact(gao):
    prog = all_outputs(W.six_loop(200, W.SEED_N8192_ROWS, rowscale_a=True))
    ref = oracle.run_program(prog)
    for mask in (0b111111, 0b111110):
        out, _, _ = run_prog(gao, prog, mask)
        assert np.array_equal(out["A"], ref["A"].astype(np.float32))
        check_six(out, ref)


@pytest.mark.parametrize("m,k", [(200, 72), (129, 33), (64, 256)])
def test_twelve_loop_program(gao, m, k):
    prog = all_outputs(W.twelve_loop(m, k, W.SEED_TWELVE_LOOP))
    ref = oracle.run_program(prog)
    rng = np.random.default_rng(m + k)
    for mask in [(1 << 12) - 1, 0] + [int(x) for x in rng.integers(0, 1 << 12, size=3)]:
        out, _, stats = run_prog(gao, prog, mask)
        # every output under the 1e-6 gate; H = G (.) G roughly doubles G's relative error
        # (measured at most 5.5e-7 for H, P and q, against 3e-7 for C, D, E, F, G)
        for nm in ("C", "D", "E", "F", "G", "H", "P", "r", "q"):
            err = oracle.rel_err(out[nm], ref[nm])
            assert err <= TOL, f"mask {mask:012b} {nm}: {err:.2e}"
        for nm in ("f", "s"):
            assert abs(out[nm] - ref[nm]) <= TOL * abs(ref[nm]), nm
        # exact relations among the run's own outputs
        E, F, G, H, P, D = (out[x] for x in "EFGHPD")
        assert np.array_equal(F, np.maximum(E, 0).astype(np.float32))
        assert np.array_equal(H, (G.astype(np.float64) ** 2).astype(np.float32))
        assert np.array_equal(out["q"].ravel(), P.max(axis=0))
        s_ref = float(P.astype(np.float64).sum())
        assert abs(out["s"] - s_ref) <= 1e-6 * float(np.abs(P).astype(np.float64).sum())


@pytest.mark.parametrize("n,prec,cfg", [(2048, "BF16X6", 0), (2500, "BF16X3", 0), (2304, "BF16", 0),
                                        (2500, "BF16X6", 8), (2304, "BF16X3", 8)])
def test_overlapped_host_gemm_is_bit_identical(gao, n, prec, cfg):
    """A GEMM loop whose A comes from the host runs in row blocks overlapped with the copy;
    its C must carry the same bits as the one-launch GEMM on device-resident inputs (with
    tile configuration 8 on CTA pairs, row blocks of whole 256-row tiles)."""
    seed = 91
    pr = getattr(gao, prec)
    dev = W.six_loop(n, seed, outputs=("C", "r", "f"))
    p = gao.prog_from_workload(dev, gemm_prec=pr, tile_cfg=cfg)
    gao.prog_run(p, 0b111111)
    C_dev = gao.prog_output(p, dev.index("C")).copy()
    r_dev = gao.prog_output(p, dev.index("r")).copy()
    gao.prog_run(p, 0b111110)  # INIT on the CPU: A, B and C reach the GEMM from the host
    st = gao.prog_stats(p)
    assert st[1]["h2d_bytes"] == 3 * n * n * 4
    C_mix = gao.prog_output(p, dev.index("C"))
    assert np.array_equal(C_mix.view(np.uint32), C_dev.view(np.uint32))
    assert np.array_equal(gao.prog_output(p, dev.index("r")), r_dev)
    gao.prog_destroy(p)
    hp = W.host_input_program(n, seed, outputs=("C", "r", "f"))
    q = gao.prog_from_workload(hp, gemm_prec=pr, tile_cfg=cfg)
    for nm, b in (("A", 0), ("B", 1), ("C0", 2)):
        gao.prog_set_input(q, hp.index(nm), oracle.init_matrix(seed, b, n, n).astype(np.float32))
    gao.prog_run(q, (1 << hp.n_loops) - 1)
    assert np.array_equal(gao.prog_output(q, hp.index("C")).view(np.uint32), C_dev.view(np.uint32))
    gao.prog_destroy(q)


def test_host_input_program_matches(gao):
    n, seed = 160, 77
    prog = W.host_input_program(n, seed, outputs=("C", "r", "f"))
    ins = {"A": oracle.init_matrix(seed, 0, n, n), "B": oracle.init_matrix(seed, 1, n, n),
           "C0": oracle.init_matrix(seed, 2, n, n)}
    ref = oracle.run_program(prog, ins)
    p = gao.prog_from_workload(prog)
    for nm, v in ins.items():
        gao.prog_set_input(p, prog.index(nm), v.astype(np.float32))
    for mask in (0b11111, 0b00000, 0b10101):
        gao.prog_run(p, mask)
        st = gao.prog_stats(p)
        if mask & 1:
            assert st[0]["h2d_bytes"] == 3 * n * n * 4  # A, B, C0 copied in every run
        C = gao.prog_output(p, prog.index("C"))
        assert oracle.rel_err(C, ref["C"]) <= TOL
        assert oracle.rel_err(gao.prog_output(p, prog.index("r")), ref["r"]) <= TOL
        f = float(gao.prog_output(p, prog.index("f"))[0, 0])
        assert abs(f - ref["f"]) / ref["f"] <= TOL
    gao.prog_destroy(p)


def test_torch_arena_and_stream(gao):
    torch = pytest.importorskip("torch")
    prog = W.six_loop(128, 5, outputs=("C", "r", "f"))
    nbytes = gao.prog_device_bytes(prog.buffers, prog.loops, seed=prog.seed)
    arena = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    p = gao.prog_from_workload(prog, arena=arena, stream=s)
    gao.prog_run(p, 0b111111)
    ref = oracle.run_program(prog)
    assert oracle.rel_err(gao.prog_output(p, prog.index("C")), ref["C"]) <= TOL
    base = arena.data_ptr()
    assert base <= gao.prog_device_ptr(p, prog.index("C")) < base + nbytes
    gao.prog_destroy(p)
    with pytest.raises(gao.GaoError):  # arena too small
        gao.prog_from_workload(prog, arena=arena[: nbytes // 2])


def test_timeout_then_reusable(gao):
    prog = W.six_loop(1024, 9)
    p = gao.prog_from_workload(prog, timeout_s=1e-3)
    st, secs = gao.prog_run_status(p, 0b000000)  # CPU GEMM of 1024^3 cannot finish in 1 ms
    assert st == gao.GAO_ETIMEOUT and secs == pytest.approx(1e-3)
    st2, _ = gao.prog_run_status(p, 0b111111)
    assert st2 in (gao.GAO_OK, gao.GAO_ETIMEOUT)
    gao.prog_destroy(p)
    p = gao.prog_from_workload(prog)
    gao.prog_run(p, 0b111111)  # same program without a budget runs through
    gao.prog_destroy(p)


def test_device_wait_expires_without_trapping(gao):
    assert gao.gao_selftest_device_wait(0.05) == gao.GAO_ETIMEOUT
    # the context is still usable afterwards
    out, _, _ = run_prog(gao, W.six_loop(32, 1), 0b111111)
    assert out["f"] > 0


def test_bad_gene_bits(gao):
    p = gao.prog_from_workload(W.six_loop(16, 1))
    st, _ = gao.prog_run_status(p, 1 << 6)
    assert st == gao.GAO_EINVAL
    gao.prog_destroy(p)


def test_ga_evaluate_cache_and_ga_run_match_oracle(gao):
    """The GA over measured times: after every gene is measured once (cached), ga_run
    must follow the oracle GA's trajectory on that same time table, and the best gene
    must be the exhaustive optimum of the table."""
    prog = W.six_loop(256, W.SEED_N4096)
    p = gao.prog_from_workload(prog)
    masks = list(range(64))
    fit, secs, hits = gao.ga_evaluate([p], masks)
    assert hits == 0 and np.all(secs > 0) and np.allclose(fit, 1 / np.sqrt(secs))
    fit2, secs2, hits2 = gao.ga_evaluate([p], masks[::-1])
    assert hits2 == 64 and np.array_equal(secs2, secs[::-1])  # repeated genes are not re-measured
    table = secs.copy()
    res = gao.ga_run([p], pop=12, generations=12, pc=0.9, pm=0.05, seed=5)
    ref = oga.run(lambda m: float(table[m]), 6, 12, 12, 0.9, 0.05, 5)
    assert res.populations == ref.populations and res.best_mask == ref.best_mask
    best_m, best_t = oga.exhaustive(lambda m: float(table[m]), 6)
    assert table[res.best_mask] >= best_t
    gao.prog_destroy(p)


def test_full_size_n4096_sampled(gao):
    """The six-loop program at n = 4096, all-GPU gene, FP32 SIMT; sampled C entries against the
    oracle computed entry by entry from the counter hash, plus exact relations."""
    n, seed = 4096, W.SEED_N4096
    prog = all_outputs(W.six_loop(n, seed))
    out, _, _ = run_prog(gao, prog, 0b111111)
    rng = np.random.default_rng(0)
    ii = rng.integers(0, n, 256)
    jj = rng.integers(0, n, 256)
    want = oracle.gemm_init_entries(seed, (0, 1, 2), False, n, n, n, 1.5, 0.5, ii, jj)
    got = out["C"][ii, jj].astype(np.float64)
    err = math.sqrt(float(((got - want) ** 2).mean()) / float((want ** 2).mean()))
    assert err <= TOL, err
    check_internal_consistency(out)


def test_per_loop_transfer_mode(gao):
    """Directive-style offload without a data region: every GPU loop copies its inputs in
    and its outputs out.  Same results as resident buffers, more traffic, more time."""
    n = 512
    prog = all_outputs(W.six_loop(n, 91))
    ref = oracle.run_program(prog)
    res, naive = {}, {}
    for mode, out in ((gao.TRANSFER_RESIDENT, res), (gao.TRANSFER_PER_LOOP, naive)):
        p = gao.prog_from_workload(prog, transfer_mode=mode)
        for _ in range(2):
            out["s"] = gao.prog_run(p, 0b111111)
        out["vals"] = {b.name: gao.prog_output(p, i) for i, b in enumerate(prog.buffers)}
        out["stats"] = gao.prog_stats(p)
        gao.prog_destroy(p)
    for nm in ("A", "B", "C", "D", "E", "r", "f"):
        assert np.array_equal(res["vals"][nm], naive["vals"][nm])
    check_six({k: (float(v[0, 0]) if k == "f" else v) for k, v in naive["vals"].items()}, ref)
    st = naive["stats"]
    mat = n * n * 4
    assert st[0]["d2h_bytes"] == 3 * mat  # INIT: A, B, C out
    assert st[1]["h2d_bytes"] == 3 * mat and st[1]["d2h_bytes"] == mat  # GEMM: A, B, C in; C out
    assert st[2]["h2d_bytes"] == 2 * mat and st[3]["h2d_bytes"] == mat
    assert sum(s["h2d_bytes"] for s in res["stats"]) == 0
    assert naive["s"] > res["s"]


def test_config1_all_64_genes_n4096(gao):
    """The n = 4096 FP32 SIMT program under all 64 genes (CPU loops included).
    Every gene is measured once (cache), the fastest gene places the GEMM on the GPU, the
    paper's GA finds the exhaustive optimum of the measured times, and the outputs of
    the all-CPU and of the best gene both match the oracle on sampled GEMM entries and in
    their exact relations."""
    n, seed = 4096, W.SEED_N4096
    prog = W.six_loop(n, seed, outputs=("A", "C", "D", "E", "r", "f"))
    p = gao.prog_from_workload(prog, gemm_prec=0)
    fit, secs, hits = gao.ga_evaluate([p], list(range(64)))
    assert hits == 0 and np.all(secs > 0)
    best = int(np.argmin(secs))
    assert (best >> 1) & 1 == 1  # the GEMM belongs on the GPU
    assert secs[0] > 10 * secs[best]  # offloading pays off by an order of magnitude at least
    res = gao.ga_run([p], **W.PAPER_GA, seed=11)
    table = secs.copy()
    ref = oga.run(lambda m: float(table[m]), 6, 12, 12, 0.9, 0.05, 11)
    assert res.populations == ref.populations and res.best_mask == ref.best_mask
    rng = np.random.default_rng(4)
    ii, jj = rng.integers(0, n, 96), rng.integers(0, n, 96)
    want = oracle.gemm_init_entries(seed, (0, 1, 2), False, n, n, n, 1.5, 0.5, ii, jj)
    for mask in (0, best):
        gao.prog_run(p, mask)
        out = {nm: gao.prog_output(p, prog.index(nm)) for nm in ("A", "C", "D", "E", "r", "f")}
        out["f"] = float(out["f"][0, 0])
        got = out["C"][ii, jj].astype(np.float64)
        err = math.sqrt(float(((got - want) ** 2).mean()) / float((want ** 2).mean()))
        assert err <= TOL, (mask, err)
        check_internal_consistency(out)
    gao.prog_destroy(p)


def test_ga_checkpoint_and_resume(gao, tmp_path):
    """The measurement cache is the search's state (Sec. 4): exported after a few
    generations and imported into fresh program handles, a ga_run with the same seed
    replays those generations from the cache and continues."""
    prog = W.six_loop(192, 55, outputs=("C", "r", "f"))
    p = gao.prog_from_workload(prog, gemm_prec=gao.FP32_SIMT)
    r1 = gao.ga_run([p], pop=8, generations=3, seed=4)
    path = str(tmp_path / "search.json")
    gao.ga_checkpoint([p], path)
    genes, secs = gao.prog_cache_export(p)
    assert len(genes) == r1.evaluations and genes == sorted(genes)
    q = gao.prog_from_workload(prog, gemm_prec=gao.FP32_SIMT)
    gao.ga_resume([q], path)
    fit, s2, hits = gao.ga_evaluate([q], genes)
    assert hits == len(genes) and list(s2) == secs  # served, not measured
    r2 = gao.ga_run([q], pop=8, generations=6, seed=4)
    assert [h["best_mask"] for h in r2.history[:3]] == [h["best_mask"] for h in r1.history]
    assert [h["best_s"] for h in r2.history[:3]] == [h["best_s"] for h in r1.history]
    g2, _ = gao.prog_cache_export(q)
    assert set(genes) <= set(g2)
    with pytest.raises(gao.GaoError):
        gao.prog_cache_import(q, [1 << 6], [0.1])  # longer than the gene
    gao.prog_destroy(p)
    gao.prog_destroy(q)
