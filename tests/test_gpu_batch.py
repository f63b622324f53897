"""Batched gene evaluation over a suite of programs of uneven sizes (C ABI batch_*):
every program's outputs after every gene match the FP64 oracle, the cache serves
repeated genes, and the GA on top follows the oracle GA's trajectory on the measured
times."""
import numpy as np
import pytest

import oracle
from oracle import ga as oga
import workloads as W

pytestmark = pytest.mark.gpu

TOL = {1: 5e-3, 2: 2e-5, 3: 1e-6, 0: 1e-6, 4: 6e-2}  # by gemm_prec


@pytest.fixture(scope="module")
def gao():
    from paper_1806_01430_gb300 import _build
    _build.build()
    import paper_1806_01430_gb300 as g
    return g


def suite(gao, sizes, prec, outputs=("C", "D", "E", "r", "f")):
    progs = [W.six_loop(n, 3000 + i, outputs=outputs) for i, n in enumerate(sizes)]
    handles = [gao.prog_from_workload(p, gemm_prec=prec) for p in progs]
    return progs, handles


def check_outputs(gao, progs, handles, refs, mask, prec):
    tol = TOL[prec] if (mask >> 1) & 1 else 1e-6
    for prog, h, ref in zip(progs, handles, refs):
        for nm in ("C", "D", "E", "r"):
            got = gao.prog_output(h, prog.index(nm))
            err = oracle.rel_err(got, ref[nm])
            assert err <= tol, (prog.name, mask, nm, err)
        f = float(gao.prog_output(h, prog.index("f"))[0, 0])
        assert abs(f - ref["f"]) <= tol * ref["f"]


@pytest.mark.parametrize("prec", [3, 2])
def test_batch_all_genes_match_oracle(gao, prec):
    sizes = [130, 64, 257, 200, 96, 300]
    progs, handles = suite(gao, sizes, prec)
    refs = [oracle.run_program(p) for p in progs]
    b = gao.batch_create(handles)
    st0 = gao.batch_stats(b)
    assert st0["graphs"] == 6 and st0["gemm_tiles"] == sum(((n + 127) // 128) ** 2 for n in sizes)
    for mask in range(64):
        fit, sec, hits = gao.batch_evaluate(b, [mask])
        assert hits == 0 and sec[0] > 0 and fit[0] == pytest.approx(1 / np.sqrt(sec[0]))
        check_outputs(gao, progs, handles, refs, mask, prec)
    fit, sec, hits = gao.batch_evaluate(b, list(range(64)))
    assert hits == 64
    st = gao.batch_stats(b)
    assert st["executed"] == 64 and st["served"] == 64 and st["gemm_phase_ms"] > 0
    gao.batch_destroy(b)


def test_batch_fp32_simt_and_fp8(gao):
    for prec in (0, 4):
        sizes = [70, 129, 256]
        progs, handles = suite(gao, sizes, prec)
        refs = [oracle.run_program(p) for p in progs]
        b = gao.batch_create(handles)
        for mask in (0b111111, 0b000010, 0b111101):
            gao.batch_evaluate(b, [mask])
            check_outputs(gao, progs, handles, refs, mask, prec)
        gao.batch_destroy(b)


def test_batch_ga_matches_oracle_on_measured_times(gao):
    sizes = [128, 192, 384, 160]
    progs, handles = suite(gao, sizes, 2, outputs=("f",))
    b = gao.batch_create(handles)
    _, secs, _ = gao.batch_evaluate(b, list(range(64)))
    table = secs.copy()
    res = gao.batch_ga_run(b, pop=20, generations=20, pc=0.9, pm=0.05, seed=7)
    ref = oga.run(lambda m: float(table[m]), 6, 20, 20, 0.9, 0.05, 7)
    assert res.populations == ref.populations
    assert res.best_mask == ref.best_mask and res.best_s == ref.best_s
    gao.batch_destroy(b)


def test_batch_rejects_mixed_programs(gao):
    a = gao.prog_from_workload(W.six_loop(64, 1), gemm_prec=3)
    c = gao.prog_from_workload(W.six_loop(64, 2), gemm_prec=2)
    with pytest.raises(gao.GaoError):
        gao.batch_create([a, c])
    d = gao.prog_from_workload(W.twelve_loop(32, 16, 3), gemm_prec=3)
    with pytest.raises(gao.GaoError):
        gao.batch_create([a, d])
    with pytest.raises(gao.GaoError):
        gao.batch_create([a, a])


def test_batch_l2_prefetch_changes_no_value(gao):
    """The grouped launch with tile configuration bit 2 (L2 prefetch of the operand tiles)
    gives the same bits as without it, for every program of the suite."""
    sizes = [300, 129, 520, 64]
    progs = [W.six_loop(n, 3100 + i, outputs=("C", "D", "E", "r", "f")) for i, n in enumerate(sizes)]
    outs = []
    for cfg in (0, 4):
        handles = [gao.prog_from_workload(p, gemm_prec=2, tile_cfg=cfg) for p in progs]
        b = gao.batch_create(handles)
        gao.batch_evaluate(b, [0b111111])
        outs.append([gao.prog_output(h, p.index("C")) for h, p in zip(handles, progs)])
        gao.batch_destroy(b)
        for h in handles:
            gao.prog_destroy(h)
    for x, y in zip(*outs):
        assert np.array_equal(x, y)


def test_batch_autotune_keeps_parity(gao):
    sizes = [300, 129, 520, 64]
    progs, handles = suite(gao, sizes, 3)
    refs = [oracle.run_program(p) for p in progs]
    b = gao.batch_create(handles)
    r = gao.batch_autotune(b, pop=6, generations=4, seed=2)
    assert r["evaluations"] >= 1 and r["best_ms"] > 0 and r["kchunk"] in (64, 128, 256, 512)
    assert r["best_ms"] <= r["default_ms"]  # the configuration in place stays unless beaten
    for mask in (0b111111, 0b111110, 0b101011):
        gao.batch_evaluate(b, [mask])
        check_outputs(gao, progs, handles, refs, mask, 3)
    gao.batch_destroy(b)


@pytest.mark.parametrize("prec", [3, 2])
def test_batch_fused_chain_matches_unfused(gao, prec):
    """Programs created with GAO_FUSE_ON: a gene that puts the GEMM, scale-add and transpose
    (and the row sums / norm that follow) on the GPU runs them in the grouped launch's
    epilogue.  Under every gene: C, D, E and row sums bit-identical to the unfused batch,
    the norm within its reduction's rounding, and the oracle's tolerance."""
    sizes = [130, 64, 257, 200, 96, 300]
    progs = [W.six_loop(n, 3200 + i, outputs=("C", "D", "E", "r", "f")) for i, n in enumerate(sizes)]
    refs = [oracle.run_program(p) for p in progs]
    runs = {}
    for fuse in (gao.FUSE_OFF, gao.FUSE_ON):
        handles = [gao.prog_from_workload(p, gemm_prec=prec, fuse_chains=fuse) for p in progs]
        b = gao.batch_create(handles)
        res = {}
        for mask in range(64):
            gao.batch_evaluate(b, [mask])
            res[mask] = [{nm: gao.prog_output(h, p.index(nm)).copy() for nm in ("C", "D", "E", "r", "f")}
                         for h, p in zip(handles, progs)]
            if fuse == gao.FUSE_ON:
                check_outputs(gao, progs, handles, refs, mask, prec)
        st = gao.batch_stats(b)
        runs[fuse] = (res, st)
        gao.batch_destroy(b)
        for h in handles:
            gao.prog_destroy(h)
    (plain, st0), (fused, st1) = runs[gao.FUSE_OFF], runs[gao.FUSE_ON]
    assert st0["fused_phases"] == 0
    # genes with GEMM (bit 1), scale-add (bit 2) and transpose (bit 3) on the GPU fuse
    assert st1["fused_phases"] == sum(1 for m in range(64) if (m >> 1) & 7 == 7)
    for mask in range(64):
        for a, c in zip(plain[mask], fused[mask]):
            for nm in ("C", "D", "E", "r"):
                assert np.array_equal(a[nm], c[nm]), (mask, nm)
            assert abs(float(a["f"][0, 0]) - float(c["f"][0, 0])) <= 2e-7 * abs(float(a["f"][0, 0])), mask


def test_batch_rejects_mixed_or_gene_fusion(gao):
    a = gao.prog_from_workload(W.six_loop(64, 1), gemm_prec=3, fuse_chains=gao.FUSE_ON)
    c = gao.prog_from_workload(W.six_loop(80, 2), gemm_prec=3)
    with pytest.raises(gao.GaoError):
        gao.batch_create([a, c])
    g = gao.prog_from_workload(W.six_loop(64, 3), gemm_prec=3, fuse_chains=gao.FUSE_GENE)
    with pytest.raises(gao.GaoError):
        gao.batch_create([g])


def test_batch_full_suite_sampled(gao):
    """The batched workload at full size: the bench's 64-program suite (n log-uniform in [128, 2048]),
    BF16x3 with fused chains, the all-GPU gene in one batched evaluation.  Every program: sampled
    C entries against the oracle (entry by entry from the counter hash), D = C + 2A and E = D^T
    exactly, row sums in their fixed order exactly, the norm within its rounding bound."""
    import math
    from test_gpu_rowsum import rowsum_fixed_order
    sizes = W.batch_sizes(64)
    progs = [W.six_loop(n, W.SEED_BATCH_BASE + p, outputs=("C", "D", "E", "r", "f"))
             for p, n in enumerate(sizes)]
    handles = [gao.prog_from_workload(pr, gemm_prec=2, fuse_chains=gao.FUSE_ON) for pr in progs]
    b = gao.batch_create(handles)
    fit, sec, hits = gao.batch_evaluate(b, [0b111111])
    st = gao.batch_stats(b)
    assert sec[0] > 0 and st["fused_phases"] == 1
    # one grouped INIT, two operand splits per program, one grouped GEMM, the row sums and the
    # norm from each program's partials
    assert st["kernel_launches"] == 1 + 2 * 64 + 1 + 2 * 64
    rng = np.random.default_rng(17)
    for prog, h in zip(progs, handles):
        n, seed = prog.buffers[0].rows, prog.seed
        C, D, E = (gao.prog_output(h, prog.index(nm)) for nm in ("C", "D", "E"))
        ii, jj = rng.integers(0, n, 32), rng.integers(0, n, 32)
        want = oracle.gemm_init_entries(seed, (0, 1, 2), False, n, n, n, 1.5, 0.5, ii, jj)
        got = C[ii, jj].astype(np.float64)
        err = math.sqrt(float(((got - want) ** 2).mean()) / float((want ** 2).mean()))
        assert err <= TOL[2], (n, err)
        A = oracle.init_matrix(seed, 0, n, n).astype(np.float32)
        assert np.array_equal(D, C + np.float32(2.0) * A), n
        assert np.array_equal(E, D.T), n
        assert np.array_equal(gao.prog_output(h, prog.index("r")), rowsum_fixed_order(E)), n
        E64 = E.astype(np.float64)
        fn = math.sqrt(float((E64 * E64).sum()))
        assert abs(float(gao.prog_output(h, prog.index("f"))[0, 0]) - fn) <= 2e-7 * fn, n
    gao.batch_destroy(b)
    for h in handles:
        gao.prog_destroy(h)


# ---- generations: several genes measured together, their GEMMs in one grouped launch -----------

def _replica_outputs(gao, b, progs, r):
    out = []
    for i, prog in enumerate(progs):
        h = gao.batch_replica_prog(b, r, i)
        out.append({nm: gao.prog_output(h, prog.index(nm)).copy() for nm in ("C", "D", "E", "r", "f")})
    return out


@pytest.mark.parametrize("prec,fuse", [(3, False), (2, True), (1, True)])
def test_generation_results_match_single_gene_runs(gao, prec, fuse):
    """Four genes measured together (replicas = 4): every copy of the suite ends with its gene's
    results, bit-identical to the same gene run alone (C, D, E, row sums; the norm within its
    reduction's rounding when fused), and within the oracle's tolerance; the genes that offload
    the GEMM share one grouped launch."""
    sizes = [130, 64, 257, 200, 96, 300]
    progs = [W.six_loop(n, 3300 + i, outputs=("C", "D", "E", "r", "f")) for i, n in enumerate(sizes)]
    refs = [oracle.run_program(p) for p in progs]
    fz = gao.FUSE_ON if fuse else gao.FUSE_OFF
    genes = [0b111111, 0b000010, 0b111110, 0b001111, 0b110011, 0b011011, 0b111111 ^ 0b000100, 0b000000]
    alone = {}
    handles = [gao.prog_from_workload(p, gemm_prec=prec, fuse_chains=fz) for p in progs]
    b = gao.batch_create(handles)
    for g in genes:
        gao.batch_evaluate(b, [g])
        alone[g] = _replica_outputs(gao, b, progs, 0)
    gao.batch_destroy(b)
    for h in handles:
        gao.prog_destroy(h)
    handles = [gao.prog_from_workload(p, gemm_prec=prec, fuse_chains=fz) for p in progs]
    b = gao.batch_create(handles, replicas=4)
    st0 = gao.batch_stats(b)
    assert st0["replicas"] == 4
    for k in range(0, len(genes), 4):
        group = genes[k:k + 4]
        before = gao.batch_stats(b)
        fit, sec, hits = gao.batch_evaluate(b, group)
        after = gao.batch_stats(b)
        assert hits == 0 and all(s > 0 for s in sec)
        n_gemm = sum(1 for g in group if (g >> 1) & 1)
        assert after["grouped_launches"] - before["grouped_launches"] == (1 if n_gemm else 0)
        assert after["grouped_genes"] - before["grouped_genes"] == n_gemm
        for r, g in enumerate(group):
            got = _replica_outputs(gao, b, progs, r)
            tol = TOL[prec] if (g >> 1) & 1 else 1e-6
            for a, c, ref in zip(alone[g], got, refs):
                for nm in ("C", "D", "E", "r"):
                    assert np.array_equal(a[nm], c[nm]), (g, nm)
                    assert oracle.rel_err(c[nm], ref[nm]) <= tol, (g, nm)
                assert abs(float(a["f"][0, 0]) - float(c["f"][0, 0])) <= 2e-7 * abs(float(a["f"][0, 0]))
    gao.batch_destroy(b)


def test_generation_times_rank_like_single_runs(gao):
    """All 64 genes timed one at a time (wall time of the suite) and 16 at a time (attributed
    times in shared launches): the attributed times order the genes like the single runs.
    Each mode measures every gene twice and keeps the shorter time (a shared machine's noise
    only ever adds time)."""
    sizes = [256, 384, 192, 512, 128, 320]
    progs = [W.six_loop(n, 3400 + i, outputs=("f",)) for i, n in enumerate(sizes)]
    times = {}
    for reps in (1, 16):
        handles = [gao.prog_from_workload(p, gemm_prec=2) for p in progs]
        b = gao.batch_create(handles, replicas=reps)
        gao.batch_evaluate(b, [0b111111])  # warm
        runs = []
        for rep in range(2):
            gao.batch_set_replicas(b, reps)  # clears the cache
            st0 = gao.batch_stats(b)
            _, sec, _ = gao.batch_evaluate(b, list(range(64)))
            runs.append(np.array(sec))
            st = gao.batch_stats(b)
            if reps == 16:  # four groups, each GEMM-offloading subset of 16 genes in one launch
                assert st["grouped_launches"] - st0["grouped_launches"] == 4
                assert st["grouped_genes"] - st0["grouped_genes"] == 32
        times[reps] = np.minimum(runs[0], runs[1])
        gao.batch_destroy(b)
        for h in handles:
            gao.prog_destroy(h)
    a, c = times[1], times[16]
    ra, rc = np.argsort(np.argsort(a)), np.argsort(np.argsort(c))
    rho = 1.0 - 6.0 * float(((ra - rc) ** 2).sum()) / (64 * (64 ** 2 - 1))
    print(f"Spearman rank correlation, attributed vs single-run gene times: {rho:.3f}")
    assert rho >= 0.9, rho
    # the attributed time leaves out host overheads: never far above the wall time
    assert np.all(c <= 1.5 * a + 1e-3)


@pytest.mark.parametrize("reps", [1, 8])
def test_generation_ga_follows_oracle_ga(gao, reps):
    """With every gene's time in the batch's cache, the GA (per-generation evaluation) draws
    exactly the oracle GA's populations, with or without replicas."""
    sizes = [128, 192, 384, 160]
    progs, handles = suite(gao, sizes, 2, outputs=("f",))
    b = gao.batch_create(handles, replicas=reps)
    _, secs, _ = gao.batch_evaluate(b, list(range(64)))
    table = np.array(secs)
    res = gao.batch_ga_run(b, pop=20, generations=20, pc=0.9, pm=0.05, seed=7)
    ref = oga.run(lambda m: float(table[m]), 6, 20, 20, 0.9, 0.05, 7)
    assert res.populations == ref.populations
    assert res.best_mask == ref.best_mask and res.best_s == ref.best_s
    gao.batch_destroy(b)


def test_generation_ga_measures_each_generation_together(gao):
    """batch_ga_run with replicas: the genes new in a generation are measured together, so the
    grouped launches serve several genes each."""
    sizes = W.batch_sizes(16)
    progs = [W.six_loop(n, W.SEED_BATCH_BASE + p, outputs=("f",)) for p, n in enumerate(sizes)]
    handles = [gao.prog_from_workload(pr, gemm_prec=2, fuse_chains=gao.FUSE_ON) for pr in progs]
    b = gao.batch_create(handles, replicas=20)
    res = gao.batch_ga_run(b, pop=20, generations=6, pc=0.9, pm=0.05, seed=7, timeout_s=-1.0)
    st = gao.batch_stats(b)
    assert res.evaluations >= 20 and st["grouped_launches"] >= 1
    assert st["grouped_genes"] > 2 * st["grouped_launches"]
    assert np.isfinite(res.best_s) and res.best_s > 0
    gao.batch_destroy(b)
