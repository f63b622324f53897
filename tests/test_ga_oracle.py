"""Pins of the Simple-GA oracle against the paper's definitions (Sec. 3.3, Sec. 4,
Sec. 5.1.2), brute-force search over all genes, and operator statistics."""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import ga
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _table_fn(table, calls=None):
    def f(m):
        if calls is not None:
            calls.append(m)
        return float(table[m])
    return f


def test_python_splitmix_matches_published_and_c():
    want = [int(l, 16) for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) if l.startswith("0x")]
    r = ga.SplitMix64(0)
    assert [r.next() for _ in range(3)] == want
    r = ga.SplitMix64(123456789)
    assert [r.next() for _ in range(50)] == [int(x) for x in oracle.splitmix64_stream(123456789, 50)]


def test_uniform_and_below_ranges():
    r = ga.SplitMix64(9)
    xs = [r.uniform() for _ in range(20000)]
    assert min(xs) >= 0.0 and max(xs) < 1.0
    assert abs(np.mean(xs) - 0.5) < 5 * math.sqrt(1 / 12 / len(xs))
    ks = [r.below(7) for _ in range(14000)]
    counts = np.bincount(ks, minlength=7)
    assert counts.min() > 1700 and counts.max() < 2300 and len(counts) == 7


def test_fitness_definition():
    assert ga.fitness_of(4.0) == 0.5
    assert ga.fitness_of(0.25) == 2.0
    assert ga.fitness_of(-1.0) == 0.0 and ga.fitness_of(float("inf")) == 0.0 and ga.fitness_of(float("nan")) == 0.0
    ts = [0.1, 0.5, 2.0, 9.0]
    fs = [ga.fitness_of(t) for t in ts]
    assert fs == sorted(fs, reverse=True)  # faster is fitter


def test_roulette_proportional():
    r = ga.SplitMix64(3)
    fit = [1.0, 2.0, 3.0, 4.0, 0.0]
    n = 40000
    counts = np.bincount([ga.roulette(r, fit) for _ in range(n)], minlength=5)
    expect = np.array(fit) / sum(fit) * n
    assert counts[4] == 0
    chi2 = float(((counts[:4] - expect[:4]) ** 2 / expect[:4]).sum())
    assert chi2 < 20.0  # 3 dof, p ~ 2e-4
    # all-zero fitness: uniform choice
    counts = np.bincount([ga.roulette(r, [0.0] * 4) for _ in range(8000)], minlength=4)
    assert counts.min() > 1700


def test_elite_preserved_and_best_monotone():
    table = W.random_time_table(10, seed=4)
    res = ga.run(_table_fn(table), 10, pop=12, generations=15, pc=0.9, pm=0.05, seed=11)
    for g in range(len(res.populations) - 1):
        popg = res.populations[g]
        fit = [ga.fitness_of(table[m]) for m in popg]
        e = int(np.argmax(fit))  # first index among the fittest
        assert res.populations[g + 1][0] == popg[e]
    bests = [h.best_s for h in res.history]
    running = np.minimum.accumulate(bests)
    assert res.best_s == running[-1] == table[res.best_mask]
    assert all(bests[g + 1] <= bests[g] for g in range(len(bests) - 1))  # elite keeps the best


def test_no_operators_means_copies_only():
    table = W.random_time_table(8, seed=5)
    res = ga.run(_table_fn(table), 8, pop=10, generations=8, pc=0.0, pm=0.0, seed=2)
    for g in range(len(res.populations) - 1):
        assert set(res.populations[g + 1]) <= set(res.populations[g])


def test_operator_rates():
    n_genes = 12
    flat = np.ones(1 << n_genes)
    res = ga.run(_table_fn(flat), n_genes, pop=20, generations=200, pc=0.9, pm=0.05, seed=8)
    st = res.stats
    p = st["crossovers"] / st["pairs"]
    assert abs(p - 0.9) < 5 * math.sqrt(0.9 * 0.1 / st["pairs"])
    q = st["flips"] / st["mutation_trials"]
    assert abs(q - 0.05) < 5 * math.sqrt(0.05 * 0.95 / st["mutation_trials"])
    # the elite plus the children fill every generation
    assert all(len(pg) == 20 for pg in res.populations)


def test_single_flip_mutation_mode():
    table = W.random_time_table(9, seed=6)
    res = ga.run(_table_fn(table), 9, pop=9, generations=6, pc=0.0, pm=1.0, seed=3, mutation=1)
    for g in range(len(res.populations) - 1):
        prev = set(res.populations[g])
        for m in res.populations[g + 1][1:]:
            assert any(bin(m ^ p).count("1") == 1 for p in prev)


def test_cache_measures_each_gene_once():
    table = W.random_time_table(6, seed=7)
    calls = []
    res = ga.run(_table_fn(table, calls), 6, pop=12, generations=12, pc=0.9, pm=0.05, seed=1)
    distinct = set(m for pg in res.populations for m in pg)
    assert len(calls) == len(set(calls)) == len(distinct) == res.evaluations
    assert res.evaluations + res.cache_hits == 12 * 12
    assert sum(h.evaluated for h in res.history) == res.evaluations


def test_failed_genes_never_best():
    table = W.random_time_table(6, seed=12, fail_frac=0.4)
    res = ga.run(_table_fn(table), 6, pop=12, generations=10, pc=0.9, pm=0.05, seed=4)
    assert table[res.best_mask] > 0
    for h in res.history:
        assert h.best_s > 0


@pytest.mark.parametrize("seed", list(range(10)))
def test_ga_finds_exhaustive_optimum_6bit(seed):
    """Six-loop programs have 2^6 genes; the brute-force search over all of them (the
    exhaustive prior art, Sec. 2) gives the optimum the GA must reach.  The table has a
    loop program's structure: per-loop CPU and GPU times plus a transfer cost at
    every change of side."""
    table = W.loop_time_table(6, seed=100 + seed)
    best_m, best_t = ga.exhaustive(_table_fn(table), 6)
    res = ga.run(_table_fn(table), 6, pop=12, generations=20, pc=0.9, pm=0.05, seed=seed)
    assert res.best_mask == best_m and res.best_s == best_t


def test_onemax_converges():
    a = 12
    times = np.array([(a + 1 - bin(m).count("1")) ** 2 for m in range(1 << a)], dtype=np.float64)
    res = ga.run(_table_fn(times), a, pop=20, generations=60, pc=0.9, pm=0.05, seed=21)
    assert res.best_mask == (1 << a) - 1
    assert res.history[-1].mean_s < res.history[0].mean_s


def test_seeded_run_reproducible():
    table = W.random_time_table(12, seed=9)
    r1 = ga.run(_table_fn(table), 12, 12, 12, 0.9, 0.05, seed=99)
    r2 = ga.run(_table_fn(table), 12, 12, 12, 0.9, 0.05, seed=99)
    assert r1.populations == r2.populations and r1.best_mask == r2.best_mask
    r3 = ga.run(_table_fn(table), 12, 12, 12, 0.9, 0.05, seed=100)
    assert r3.populations != r1.populations
