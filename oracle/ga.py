"""Simple GA of the paper in plain Python (oracle; TEST INFRASTRUCTURE ONLY).

Steps in the paper's order (Sec. 3.3, Sec. 4; parameters Sec. 5.1.2):

1. Initialisation: M genes of length a, each bit 0 or 1 at random.
2. Evaluation: measure each gene's processing time t.  A gene measured before is
   not measured again; its earlier time is reused (Sec. 4).
3. Fitness: t^(-1/2) (Sec. 5.1.2); a gene whose run failed gets fitness 0.
4. Selection: roulette selection (probability proportional to fitness) plus
   elite preservation: the fittest gene of the generation goes to the next
   generation with neither crossover nor mutation (Sec. 5.1.2).
5. Crossover: with rate Pc, two selected individuals exchange the genes on one
   side of one cut point (one-point crossover); otherwise they are copied.
6. Mutation: each gene value flips 0<->1 with rate Pm (Sec. 3.3, Sec. 4).
7. Termination: after T generations the fittest gene found is the answer.

Readings where the paper is silent (each also listed in the design notes):
* T counts evaluated populations: generation 1 is the random population and
  T-1 reproduction steps follow.
* The next population is the elite plus M-1 children.  Children come in pairs
  from two roulette draws (with replacement); with an odd count the second child
  of the last pair is dropped.  The cut point is uniform in [1, a-1]; bits
  [0, cut) come from the first parent.
* Fitness is computed as 1/sqrt(t) (same value as t^(-1/2), correctly rounded
  on every platform).  Ties: the elite is the lowest index among the fittest;
  the answer is the lowest time, first found on ties.
* All draws come from one SplitMix64 stream (Steele, Lea & Flood 2014) in a
  fixed order, so that any implementation that draws in this order reproduces
  the run exactly: per initial gene one draw (its top a bits); per child pair
  roulette, roulette, crossover test, [cut point], then a mutation draw per bit
  of child 1 and of child 2.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional

MASK64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15


def _finalise(z: int) -> int:
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


class SplitMix64:
    """SplitMix64: state += gamma; output = finaliser(state)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64
        self.draws = 0

    def next(self) -> int:
        self.state = (self.state + GAMMA) & MASK64
        self.draws += 1
        return _finalise(self.state)

    def uniform(self) -> float:
        """U[0,1) with 53 random bits."""
        return (self.next() >> 11) * (1.0 / 9007199254740992.0)

    def below(self, n: int) -> int:
        """Integer in [0, n) by multiply-shift of the top 32 bits."""
        return ((self.next() >> 32) * n) >> 32


def fitness_of(t: float) -> float:
    """(processing time)^(-1/2); 0 for a failed gene (non-finite or negative time)."""
    if t is None or not math.isfinite(t) or t <= 0.0:
        return 0.0
    return 1.0 / math.sqrt(t)


def roulette(rng: SplitMix64, fitness: List[float]) -> int:
    total = 0.0
    for f in fitness:
        total += f
    if total <= 0.0:
        return rng.below(len(fitness))
    r = rng.uniform() * total
    acc = 0.0
    for i, f in enumerate(fitness):
        acc += f
        if r < acc:
            return i
    for i in range(len(fitness) - 1, -1, -1):
        if fitness[i] > 0.0:
            return i
    return len(fitness) - 1


@dataclass
class GenRecord:
    best_mask: int
    best_s: float
    mean_s: float
    evaluated: int
    cache_hits: int


@dataclass
class GAResult:
    best_mask: int
    best_s: float
    evaluations: int
    cache_hits: int
    history: List[GenRecord] = field(default_factory=list)
    populations: List[List[int]] = field(default_factory=list)
    stats: Dict[str, int] = field(default_factory=dict)


def run(time_of: Callable[[int], float], n_genes: int, pop: int, generations: int, pc: float, pm: float,
        seed: int, elite: bool = True, mutation: int = 0) -> GAResult:
    """Run the Simple GA.  ``time_of(mask)`` returns the measured time of a gene
    (non-finite or negative for a failed run)."""
    assert 1 <= n_genes <= 64 and pop >= 1 and generations >= 1
    rng = SplitMix64(seed)
    stats = {"pairs": 0, "crossovers": 0, "mutation_trials": 0, "flips": 0}
    population = [rng.next() >> (64 - n_genes) for _ in range(pop)]
    cache: Dict[int, float] = {}
    res = GAResult(best_mask=0, best_s=math.inf, evaluations=0, cache_hits=0, stats=stats)
    have_best = False
    for g in range(generations):
        times = []
        ev = hits = 0
        for m in population:
            if m in cache:
                hits += 1
            else:
                cache[m] = float(time_of(m))
                ev += 1
            times.append(cache[m])
        fit = [fitness_of(t) for t in times]
        res.evaluations += ev
        res.cache_hits += hits
        res.populations.append(list(population))
        ok_sum, ok_n = 0.0, 0
        for t, f in zip(times, fit):
            if f > 0.0:  # plain left-to-right sum (Python's sum() is compensated)
                ok_sum += t
                ok_n += 1
        gbest_i = -1
        for i, (t, f) in enumerate(zip(times, fit)):
            if f > 0.0 and (gbest_i < 0 or t < times[gbest_i]):
                gbest_i = i
            if f > 0.0 and (not have_best or t < res.best_s):
                res.best_mask, res.best_s, have_best = population[i], t, True
        res.history.append(GenRecord(
            best_mask=population[gbest_i] if gbest_i >= 0 else population[0],
            best_s=times[gbest_i] if gbest_i >= 0 else math.inf,
            mean_s=(ok_sum / ok_n) if ok_n else math.inf,
            evaluated=ev, cache_hits=hits))
        if g == generations - 1:
            break
        nxt: List[int] = []
        if elite:
            e = 0
            for i in range(1, pop):
                if fit[i] > fit[e]:
                    e = i
            nxt.append(population[e])
        while len(nxt) < pop:
            c1 = population[roulette(rng, fit)]
            c2 = population[roulette(rng, fit)]
            stats["pairs"] += 1
            if rng.uniform() < pc and n_genes >= 2:
                cut = 1 + rng.below(n_genes - 1)
                low = (1 << cut) - 1
                c1, c2 = (c1 & low) | (c2 & ~low & MASK64), (c2 & low) | (c1 & ~low & MASK64)
                stats["crossovers"] += 1
            c1 = _mutate(rng, c1, n_genes, pm, mutation, stats)
            c2 = _mutate(rng, c2, n_genes, pm, mutation, stats)
            nxt.append(c1)
            if len(nxt) < pop:
                nxt.append(c2)
        population = nxt
    if not have_best:
        res.best_mask, res.best_s = res.populations[0][0], math.inf
    return res


def _mutate(rng: SplitMix64, c: int, n_genes: int, pm: float, mode: int, stats) -> int:
    if mode == 0:
        for b in range(n_genes):
            stats["mutation_trials"] += 1
            if rng.uniform() < pm:
                c ^= 1 << b
                stats["flips"] += 1
    else:
        stats["mutation_trials"] += 1
        if rng.uniform() < pm:
            c ^= 1 << rng.below(n_genes)
            stats["flips"] += 1
    return c


def exhaustive(time_of: Callable[[int], float], n_genes: int):
    """Brute force over all 2^a genes (the exhaustive prior-art search, Sec. 2):
    returns (best mask, best time), lowest mask on ties."""
    best_m, best_t = -1, math.inf
    for m in range(1 << n_genes):
        t = float(time_of(m))
        if fitness_of(t) > 0.0 and t < best_t:
            best_m, best_t = m, t
    return best_m, best_t
