"""One GA search shared by several processes (one GPU each).

Genes are independent to measure, so the search shards by gene: every process runs
the same seeded Simple GA (identical populations, since the draws do not depend on
the times until the times are known), and in each generation process r measures the
new genes at positions r, r + world, ... of the generation's list; the times are
exchanged with one all-gather, and every process continues with the same table.  The
result equals a single-process run on the same times.  A process that fails (its
measurement raises) stops its own GA; the others see the failure as an error from
the all-gather (the process group's timeout), not as a hang.
"""
from __future__ import annotations

from typing import Callable, Dict, Optional, Sequence

from . import GaoError, GAResult, STATUS_NAMES, ga_run_callback, prog_run_status, GAO_OK, GAO_ETIMEOUT


def sharded_ga_run(measure: Callable[[int], float], n_genes: int, pop: int = 12, generations: int = 12,
                   pc: float = 0.9, pm: float = 0.05, seed: int = 0, elite: int = 1, mutation: int = 0,
                   group=None, counts: Optional[Dict[str, int]] = None) -> GAResult:
    """``measure(gene) -> seconds`` measures one gene on this process's GPU."""
    import torch.distributed as dist

    world = dist.get_world_size(group)
    rank = dist.get_rank(group)

    def evaluate(genes: Sequence[int]):
        mine = {}
        for j, g in enumerate(genes):
            if j % world == rank:
                mine[g] = float(measure(g))
                if counts is not None:
                    counts["measured"] = counts.get("measured", 0) + 1
        parts = [None] * world
        dist.all_gather_object(parts, mine, group=group)
        merged = {}
        for d in parts:
            merged.update(d)
        return [merged[g] for g in genes]

    return ga_run_callback(evaluate, n_genes, pop=pop, generations=generations, pc=pc, pm=pm, seed=seed,
                           elite=elite, mutation=mutation)


def program_measure(progs, budget_s: float = 0.0) -> Callable[[int], float]:
    """Time of a gene over programs on this process's GPU: the sum of prog_run wall
    times; a timed-out run counts as its budget, a failed run as -1 (fitness 0)."""

    def measure(gene: int) -> float:
        total = 0.0
        for p in progs:
            st, s = prog_run_status(p, gene)
            if st == GAO_ETIMEOUT:
                s = budget_s
            elif st != GAO_OK:
                if STATUS_NAMES[st] in ("EINVAL", "ENODEV", "ENOMEM", "ECUDA"):
                    raise GaoError(st, "prog_run")
                return -1.0
            total += s
        return total

    return measure
