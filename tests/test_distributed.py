"""Multi-process paths on the CPU (gloo, world size 2): the sharded GA gives exactly the
single-process result with each rank measuring its share, a failing rank ends the other
rank's search with an error instead of a hang, and bench.py's cross-rank reductions."""
import datetime
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, mode, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    try:
        import torch.distributed as dist
        dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=8))
        import workloads as W
        from paper_1806_01430_gb300 import _build
        _build.build()
        import paper_1806_01430_gb300 as gao
        from paper_1806_01430_gb300 import parallel
        table = W.loop_time_table(8, seed=5)
        if mode == "ga":
            counts = {}
            res = parallel.sharded_ga_run(lambda g: float(table[g]), 8, pop=12, generations=10, seed=3,
                                          counts=counts)
            q.put((rank, "ok", res.populations, res.best_mask, res.best_s, res.evaluations, counts.get("measured", 0)))
        elif mode == "fail":
            calls = [0]

            def measure(g):
                calls[0] += 1
                if rank == 1 and calls[0] == 3:
                    raise RuntimeError("injected failure of rank 1")
                return float(table[g])
            try:
                parallel.sharded_ga_run(measure, 8, pop=12, generations=10, seed=3)
                q.put((rank, "finished"))
            except Exception as e:  # noqa: BLE001
                q.put((rank, "error", type(e).__name__, str(e)[:200]))
        elif mode == "reduce":
            import bench
            q.put((rank, "ok", bench.allmax(world, float(rank + 1)), bench.allsum(world, float(rank + 1))))
        dist.destroy_process_group()
    except Exception as e:  # noqa: BLE001
        q.put((rank, "crash", repr(e)[:300]))


def _run(mode, world=2, timeout=90):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, mode, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(world):
        item = q.get(timeout=timeout)
        out[item[0]] = item[1:]
    for p in procs:
        p.join(timeout=30)
        if p.is_alive():
            p.kill()
    return out


def test_sharded_ga_equals_single_process():
    import workloads as W
    from paper_1806_01430_gb300 import _build
    _build.build()
    import paper_1806_01430_gb300 as gao
    out = _run("ga")
    table = W.loop_time_table(8, seed=5)
    ref = gao.ga_run_table(table, 8, pop=12, generations=10, seed=3)
    measured = 0
    for rank in (0, 1):
        status, pops, best_mask, best_s, evals, n_measured = out[rank]
        assert status == "ok"
        assert pops == ref.populations and best_mask == ref.best_mask and best_s == ref.best_s
        assert evals == ref.evaluations
        measured += n_measured
    assert measured == ref.evaluations  # every new gene measured exactly once, across the ranks
    assert abs(out[0][5] - out[1][5]) <= 10  # shares are balanced to within one gene per generation


def test_failing_rank_stops_the_other_without_hanging():
    out = _run("fail", timeout=120)
    assert out[1][0] == "error" and "GaoError" in out[1][1]
    assert out[0][0] == "error"  # the all-gather ends with an error (timeout / closed peer)


def test_bench_reductions_across_ranks():
    out = _run("reduce")
    for rank in (0, 1):
        assert out[rank][0] == "ok"
        assert out[rank][1] == 2.0 and out[rank][2] == 3.0
