"""The data-parallel path on CPU: two gloo ranks combine per-channel statistics, and the event
ranges of ranks and steps are disjoint (no GPU needed)."""
import os

import pytest
import torch.multiprocessing as mp

from paper_2602_06895_gb300 import distributed as D


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    stats = [{"n": 10.0 + rank, "n_nonzero": 9.0, "sum_w": 1.5 * (rank + 1), "sum_w2": 0.25 * (rank + 1),
              "max_w": 0.1 * (rank + 3)},
             {"n": 0.0, "n_nonzero": 0.0, "sum_w": 0.0, "sum_w2": 0.0, "max_w": 0.0}]
    out = D.combine_stats(stats)
    q.put((rank, out))
    dist.destroy_process_group()


def test_combine_stats_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        a, b = res[r]
        assert a["n"] == 21.0 and a["n_nonzero"] == 18.0
        assert a["sum_w"] == pytest.approx(4.5) and a["sum_w2"] == pytest.approx(0.75)
        assert a["max_w"] == pytest.approx(0.4)
        assert b == {"n": 0.0, "n_nonzero": 0.0, "sum_w": 0.0, "sum_w2": 0.0, "max_w": 0.0}
    est = D.estimate(res[0])
    assert est["integral"] == pytest.approx(4.5 / 21.0)


def test_event_ranges_are_disjoint():
    N, world, steps = 1000, 4, 5
    seen = set()
    for step in range(steps):
        for rank in range(world):
            o = D.step_offset(rank, world, N, step)
            rng = range(o, o + N)
            assert not seen.intersection((rng.start, rng.stop - 1))
            seen.update(range(o, o + N))
    assert len(seen) == N * world * steps
    assert min(seen) == 0 and max(seen) == N * world * steps - 1
