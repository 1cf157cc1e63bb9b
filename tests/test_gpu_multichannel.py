"""Multichannel generation in one persistent launch, CUDA-graph replay and the autotuner.

The six 2->5 channels of mixed topology with uneven event counts run in a single launch of the
map kernel; the CUDA-graph executor replays that launch with new seeds and offsets and must
reproduce ps_generate bit for bit; the autotuner returns a configuration that is valid and at
least as fast as the default."""
import numpy as np
import pytest

from paper_2602_06895_gb300 import ps
from paper_2602_06895_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2602_06895_gb300 import build

    build.build()
    return torch


def test_exec_replay_matches_generate(torch_cuda):
    chans = W.multichannel_2to5()
    counts = [1000, 40_000, 40_000, 40_000, 40_000, 39_000]
    prog = ps.program_for(chans)
    ref, ws_ref = prog.alloc(counts, 7, alpha=True)
    out, ws = prog.alloc(counts, 7, alpha=True)
    ex = prog.exec_create(counts, out, ws)
    for seed, off in [(1003, 0), (1003, 200_000), (42, 7)]:
        launches = ps.launch_count()
        ex.launch(seed, off)
        assert ps.launch_count() - launches == 2
        ex_stats = prog.stats()
        prog.generate(counts, seed, ref, ws_ref, event_offset=off)
        ref_stats = prog.stats()
        torch_cuda.cuda.synchronize()
        for k in ref:
            assert torch_cuda.equal(out[k], ref[k]), (seed, off, k)
        for a, b in zip(ex_stats, ref_stats):
            assert a == b


def test_single_launch_for_all_channels(torch_cuda):
    chans = W.multichannel_2to5()
    counts = [100_000, 400_000, 400_000, 400_000, 400_000, 390_000]
    prog = ps.program_for(chans)
    out, ws = prog.alloc(counts, 7, alpha=True)
    before = ps.launch_count()
    prog.generate(counts, 1003, out, ws)
    torch_cuda.cuda.synchronize()
    assert ps.launch_count() - before == 2  # one map launch for all six channels + one reduction
    st = prog.stats()
    assert [s["n"] for s in st] == counts
    assert all(s["n_nonzero"] > 0.99 * s["n"] for s in st)


def test_autotune_returns_valid_choice(torch_cuda):
    chans = W.multichannel_2to5()
    counts = [10_000, 100_000, 100_000, 100_000, 100_000, 90_000]
    best, table = ps.autotune(chans, counts, blocks=(64, 128), ctas=(2, 3), reps=2)
    assert best["block_threads"] in (64, 128) and best["ctas_per_sm"] in (2, 3)
    assert len(table) >= 2
    assert min(t["ms"] for t in table) == next(t["ms"] for t in table if
                                               t["block_threads"] == best["block_threads"] and
                                               t["ctas_per_sm"] == best["ctas_per_sm"])


def test_programs_with_different_slot_files_coexist(torch_cuda):
    """A program created after another one with a larger shared-memory slot file must not lower
    the kernel's dynamic shared-memory limit below what the first one launches with."""
    torch = torch_cuda
    big = ps.program_for(W.multichannel_2to5(), block_threads=128)
    small = ps.program_for([W.two_body_fixed()], block_threads=64)
    n = [0, 1000, 0, 0, 0, 0]
    out, ws = big.alloc(n, 7, alpha=True)
    big.generate(n, 3, out, ws)
    o2, w2 = small.alloc([1000], 4, x=False)
    small.generate([1000], 3, o2, w2)
    torch.cuda.synchronize()
    assert big.stats()[1]["n"] == 1000 and small.stats()[0]["n"] == 1000


def test_stats_accumulate_adds_launches_in_order(torch_cuda):
    """Streaming statistics: generate and CUDA-graph launches add their per-channel sums, in stream
    order, to the running totals; turning the mode off restores per-launch statistics."""
    chans = W.multichannel_2to5()
    counts = [1000, 5000, 0, 3000, 2000, 777]
    prog = ps.program_for(chans)
    out, ws = prog.alloc(counts, 7, alpha=True)
    per = []
    for k in range(3):
        prog.generate(counts, 11, out, ws, event_offset=k * 10_000)
        per.append(prog.stats())
    prog.stats_accumulate(True)
    ex = prog.exec_create(counts, out, ws)
    for k in range(3):
        if k == 1:
            ex.launch(11, k * 10_000)
        else:
            prog.generate(counts, 11, out, ws, event_offset=k * 10_000)
    acc = prog.stats()
    prog.stats_accumulate(False)
    for c in range(len(chans)):
        for key in ("n", "n_nonzero", "sum_w", "sum_w2"):
            expect = 0.0
            for k in range(3):
                expect += per[k][c][key]
            assert acc[c][key] == expect, (c, key)
        assert acc[c]["max_w"] == max(per[k][c]["max_w"] for k in range(3))
    prog.generate(counts, 11, out, ws, event_offset=0)
    assert prog.stats() == per[0]
