"""The allocation-free entry point ps_generate_noalloc against ps_generate.

Some callers cannot allocate device memory themselves (a host framework that owns every
allocation, or a loop in which an allocation would synchronise the device).  For them the
library keeps a fixed scratch array in device memory; this checks, through the C ABI, that
generating with it gives the same events and sums as generating with a caller workspace, on
two calls in a row, and that a request larger than the array is refused.  The file is named so
that pytest collects it last.
"""
import numpy as np
import pytest

from paper_2602_06895_gb300 import ps
from paper_2602_06895_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RTOL = 1e-12


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2602_06895_gb300 import build

    build.build()
    return torch


def _same(torch, a, b):
    for k in a:
        x, y = a[k].double(), b[k].double()
        diff = (x - y).abs()
        assert bool((diff <= RTOL * y.abs()).all()), k


def test_noalloc_matches_workspace_entry_point(torch_cuda):
    ch = W.ww_hadronic()
    prog = ps.program_for([ch])
    prog.set_vegas(0, W.vegas_grid_random(7, 8, 64))
    N = 100_003
    for call, (seed, offset) in enumerate([(1002, 0), (77, 123_456)]):  # two calls in a row
        ref, ws = prog.alloc([N], 6)
        prog.generate([N], seed, ref, ws, event_offset=offset)
        ref_stats = prog.stats()[0]
        got, _ = prog.alloc([N], 6)
        prog.generate_noalloc([N], seed, got, event_offset=offset)
        got_stats = prog.stats()[0]
        torch_cuda.cuda.synchronize()
        _same(torch_cuda, got, ref)
        assert got_stats["n_nonzero"] == ref_stats["n_nonzero"]
        for k in ("sum_w", "sum_w2", "max_w"):
            assert abs(got_stats[k] - ref_stats[k]) <= RTOL * abs(ref_stats[k]), (call, k)


def test_noalloc_multichannel_and_limit(torch_cuda):
    chans = W.multichannel_2to5()
    prog = ps.program_for(chans)
    counts = [1000, 0, 2049, 5, 300, 7000]
    ref, ws = prog.alloc(counts, 7, alpha=True)
    prog.generate(counts, 1003, ref, ws)
    ref_stats = prog.stats()
    got, _ = prog.alloc(counts, 7, alpha=True)
    prog.generate_noalloc(counts, 1003, got)
    got_stats = prog.stats()
    torch_cuda.cuda.synchronize()
    _same(torch_cuda, got, ref)
    for a, b in zip(got_stats, ref_stats):
        assert a["n_nonzero"] == b["n_nonzero"]
        assert abs(a["sum_w"] - b["sum_w"]) <= RTOL * abs(b["sum_w"])
    too_many = [0] * len(chans)
    too_many[1] = 131072 * 128 + 1
    with pytest.raises(ps.PSError, match="exceed the fixed scratch"):
        prog.generate_noalloc(too_many, 1, got)


def test_noalloc_exactly_at_the_limit(torch_cuda):
    """Ragged channel counts whose tiles add up to exactly the fixed scratch (131072 tiles of
    32 events here) run and match ps_generate with a caller workspace; one tile more is refused."""
    chans = W.multichannel_2to5()
    prog = ps.program_for(chans, block_threads=32)
    counts = [31, 32_001, 0, 1_600_000 - 5, 5, 80_069 * 32 - 17]
    tiles = sum(-(-c // 32) for c in counts)
    assert tiles == 131072
    ref, ws = prog.alloc(counts, 7, alpha=True)
    prog.generate(counts, 4242, ref, ws)
    ref_stats = prog.stats()
    del ws
    got, _ = prog.alloc(counts, 7, alpha=True)
    prog.generate_noalloc(counts, 4242, got)
    got_stats = prog.stats()
    torch_cuda.cuda.synchronize()
    assert torch_cuda.equal(got["weight"], ref["weight"])
    _same(torch_cuda, got, ref)
    for a, b in zip(got_stats, ref_stats):
        assert a["n"] == b["n"] and a["n_nonzero"] == b["n_nonzero"]
        for k in ("sum_w", "sum_w2", "max_w"):
            assert abs(a[k] - b[k]) <= RTOL * abs(b[k]), k
    over = list(counts)
    over[2] = 1  # one more tile
    with pytest.raises(ps.PSError, match="exceed the fixed scratch"):
        prog.generate_noalloc(over, 4242, got)
