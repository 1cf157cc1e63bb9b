"""Data-parallel generation across ranks (one process per GPU).

Events are independent and the generator is counter-based, so ranks take disjoint event ranges
and need no exchange while generating.  The one exchange is the combination of the per-channel
sums into the global estimate: sum of (n, nonzero, sum w, sum w^2) and max of max w.
"""
from __future__ import annotations


def step_offset(rank, world, events_per_rank, step):
    """Event id of the first event of `rank` in `step`: disjoint across ranks and steps."""
    return (step * world + rank) * events_per_rank


def combine_stats(stats, group=None, device=None):
    """All-reduce per-channel statistics (list of dicts from Program.stats()) over the process
    group: counts and sums add, max w takes the maximum.  Returns the combined list."""
    import torch
    import torch.distributed as dist

    keys = ("n", "n_nonzero", "sum_w", "sum_w2")
    sums = torch.tensor([[s[k] for k in keys] for s in stats], dtype=torch.float64, device=device)
    mx = torch.tensor([s["max_w"] for s in stats], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(sums, op=dist.ReduceOp.SUM, group=group)
        dist.all_reduce(mx, op=dist.ReduceOp.MAX, group=group)
    out = []
    for i in range(len(stats)):
        d = dict(zip(keys, sums[i].tolist()))
        d["max_w"] = float(mx[i])
        out.append(d)
    return out


def estimate(stats):
    """Integral estimate, its Monte Carlo error and the effective sample size from summed stats."""
    n = sum(s["n"] for s in stats)
    s1 = sum(s["sum_w"] for s in stats)
    s2 = sum(s["sum_w2"] for s in stats)
    mean = s1 / n
    var = max(s2 / n - mean * mean, 0.0)
    return {"integral": mean, "error": (var / n) ** 0.5, "ess": s1 * s1 / s2 if s2 > 0 else 0.0}
