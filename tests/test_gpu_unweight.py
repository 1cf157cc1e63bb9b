"""GPU parity of the unweighting (Sec. "Unweighting and file output") against the oracle
(oracle/unweight.py), through the C ABI.

  w_max     relative 1e-12 against the oracle's closed form (both are (A - eps S)/K over the same
            set of weights; only the summation order differs), and the defining property checked
            with the oracle's sums
  sums      relative 1e-12; counts (over-weight events, invalid weights) exact
  accepted  indices and weights bit-exact against the oracle's decisions taken with the GPU's
            w_max (the decision u w_max < w is unique once w_max is fixed)
"""
import numpy as np
import pytest

from oracle import unweight as U
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


def weights(seed, n):
    g = np.random.default_rng(seed)
    w = g.lognormal(0.0, 1.3, n) * (g.random(n) < 0.85)
    if n > 10:
        w[g.integers(0, n, 5)] = w.max()  # ties at the top
    return w


def run(torch, w, eps, seed=5, offset=0):
    uw = ps.Unweighter(max(len(w), 1))
    wd = torch.tensor(w, dtype=torch.float64, device="cuda")
    uw.max_weight(wd, eps)
    idx = torch.empty(max(len(w), 1), dtype=torch.int64, device="cuda")
    wo = torch.empty(max(len(w), 1), dtype=torch.float64, device="cuda")
    uw.select(wd, seed, idx, wo, event_offset=offset)
    torch.cuda.synchronize()
    res = uw.result.cpu().numpy()
    na = int(uw.n_accepted.item())
    return res, idx[:na].cpu().numpy(), wo[:na].cpu().numpy()


@pytest.mark.parametrize("n", [1, 2, 100, 4099, 300_001])
@pytest.mark.parametrize("eps", [0.0, 1e-3, 0.05])
def test_max_weight_and_selection_match_oracle(torch_cuda, n, eps):
    w = weights(n, n)
    res, idx, wo = run(torch_cuda, w, eps, seed=n, offset=17)
    t_o = U.max_weight(w, eps)
    t = res[0]
    assert t == pytest.approx(t_o, rel=1e-12, abs=1e-300), (t, t_o)
    assert res[1] == pytest.approx(w.sum(), rel=1e-12)
    assert res[2] == w.max()
    assert res[3] == np.count_nonzero(w > t)
    assert res[4] == 0
    S = w.sum()
    assert U.excess(w, t) <= eps * S * (1 + 1e-10) + 1e-300
    i_o, w_o = U.accept(w, t, seed=n, ev0=17)
    assert np.array_equal(idx, i_o)
    assert np.array_equal(wo, w_o)


def test_degenerate_inputs(torch_cuda):
    torch = torch_cuda
    res, idx, _ = run(torch, np.zeros(1000), 1e-3)
    assert res[0] == 0.0 and len(idx) == 0
    res, idx, wo = run(torch, np.full(777, 2.5), 0.0)
    assert res[0] == 2.5 and len(idx) == 777 and np.all(wo == 2.5)
    res, idx, _ = run(torch, np.array([3.0, 1.0]), 1.5)  # eps >= 1: everything over-weight
    assert res[0] == 0.0 and list(idx) == [0, 1]
    uw = ps.Unweighter(1)
    e = torch.empty(0, dtype=torch.float64, device="cuda")
    uw.max_weight(e, 1e-3)
    uw.select(e, 1, torch.empty(1, dtype=torch.int64, device="cuda"), torch.empty(1, dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    assert uw.result[0].item() == 0.0 and uw.n_accepted.item() == 0


def test_invalid_weights_are_counted_and_skipped(torch_cuda):
    w = weights(3, 5000)
    bad = w.copy()
    bad[[3, 10, 4000]] = [-1.0, np.nan, np.inf]
    res, idx, _ = run(torch_cuda, bad, 1e-3, seed=9)
    keep = np.ones(len(w), bool)
    keep[[3, 10, 4000]] = False
    clean = np.where(keep, bad, 0.0)
    assert res[4] == 3
    assert res[0] == pytest.approx(U.max_weight(clean, 1e-3), rel=1e-12)
    assert not set([3, 10, 4000]) & set(idx.tolist())


def test_reproducible(torch_cuda):
    w = weights(4, 1_000_003)
    a = run(torch_cuda, w, 1e-3)
    b = run(torch_cuda, w, 1e-3)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_full_size_generated_weights(torch_cuda):
    """C2's weights at the benchmark size (1e7 events): w_max and the accepted set against the
    oracle, with the unweighted sum within its statistical error of sum w."""
    torch = torch_cuda
    ch = W.ww_hadronic()
    prog = ps.program_for([ch])
    N = 10_000_000
    out, ws = prog.alloc([N], 6)
    prog.generate([N], 1002, out, ws)
    uw = ps.Unweighter(N)
    uw.max_weight(out["weight"], 1e-3)
    idx = torch.empty(N, dtype=torch.int64, device="cuda")
    wo = torch.empty(N, dtype=torch.float64, device="cuda")
    uw.select(out["weight"], 77, idx, wo)
    torch.cuda.synchronize()
    w = out["weight"].cpu().numpy()
    t = uw.result[0].item()
    assert t == pytest.approx(U.max_weight(w, 1e-3), rel=1e-12)
    na = int(uw.n_accepted.item())
    i_o, w_o = U.accept(w, t, seed=77)
    assert na == len(i_o)
    assert np.array_equal(idx[:na].cpu().numpy(), i_o) and np.array_equal(wo[:na].cpu().numpy(), w_o)
    var = np.sum(w * np.maximum(w, t) - w * w)
    assert abs(w_o.sum() - w.sum()) <= 5 * np.sqrt(var)
