"""Oracle pins for the VEGAS grid (Lepage 1978; adapted then frozen, Sec. 4.2):
identity grid, monotone piecewise-linear map with the bin-width Jacobian,
inverse, rebinning invariants, and an end-to-end check that adaptation lowers
the variance of an unbiased estimate."""
import math

import numpy as np

from paper_2602_06895_gb300 import workloads as W


def test_identity_grid(oracle_mod):
    e = W.vegas_grid_uniform(1, 64)[0]
    for r in W.uniform_r(1, 1000, 1)[:, 0]:
        v, j = oracle_mod.vegas_map(r, e)
        assert abs(v - r) <= 2.3e-16 and j == 1.0


def test_random_grid_map_jacobian_inverse(oracle_mod):
    e = W.vegas_grid_random(5, 1, 64)[0]
    r = np.sort(W.uniform_r(2, 2000, 1)[:, 0])
    vals = [oracle_mod.vegas_map(x, e) for x in r]
    v = np.array([a for a, _ in vals])
    j = np.array([b for _, b in vals])
    assert np.all(np.diff(v) >= 0)
    k = np.minimum((r * 64).astype(int), 63)
    assert np.allclose(j, 64 * (e[k + 1] - e[k]), rtol=1e-15, atol=0)
    back = np.array([oracle_mod.vegas_inv(x, e) for x in v])
    assert np.max(np.abs(back - r)) < 1e-15
    # the Jacobian integrates to one (each bin: width 1/N in r times N (e_{k+1}-e_k))
    mids = (np.arange(64) + 0.5) / 64
    assert abs(sum(oracle_mod.vegas_map(x, e)[1] for x in mids) / 64 - 1.0) < 1e-14


def test_rebin_invariants(oracle_mod):
    e = W.vegas_grid_uniform(1, 16)
    flat = oracle_mod.vegas_rebin(np.ones((1, 16)), e)
    assert np.max(np.abs(flat - e)) < 1e-15
    h = np.zeros((1, 16))
    h[0, 5] = 3.0
    new = oracle_mod.vegas_rebin(h, e)[0]
    assert new[0] == 0.0 and new[-1] == 1.0 and np.all(np.diff(new) > 0)
    # smoothing spreads bin 5 to bins 4..6; every interior edge lies inside them
    assert np.all(new[1:-1] >= e[0, 4]) and np.all(new[1:-1] <= e[0, 7])
    # zero histogram leaves the grid alone
    assert np.array_equal(oracle_mod.vegas_rebin(np.zeros((1, 16)), e), e)


def test_adaptation_reduces_variance(oracle_mod):
    """1-D integrand f(x) = exp(-(x-0.3)^2/(2 0.02^2)) + 0.01; VEGAS iterations keep the
    estimate unbiased and cut its variance by a large factor."""
    f = lambda x: np.exp(-((x - 0.3) ** 2) / (2 * 0.02 ** 2)) + 0.01
    exact = 0.02 * math.sqrt(2 * math.pi) * 0.5 * (math.erf(0.7 / (0.02 * math.sqrt(2))) +
                                                 math.erf(0.3 / (0.02 * math.sqrt(2)))) + 0.01
    e = W.vegas_grid_uniform(1, 64)
    var0 = None
    for it in range(8):
        r = W.uniform_r(40 + it, 20_000, 1)
        xs, js = zip(*[oracle_mod.vegas_map(x, e[0]) for x in r[:, 0]])
        w = f(np.array(xs)) * np.array(js)
        if var0 is None:
            var0 = w.var()
        hist = oracle_mod.vegas_accumulate(r, w, 1, 64)
        e = oracle_mod.vegas_rebin(hist, e)
    r = W.uniform_r(99, 200_000, 1)
    xs, js = zip(*[oracle_mod.vegas_map(x, e[0]) for x in r[:, 0]])
    w = f(np.array(xs)) * np.array(js)
    assert abs(w.mean() - exact) < 4.5 * w.std() / math.sqrt(w.size)
    assert w.var() < var0 / 20


def test_accumulate_counts_bins(oracle_mod):
    r = np.array([[0.01, 0.99], [0.02, 0.5], [0.99, 0.51]])
    w = np.array([1.0, 2.0, 3.0])
    h = oracle_mod.vegas_accumulate(r, w, 2, 4)
    assert np.array_equal(h[0], [5.0, 0.0, 0.0, 9.0])
    assert np.array_equal(h[1], [0.0, 0.0, 13.0, 1.0])
