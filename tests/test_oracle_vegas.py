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


def _refine_by_interp(h, e, alpha):
    """The refinement rule restated with numpy: neighbour-mean importances, damped shares,
    and the inverse of the piecewise-linear cumulative by linear interpolation."""
    N = h.size
    pad = np.concatenate([[0.0], h, [0.0]])
    counts = np.full(N, 3.0)
    counts[0] = counts[-1] = 2.0
    if N == 1:
        counts[:] = 1.0
    s = (pad[:-2] + pad[1:-1] + pad[2:]) / counts
    d = s / s.sum()
    m = ((1.0 - d) / np.log(1.0 / d)) ** alpha
    cum = np.concatenate([[0.0], np.cumsum(m)])
    return np.interp(cum[-1] * np.arange(N + 1) / N, cum, e)


def _mass_per_new_bin(h, e, new, alpha):
    """Integral of the damped importance density (m_k spread evenly over old bin k) over
    each new bin, and the total."""
    N = h.size
    pad = np.concatenate([[0.0], h, [0.0]])
    counts = np.full(N, 3.0)
    counts[0] = counts[-1] = 2.0
    s = (pad[:-2] + pad[1:-1] + pad[2:]) / counts
    d = s / s.sum()
    m = np.zeros(N)
    pos = d > 0
    m[pos] = ((1.0 - d[pos]) / np.log(1.0 / d[pos])) ** alpha
    dens = m / np.diff(e)
    out = np.zeros(N)
    for j in range(N):
        a, b = new[j], new[j + 1]
        lo = np.clip(e[:-1], a, b)
        hi = np.clip(e[1:], a, b)
        out[j] = np.sum(dens * (hi - lo))
    return out, m.sum()


def test_rebin_matches_interpolated_cumulative(oracle_mod):
    """Random positive histograms on random grids, alpha 0.5 and 1.5: the oracle's new edges
    equal the numpy restatement (cumulative of the damped weights inverted by np.interp)."""
    rng = np.random.default_rng(17)
    for alpha in (0.5, 1.5):
        for trial in range(6):
            N = int(rng.choice([4, 16, 64]))
            e = W.vegas_grid_random(100 + trial, 1, N)
            h = rng.gamma(0.7, 1.0, size=(1, N)) * 10.0 ** rng.uniform(-3, 3)
            new = oracle_mod.vegas_rebin(h, e, alpha=alpha)[0]
            ref = _refine_by_interp(h[0], e[0], alpha)
            assert np.max(np.abs(new - ref)) <= 1e-13, (alpha, trial)


def test_rebin_equalises_damped_mass(oracle_mod):
    """The defining property of the refinement: every new bin holds 1/N of the damped
    importance, with zero-importance bins and fixed end points included."""
    rng = np.random.default_rng(23)
    for alpha in (0.5, 1.0, 1.5):
        for N in (3, 8, 64):
            e = W.vegas_grid_random(200 + N, 1, N)
            h = rng.exponential(1.0, size=(1, N))
            h[0, rng.random(N) < 0.3] = 0.0
            h[0, N // 2] = 1.0  # never all zero
            new = oracle_mod.vegas_rebin(h, e, alpha=alpha)[0]
            assert new[0] == e[0, 0] and new[-1] == e[0, -1]
            assert np.all(np.diff(new) >= 0)
            mass, tot = _mass_per_new_bin(h[0], e[0], new, alpha)
            assert np.max(np.abs(mass / (tot / N) - 1.0)) <= 1e-12, (alpha, N)


def test_rebin_hand_computed_four_bins(oracle_mod):
    """N = 4 on the uniform grid with h = (0, 0, 3, 3): the neighbour means are (0, 1, 2, 3),
    so d = (0, 1/6, 1/3, 1/2); at alpha = 1 the damped weights are m1 = (5/6)/ln 6,
    m2 = (2/3)/ln 3, m3 = (1/2)/ln 2 and m0 = 0.  Each new edge sits where the running sum
    of m reaches j/4 of the total, linearly inside its old bin of width 1/4."""
    e = W.vegas_grid_uniform(1, 4)
    new = oracle_mod.vegas_rebin(np.array([[0.0, 0.0, 3.0, 3.0]]), e, alpha=1.0)[0]
    m1, m2, m3 = (5 / 6) / math.log(6), (2 / 3) / math.log(3), 0.5 / math.log(2)
    q = (m1 + m2 + m3) / 4
    assert q < m1 < 2 * q < m1 + m2 < 3 * q < m1 + m2 + m3  # edge j lies in old bin j
    want = [0.0, 0.25 + 0.25 * q / m1, 0.5 + 0.25 * (2 * q - m1) / m2,
            0.75 + 0.25 * (3 * q - m1 - m2) / m3, 1.0]
    assert np.max(np.abs(new - np.array(want))) <= 1e-15
    # numerically: 0.4910, 0.6778, 0.8446
    assert np.allclose(new[1:4], [0.49098, 0.67778, 0.84463], atol=5e-5)
