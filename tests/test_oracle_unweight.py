"""Pins of the unweighting oracle (oracle/unweight.py): closed forms on small inputs, the defining
property of w_max (excess at w_max equals eps S, the excess just below is larger) against brute
force, the special cases eps = 0 (w_max = max w) and eps >= 1 (w_max = 0), and unbiasedness of
the accepted weights (their sum estimates sum w)."""
import numpy as np
import pytest

import oracle as O
from oracle import unweight as U


def test_closed_forms():
    assert U.max_weight([1.0, 1.0, 1.0, 1.0], 0.0) == 1.0
    # excess(t) = 4 (1 - t) = 0.25 * 4  ->  t = 0.75
    assert U.max_weight([1.0, 1.0, 1.0, 1.0], 0.25) == pytest.approx(0.75, rel=1e-15)
    # one big weight: excess(t) = 10 - t for t in [1, 10]; S = 13; eps = 0.1 -> t = 8.7
    assert U.max_weight([10.0, 1.0, 1.0, 1.0], 0.1) == pytest.approx(8.7, rel=1e-15)
    # eps large enough to reach the second weight: 10 + 4 - 2 t = 0.5 * 15 -> t = 3.25
    assert U.max_weight([10.0, 4.0, 1.0], 0.5) == pytest.approx(3.25, rel=1e-15)
    assert U.max_weight([0.0, 0.0], 0.001) == 0.0
    assert U.max_weight([], 0.001) == 0.0
    assert U.max_weight([2.0, 3.0], 1.0) == 0.0


@pytest.mark.parametrize("seed", range(6))
def test_defining_property_against_brute_force(seed):
    g = np.random.default_rng(seed)
    n = int(g.integers(1, 400))
    w = g.lognormal(0.0, 1.5, n) * (g.random(n) < 0.9)
    w[g.integers(0, n, 3)] = w.max()  # ties at the top
    for eps in (0.0, 1e-3, 0.01, 0.2):
        t = U.max_weight(w, eps)
        S = w.sum()
        assert U.excess(w, t) <= eps * S * (1 + 1e-12) + 1e-300
        if t > 0:
            below = np.nextafter(t, 0.0) * (1 - 1e-9)
            assert U.excess(w, below) > eps * S
        # brute force: the root lies on a segment between consecutive sorted weights
        cand = np.concatenate([[0.0], np.sort(w)])
        ex = np.array([U.excess(w, c) for c in cand])
        j = np.nonzero(ex <= eps * S * (1 + 1e-12))[0][0]
        assert (cand[j - 1] if j > 0 else 0.0) <= t * (1 + 1e-12) and t <= cand[j] * (1 + 1e-12)


def test_eps_zero_is_max():
    w = np.random.default_rng(3).random(1000)
    assert U.max_weight(w, 0.0) == w.max()


def test_rejects_negative():
    with pytest.raises(ValueError):
        U.max_weight([1.0, -1.0], 0.1)


def test_uniforms_are_the_generator_point():
    u = U.uniforms(99, 5, 3)
    for b in range(3):
        ev = 5 + b
        o = O.philox([ev & 0xFFFFFFFF, ev >> 32, U.UNWEIGHT_STREAM, 0], [99, 0])
        bits = (o[1] << 32) | o[0]
        assert u[b] == ((bits >> 12) + 0.5) * 2.0 ** -52


def test_accepted_weights_are_unbiased():
    g = np.random.default_rng(7)
    n = 200_000
    w = g.lognormal(0.0, 1.0, n)
    t = U.max_weight(w, 1e-3)
    idx, wa = U.accept(w, t, seed=11)
    assert np.all(np.diff(idx) > 0) and np.all(wa >= t)
    # sum of accepted weights estimates sum w; var per event = w max(w, t) - w^2
    var = np.sum(w * np.maximum(w, t) - w * w)
    assert abs(wa.sum() - w.sum()) <= 5 * np.sqrt(var)
    # the over-weight events carry the allowed share of the cross section
    assert np.sum(np.maximum(w - t, 0)) == pytest.approx(1e-3 * w.sum(), rel=1e-9)
