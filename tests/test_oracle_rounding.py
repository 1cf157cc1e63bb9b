"""The oracle's rounding sensitivity: the condition numbers it reports and the stochastic-arithmetic
spread of the rounding-probe copy (oracle/rounding_probe.h) that the GPU parity tests use as
tolerances.  CPU only."""
import numpy as np

import oracle as O
from paper_2602_06895_gb300 import workloads as W

EPS = 2.0 ** -52


def _c5_event(which, ev):
    chans = W.channels_2to8()
    r = W.uniform_r(4242 + which, 4999, O.dims(chans[which]), edge_fraction=0.02)
    return chans, r


def test_probe_is_deterministic_and_small_when_well_conditioned():
    ch = W.two_body_fixed()
    r = W.uniform_r(5, 2000, O.dims(ch))
    a = O.rounding_spread(ch, r)
    b = O.rounding_spread(ch, r)
    for k in ("w", "alpha", "mom", "flip"):
        assert np.array_equal(a[k], b[k])
    # 2 -> 2 at fixed energy: the weight is a constant and the momenta come from one cos/sin pair,
    # so a 2-ulp move of an elementary function changes them by a few ulps at most
    assert a["mom"].max() > 0.0
    assert a["mom"].max() < 64 * EPS and a["w"].max() < 64 * EPS
    assert not a["flip"].any()


def test_t_range_width_enters_the_condition_number():
    """A light block with spacelike incoming legs: |t| ~ 1239 GeV^2 with a range only ~3e-9 wide,
    so both bounds' rounding (relative to |t|_max) is amplified by |t|_max/(|t|_max - |t|_min)
    ~ 4e11 in the Jacobian of the |t| map (Sec. 2.2.8, t range from the 2 -> 2 kinematics)."""
    chans, r = _c5_event(22, 3242)
    o = O.forward(chans[22], r[3242:3243], channels=chans, chan=22, aux=True)
    assert o["w"][0] > 0.0
    assert o["aux"][0, O.AUX["cond"]] > 1e11


def test_collapsed_t_range_is_undetermined():
    """A t range that rounds to zero width (upper == lower bound) gives w = 0 in one rounding and a
    tiny nonzero weight in another: the condition number is infinite there."""
    chans, r = _c5_event(6, 3117)
    o = O.forward(chans[6], r[3117:3118], channels=chans, chan=6, aux=True)
    assert o["w"][0] == 0.0 and o["aux"][0, O.AUX["cond"]] >= 1e300


def test_nested_sliver_ranges_compound_beyond_the_analytic_bound():
    """2 -> 8 channel with an s-channel invariant at the top of a range spanning ~11 decades (its
    map's exponent ~26 turns a libm ulp into ~20 ulps) feeding a sliver range of width 2.6e-3
    at 346^2 (kappa ~ 1e9), which feeds further light invariants: the spread of the weight
    under 2-ulp moves of the elementary functions exceeds 32 eps kappa, the analytic bound that
    assumes inputs good to an ulp -- which is why the parity tolerance takes the larger of the two."""
    chans, r = _c5_event(8, 1597)
    rr = r[1597:1598]
    o = O.forward(chans[8], rr, channels=chans, chan=8, aux=True)
    sp = O.rounding_spread(chans[8], rr, channels=chans, chan=8, base=o, runs=16)
    kappa = o["aux"][0, O.AUX["cond"]]
    assert 1e8 < kappa < 1e10
    assert sp["w"][0] > 32 * EPS * kappa
    assert sp["w"][0] < 1e-3
