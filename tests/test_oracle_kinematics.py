"""Oracle pins for the two-particle blocks (Secs. 2.2.3, 2.2.4) and whole-event
kinematics: closed-form two-body phase space, the t-range from the literal
Eq. t_invariant_theta, t recovered from the constructed momenta, momentum
conservation and on-shell conditions (Sec. 4.1 acceptance criteria)."""
import math

import mpmath as mp
import numpy as np
import pytest

from paper_2602_06895_gb300 import workloads as W

mp.mp.dps = 40


def mdot(p, q):
    return p[..., 0] * q[..., 0] - p[..., 1] * q[..., 1] - p[..., 2] * q[..., 2] - p[..., 3] * q[..., 3]


def test_two_body_closed_form(oracle_mod):
    # (2 pi)^-2 * J integrated over the unit square = sqrt(lambda)/(8 pi s): J is constant
    for s0, m1, m2 in [(1e6, 0.0, 0.0), (1e6, 173.0, 173.0), (4e4, 80.4, 0.0), (1e4, 0.0, 91.2)]:
        lam = (s0 - m1 ** 2 - m2 ** 2) ** 2 - 4 * m1 ** 2 * m2 ** 2
        for rphi, rth in [(0.1, 0.2), (0.7, 0.999), (0.5, 1e-9)]:
            p1, p2, jac = oracle_mod.two_body_decay(rphi, rth, s0, m1, m2)
            assert abs(jac / (2 * math.pi) ** 2 - math.sqrt(lam) / (8 * math.pi * s0)) < 1e-15 * jac
            assert np.allclose(p1 + p2, [math.sqrt(s0), 0, 0, 0], rtol=0, atol=1e-12 * math.sqrt(s0))
            assert abs(mdot(p1, p1) - m1 ** 2) < 1e-12 * s0
            assert abs(mdot(p2, p2) - m2 ** 2) < 1e-12 * s0
            ct = p1[3] / np.linalg.norm(p1[1:])
            assert abs(ct - (2 * rth - 1)) < 1e-12
            ph = math.atan2(p1[2], p1[1]) % (2 * math.pi)
            assert abs(ph - 2 * math.pi * rphi) < 1e-12
    # boosted: conservation with the parent momentum
    p0 = np.array([500.0, 100.0, -50.0, 300.0])
    s0 = mdot(p0, p0)
    p1, p2, _ = oracle_mod.two_body_decay(0.3, 0.4, s0, 10.0, 20.0, p0)
    assert np.allclose(p1 + p2, p0, rtol=0, atol=1e-12 * 500)
    assert abs(mdot(p1, p1) - 100.0) < 1e-10 and abs(mdot(p2, p2) - 400.0) < 1e-10


def literal_t_range(s, mA2, mB2, m1, m2):
    s, mA2, mB2, m1, m2 = map(mp.mpf, (s, mA2, mB2, m1, m2))
    lam = lambda x, y, z: (x - y - z) ** 2 - 4 * y * z
    A = m1 ** 2 + mA2 - (s + m1 ** 2 - m2 ** 2) * (s + mA2 - mB2) / (2 * s)
    B = mp.sqrt(lam(s, m1 ** 2, m2 ** 2) * lam(s, mA2, mB2)) / (2 * s)
    return -(A + B), -(A - B)  # |t|_min, |t|_max


@pytest.mark.parametrize("args", [(1e6, 0.0, 0.0, 0.0, 0.0), (1e6, 0.0, 0.0, 0.0, 300.0),
                                  (1e6, 0.0, 0.0, 173.0, 173.0), (5e5, -2000.0, 0.0, 0.0, 200.0),
                                  (5e5, -2000.0, -30.0, 91.2, 10.0), (2e4, 0.0, 0.0, 80.4, 0.0)])
def test_t_range(oracle_mod, args):
    lo, hi = oracle_mod.t_min_max(*args)
    llo, lhi = literal_t_range(*args)
    assert abs(lo - float(llo)) <= 1e-13 * abs(float(lhi)) + 1e-300
    assert abs(hi - float(lhi)) <= 1e-14 * abs(float(lhi))
    if args[1] == 0.0 and args[2] == 0.0 and args[3] == 0.0:
        assert lo == 0.0  # massless leg next to a massless incoming leg


def test_two_to_two_reproduces_t(oracle_mod):
    rs = 1000.0
    pa = np.array([rs / 2, 0, 0, rs / 2])
    pb = np.array([rs / 2, 0, 0, -rs / 2])
    for m1, m2 in [(0.0, 0.0), (0.0, 400.0), (173.0, 173.0)]:
        lo, hi = oracle_mod.t_min_max(rs * rs, 0.0, 0.0, m1, m2)
        for f in [1e-9, 0.3, 0.77, 1 - 1e-9]:
            tabs = lo + f * (hi - lo)
            p1, p2, jac = oracle_mod.two_to_two(0.37, pa, pb, tabs, m1, m2, rs * rs, 0.0, 0.0)
            d = pa - p1
            assert abs(-mdot(d, d) - tabs) < 1e-12 * hi
            assert np.allclose(p1 + p2, pa + pb, rtol=0, atol=1e-12 * rs)
            assert abs(jac - 2 * math.pi / (4 * rs * rs)) < 1e-15 * jac
    # a spacelike incoming leg (as later in a t-chain)
    pA = np.array([300.0, 40.0, -10.0, 320.0])
    pB = np.array([400.0, -20.0, 30.0, -380.0])
    p0 = pA + pB
    s, mA2, mB2 = mdot(p0, p0), mdot(pA, pA), mdot(pB, pB)
    lo, hi = oracle_mod.t_min_max(s, mA2, mB2, 20.0, 50.0)
    tabs = 0.5 * (lo + hi)
    p1, p2, _ = oracle_mod.two_to_two(0.8, pA, pB, tabs, 20.0, 50.0, s, mA2, mB2)
    d = pA - p1
    assert abs(-mdot(d, d) - tabs) < 1e-10 * hi
    assert np.allclose(p1 + p2, p0, rtol=0, atol=1e-11 * p0[0])


def all_channels():
    chans = [W.two_body_fixed(), W.ww_hadronic(vegas_dims=0)]
    chans += W.volume_topologies(3) + W.volume_topologies(4)
    chans += [W.with_masses(t, [173.0, 173.0, 0.0, 0.0]) for t in W.volume_topologies(4)]
    return chans


@pytest.mark.parametrize("idx", range(9))
def test_conservation_and_on_shell(oracle_mod, idx):
    ch = all_channels()[idx]
    d = oracle_mod.dims(ch)
    r = W.uniform_r(100 + idx, 4000, d, edge_fraction=0.02)
    o = oracle_mod.forward(ch, r)
    mom = o["mom"]
    ok = o["w"] != 0
    assert ok.mean() > 0.99
    scale = mom[:, :2, 0].sum(axis=1)
    pin = mom[:, 0] + mom[:, 1]
    pout = mom[:, 2:].sum(axis=1)
    assert np.all(np.abs(pin - pout)[ok].max(axis=1) <= 1e-12 * scale[ok])
    masses = np.zeros(ch["n"])
    for nd in ch["nodes"]:
        if nd["kind"] == "leaf":
            masses[nd["leaf"]] = nd["mass"]
    m2 = mdot(mom[:, 2:], mom[:, 2:])
    assert np.all(np.abs(m2 - masses ** 2)[ok] <= 1e-12 * (scale[ok, None] ** 2))
    assert np.all(np.abs(mdot(mom[:, 0], mom[:, 0])[ok]) <= 1e-12 * scale[ok] ** 2)


def test_two_body_fixed_energy_constant_weight(oracle_mod):
    ch = W.two_body_fixed(integrand="none")
    r = W.uniform_r(1001, 100_000, 2)
    o = oracle_mod.forward(ch, r)
    assert np.all(np.abs(o["w"] * 8 * math.pi - 1.0) < 1e-15)
    ch = W.two_body_fixed()
    o = oracle_mod.forward(ch, r)
    w = o["w"]
    err = w.std() / math.sqrt(w.size)
    assert abs(w.mean() - 1.0 / (6 * math.pi)) < 4 * err
