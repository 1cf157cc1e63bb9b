"""Oracle pins for whole maps: the closed-form massless n-body volume (Sec. 4.1)
for pure-t, mixed and pure-s topologies, a textbook Dalitz-area integral for a
massive 3-body final state, per-event Jacobians against finite-difference
determinants of the map, and the forward -> inverse round trip."""
import math

import numpy as np
import pytest
from scipy import integrate

from paper_2602_06895_gb300 import workloads as W


def massless_volume(n, e):
    return e ** (2 * n - 4) / (math.gamma(n) * math.gamma(n - 1) * math.pi ** (2 * n - 3) * 2 ** (4 * n - 5))


@pytest.mark.parametrize("n", [3, 4])
def test_massless_volume_mc(oracle_mod, n):
    for ch in W.volume_topologies(n):
        d = oracle_mod.dims(ch)
        assert d == 3 * n - 4
        r = W.uniform_r(7 + n, 400_000, d)
        w = oracle_mod.forward(ch, r)["w"]
        exact = massless_volume(n, 1000.0)
        err = w.std() / math.sqrt(w.size)
        assert abs(w.mean() - exact) < 4.5 * err, (ch["name"], w.mean() / exact, err / exact)
        assert err / exact < 3e-3


def test_massless_volume_quadrature_pure_s3(oracle_mod):
    """Pure-s n = 3: the weight depends on the one invariant only; 1-D Gauss-Legendre
    in r reproduces the closed form to near machine precision."""
    ch = W.volume_topologies(3)[2]
    t, wq = np.polynomial.legendre.leggauss(80)
    g = np.geomspace(1e-12, 0.5, 40)
    edges = np.unique(np.concatenate([[0.0, 1.0], g, 1.0 - g]))
    acc = 0.0
    for lo, hi in zip(edges[:-1], edges[1:]):
        rr = 0.5 * (hi - lo) * t + 0.5 * (hi + lo)
        r = np.full((rr.size, 5), 0.3)
        r[:, 0] = rr
        acc += 0.5 * (hi - lo) * np.dot(wq, oracle_mod.forward(ch, r)["w"])
    exact = massless_volume(3, 1000.0)
    assert abs(acc / exact - 1.0) < 1e-10


def dalitz_area(s, m1, m2, m3):
    def width(s12):
        r12 = math.sqrt(s12)
        e2 = (s12 - m1 ** 2 + m2 ** 2) / (2 * r12)
        e3 = (s - s12 - m3 ** 2) / (2 * r12)
        a2 = math.sqrt(max(e2 * e2 - m2 ** 2, 0.0))
        a3 = math.sqrt(max(e3 * e3 - m3 ** 2, 0.0))
        return (e2 + e3) ** 2 - (a2 - a3) ** 2 - ((e2 + e3) ** 2 - (a2 + a3) ** 2)
    lo, hi = (m1 + m2) ** 2, (math.sqrt(s) - m3) ** 2
    val, _ = integrate.quad(width, lo, hi, epsabs=0, epsrel=1e-12, limit=200)
    return val


def test_massive_three_body_volume(oracle_mod):
    """Phi_3 = (2 pi)^-5 pi^2/(4 s) x (Dalitz area), the textbook 3-body phase space."""
    masses = [173.0, 173.0, 0.0]
    s = 1000.0 ** 2
    exact = (2 * math.pi) ** -5 * math.pi ** 2 / (4 * s) * dalitz_area(s, *masses)
    for ch in W.volume_topologies(3):
        ch = W.with_masses(ch, masses)
        r = W.uniform_r(31, 400_000, 5)
        w = oracle_mod.forward(ch, r)["w"]
        err = w.std() / math.sqrt(w.size)
        assert abs(w.mean() - exact) < 4.5 * err, (ch["name"], w.mean() / exact)


def chart(mom, n, hadronic, x):
    """Chart coordinates: (x1, x2,) p_1..p_{n-2} 3-momenta, (cos theta, phi) of p_{n-1}."""
    y = []
    if hadronic:
        y += [x[0], x[1]]
    for i in range(n - 2):
        y += list(mom[2 + i, 1:])
    p = mom[2 + n - 2, 1:]
    y += [p[2] / np.linalg.norm(p), math.atan2(p[1], p[0])]
    return np.array(y)


def density(mom, n):
    """(2 pi)^(4-3n) prod_{i<n-1} 1/(2E_i) |p_{n-1}|^2/(2E_{n-1}) 1/(2E_n) / |d(sum E)/d|p_{n-1}||."""
    E = mom[2:, 0]
    pv = mom[2 + n - 2, 1:]
    a = np.linalg.norm(pv)
    nh = pv / a
    dE = a / E[n - 2] - np.dot(mom[2 + n - 1, 1:], nh) / E[n - 1]
    rho = (2 * math.pi) ** (4 - 3 * n) * np.prod(1.0 / (2 * E[: n - 2])) * a * a / (2 * E[n - 2]) / (2 * E[n - 1])
    return rho / abs(dE)


def fd_jacobian(oracle_mod, ch, r0, h=1e-5):
    d = r0.size
    n = ch["n"]

    def y_of(rr):
        o = oracle_mod.forward(ch, rr)
        return np.array([chart(o["mom"][k], n, ch["hadronic"], o["x"][k]) for k in range(rr.shape[0])])

    rows = []
    for hh in (h, h / 2):
        pts = np.repeat(r0[None, :], 2 * d, axis=0)
        for j in range(d):
            pts[2 * j, j] += hh
            pts[2 * j + 1, j] -= hh
        y = y_of(pts)
        rows.append(np.array([(y[2 * j] - y[2 * j + 1]) / (2 * hh) for j in range(d)]).T)
    Jm = (4 * rows[1] - rows[0]) / 3  # Richardson
    return abs(np.linalg.det(Jm))


@pytest.mark.parametrize("which", ["pure_t_4", "mixed_4", "pure_s_4", "pure_t_3", "massive_mixed_4", "hadronic_ww"])
def test_jacobian_against_finite_differences(oracle_mod, which):
    if which == "hadronic_ww":
        ch = W.ww_hadronic(vegas_dims=0)
        ch["integrand"] = "none"
    elif which == "massive_mixed_4":
        ch = W.with_masses(W.volume_topologies(4)[1], [173.0, 173.0, 0.0, 0.0])
    else:
        ch = {t["name"]: t for t in W.volume_topologies(3) + W.volume_topologies(4)}[which]
    d = oracle_mod.dims(ch)
    rng = np.random.default_rng(17)
    checked = 0
    for _ in range(12):
        r0 = 0.1 + 0.8 * rng.random(d)
        if ch["hadronic"]:
            # moderate shat and boost, so that finite differences of the lab momenta stay accurate
            r0[0] = 0.8 + 0.15 * rng.random()
            r0[3] = 0.3 + 0.4 * rng.random()
        o = oracle_mod.forward(ch, r0[None, :], aux=True)
        mom = o["mom"][0]
        p = mom[2 + ch["n"] - 2, 1:]
        if abs(math.atan2(p[1], p[0])) > 3.0:
            continue  # keep the phi chart away from its branch cut
        w = o["aux"][0, oracle_mod.AUX["w_ps"]]
        det = fd_jacobian(oracle_mod, ch, r0)
        assert abs(density(mom, ch["n"]) * det / w - 1.0) < 2e-6, which
        checked += 1
    assert checked >= 6


def round_trip(oracle_mod, ch, B, seed, grid=None, channels=None, chan=0):
    d = oracle_mod.dims(ch)
    r = W.uniform_r(seed, B, d)
    o = oracle_mod.forward(ch, r, grid=grid, channels=channels, chan=chan)
    ok = o["w"] != 0
    ri = oracle_mod.inverse(ch, o["mom"], o["x"], grid=grid)
    dev = np.abs(ri - r)
    dev = np.minimum(dev, 1.0 - dev)  # azimuths are periodic
    return dev[ok]


@pytest.mark.parametrize("n", [3, 4])
def test_round_trip_fixed_energy(oracle_mod, n):
    for ch in W.volume_topologies(n) + [W.with_masses(t, [173.0, 173.0] + [0.0] * (n - 2))
                                         for t in W.volume_topologies(n)]:
        dev = round_trip(oracle_mod, ch, 50_000, 3)
        assert np.median(dev) < 1e-15
        assert (dev < 1e-12).mean() > 0.999, ch["name"]
        assert (dev < 1e-9).mean() > 0.99999


def test_round_trip_hadronic(oracle_mod):
    """Partonic-frame round trip: most deviations at machine precision, with a tail
    from invariants recovered from nearly collinear momenta and narrow resonances."""
    c2 = W.ww_hadronic()
    c2["partonic"] = True
    grid = W.vegas_grid_random(3, 8, 64)
    dev = round_trip(oracle_mod, c2, 50_000, 5, grid=grid)
    assert np.median(dev) < 1e-15 and (dev < 1e-12).mean() > 0.99 and (dev < 1e-9).mean() > 0.9999
    chans = W.multichannel_2to5()
    for i, ch in enumerate(chans):
        ch = dict(ch)
        ch["partonic"] = True
        dev = round_trip(oracle_mod, ch, 20_000, 11 + i, channels=chans, chan=i)
        assert np.median(dev) < 1e-14 and (dev < 1e-12).mean() > 0.9 and (dev < 1e-8).mean() > 0.99, ch["name"]
