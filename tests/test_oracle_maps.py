"""Oracle pins for the analytic invariant maps (Sec. 2.2.1) and the PDF
convolution (Sec. 2.2.2): the paper's literal formulas evaluated at 50 digits
with mpmath, endpoint values, the Jacobian as the true derivative
(integral of J over r equals the interval length), special cases
(nu -> 0 flat, nu -> 1 continuity) and inverse round trips."""
import math

import mpmath as mp
import numpy as np
import pytest

mp.mp.dps = 50
A = 1e-4


def literal_nu(r, m, nu, xmin, xmax, a=A):
    m2 = mp.mpf(m) ** 2 if m > 0 else -mp.mpf(a)
    r, nu, xmin, xmax = mp.mpf(r), mp.mpf(nu), mp.mpf(xmin), mp.mpf(xmax)
    if nu == 1:
        x = mp.e ** (r * mp.log(xmax - m2) + (1 - r) * mp.log(xmin - m2)) + m2
        g = 1 / ((x - m2) * (mp.log(xmax - m2) - mp.log(xmin - m2)))
    else:
        x = (r * (xmax - m2) ** (1 - nu) + (1 - r) * (xmin - m2) ** (1 - nu)) ** (1 / (1 - nu)) + m2
        g = (1 - nu) / (((xmax - m2) ** (1 - nu) - (xmin - m2) ** (1 - nu)) * (x - m2) ** nu)
    return x, 1 / g


def literal_bw(r, M, G, xmin, xmax):
    M, G, r = mp.mpf(M), mp.mpf(G), mp.mpf(r)
    u1 = mp.atan((xmin - M * M) / (M * G))
    u2 = mp.atan((xmax - M * M) / (M * G))
    x = M * G * mp.tan(u1 + (u2 - u1) * r) + M * M
    g = M * G / ((u2 - u1) * ((x - M * M) ** 2 + M * M * G * G))
    return x, 1 / g


def rel(a, b):
    return abs(float((mp.mpf(a) - b) / b))


NU_CASES = [  # (m, nu, xmin, xmax)
    (0.0, 0.8, 0.0, 1.69e8), (0.0, 0.3, 0.0, 1e6), (0.0, 1.0, 0.0, 1.69e8), (173.0, 0.8, 4e4, 9e6),
    (0.0, 0.8, 10.0, 5e3), (0.0, 2.0, 1.0, 1e4), (0.0, 0.8, 100.0, 100.5),
]


@pytest.mark.parametrize("case", NU_CASES)
def test_power_law_matches_literal_formula(oracle_mod, case):
    m, nu, xmin, xmax = case
    for r in [1e-12, 1e-6, 0.013, 0.31, 0.5, 0.77, 0.999, 1 - 1e-9]:
        x, j, st = oracle_mod.map_nu(r, m, nu, xmin, xmax)
        xl, jl = literal_nu(r, m, nu, xmin, xmax)
        assert st == 0
        # a few ulp of x, plus relative precision of x - (anchoring endpoint): the stable form
        # keeps x - x_min exact for nu <= 1 and x_max - x for nu > 1
        m2 = m * m if m > 0 else -1e-4
        anchor = xmin if nu <= 1.0 else m2
        assert abs(float(x - xl)) <= 4e-16 * abs(x) + 1e-13 * float(abs(xl - anchor)) + 1e-300
        assert rel(j, jl) < 1e-13


@pytest.mark.parametrize("case", NU_CASES)
def test_power_law_endpoints_jacobian_inverse(oracle_mod, case):
    m, nu, xmin, xmax = case
    x0, _, _ = oracle_mod.map_nu(0.0, m, nu, xmin, xmax)
    x1, _, _ = oracle_mod.map_nu(1.0, m, nu, xmin, xmax)
    assert x0 == xmin
    assert abs(x1 - xmax) <= 1e-14 * xmax
    # Gauss-Legendre: integral of dx/dr over [0,1] = xmax - xmin (J is the true Jacobian)
    t, wq = np.polynomial.legendre.leggauss(200)
    acc = 0.0
    edges = np.linspace(0.0, 1.0, 41) ** 3  # graded towards r = 0 for the steep power laws
    for lo, hi in zip(edges[:-1], edges[1:]):
        rr = 0.5 * (hi - lo) * t + 0.5 * (hi + lo)
        acc += 0.5 * (hi - lo) * sum(w * oracle_mod.map_nu(r, m, nu, xmin, xmax)[1] for r, w in zip(rr, wq))
    assert abs(acc - (xmax - xmin)) < 1e-10 * (xmax - xmin)
    for r in [1e-9, 0.2, 0.5, 0.9, 1 - 1e-7]:
        x, j, _ = oracle_mod.map_nu(r, m, nu, xmin, xmax)
        assert abs(oracle_mod.inv_nu(x, m, nu, xmin, xmax) - r) < 1e-13 + 2.0 * np.spacing(x) / j


def test_power_law_special_cases(oracle_mod):
    # nu = 0 is the flat map of Eq. prop_flat
    for r in [0.1, 0.5, 0.9]:
        x, j, _ = oracle_mod.map_nu(r, 0.0, 0.0, 10.0, 30.0)
        assert abs(x - (10.0 + 20.0 * r)) < 1e-12 and abs(j - 20.0) < 1e-12
    # nu -> 1 limit is continuous
    for r in [0.1, 0.5, 0.9]:
        x1, j1, _ = oracle_mod.map_nu(r, 0.0, 1.0, 0.0, 1.69e8)
        xa, ja, _ = oracle_mod.map_nu(r, 0.0, 1.0 - 1e-7, 0.0, 1.69e8)
        xb, jb, _ = oracle_mod.map_nu(r, 0.0, 1.0 + 1e-7, 0.0, 1.69e8)
        assert abs(xa - x1) / x1 < 1e-5 and abs(xb - x1) / x1 < 1e-5
        assert abs(ja - j1) / j1 < 1e-5 and abs(jb - j1) / j1 < 1e-5
    # invalid interval is reported
    assert oracle_mod.map_nu(0.5, 10.0, 0.8, 50.0, 200.0)[2] == 1


BW_CASES = [  # (M, G, xmin, xmax)
    (80.4, 2.1, 0.0, 1.69e8), (80.4, 2.1, 0.0, 100.0), (125.0, 0.004, 0.0, 1.69e8), (91.2, 2.5, 8000.0, 8400.0),
    (173.0, 1.4, 1e4, 3.1e4), (125.0, 0.004, 15620.0, 15630.0), (80.4, 2.1, 6000.0, 6000.001),
]


@pytest.mark.parametrize("case", BW_CASES)
def test_breit_wigner_matches_literal_formula(oracle_mod, case):
    M, G, xmin, xmax = case
    for r in [1e-12, 1e-6, 0.013, 0.31, 0.5, 0.77, 0.999, 1 - 1e-9]:
        x, j, st = oracle_mod.map_bw(r, M, G, xmin, xmax)
        xl, jl = literal_bw(r, M, G, xmin, xmax)
        assert st == 0
        # accurate to a few ulp of x, and relative to the distance from the nearer endpoint
        ref = min(abs(float(xl - xmin)), abs(float(xmax - xl)))
        assert abs(float(x - xl)) <= 1e-13 * max(ref, 1e-300) + 4e-16 * abs(float(xl)) + 1e-15 * M * G
        assert rel(j, jl) < 1e-12


@pytest.mark.parametrize("case", BW_CASES)
def test_breit_wigner_endpoints_jacobian_inverse(oracle_mod, case):
    M, G, xmin, xmax = case
    assert oracle_mod.map_bw(0.0, M, G, xmin, xmax)[0] == xmin
    assert abs(oracle_mod.map_bw(1.0, M, G, xmin, xmax)[0] - xmax) <= 4.5e-16 * xmax
    t, wq = np.polynomial.legendre.leggauss(60)
    # J is smooth in r but very peaked at the ends of wide ranges: geometric panels towards 0 and 1
    g = np.geomspace(1e-14, 0.5, 120)
    edges = np.unique(np.concatenate([[0.0, 1.0], g, 1.0 - g, np.linspace(0.0, 1.0, 101)]))
    acc = 0.0
    for lo, hi in zip(edges[:-1], edges[1:]):
        rr = 0.5 * (hi - lo) * t + 0.5 * (hi + lo)
        acc += 0.5 * (hi - lo) * sum(w * oracle_mod.map_bw(r, M, G, xmin, xmax)[1] for r, w in zip(rr, wq))
    # (quadrature nodes within 1e-9 of r = 1 are themselves only representable to ~1e-7 relative
    #  in 1 - r, which bounds this check for the narrowest widths)
    assert abs(acc - (xmax - xmin)) < 1e-8 * (xmax - xmin)
    for r in [1e-9, 0.2, 0.5, 0.9, 1 - 1e-7]:
        x, j, _ = oracle_mod.map_bw(r, M, G, xmin, xmax)
        # x itself is only known to its ulp: allow that much, mapped back through dr/dx = 1/J
        assert abs(oracle_mod.inv_bw(x, M, G, xmin, xmax) - r) < 1e-12 + 2.0 * np.spacing(x) / j


def test_r_to_x1x2(oracle_mod):
    S = 13000.0 ** 2
    for r in [1e-9, 0.25, 0.5, 0.8]:
        for shat in [1.0, 1e4, 1e7, 1.6e8]:
            x1, x2, j = oracle_mod.r_to_x1x2(r, shat, S)
            assert abs(x1 * x2 - shat / S) < 1e-14 * shat / S
            xl = mp.mpf(shat / S) ** mp.mpf(r)
            assert rel(x1, xl) < 1e-14
            assert abs(j - (-math.log(shat / S) / S)) < 1e-15 * j


def test_luminosity_area_closed_form(oracle_mod):
    """Integral of J_shat * J_x over r_shat, r_x in [0,1]^2 with shat in [tau0 S, S]
    is the area {x1 x2 >= tau0} of the unit square, 1 - tau0 + tau0 log tau0."""
    S = 13000.0 ** 2
    tau0 = 1e-3
    t, wq = np.polynomial.legendre.leggauss(120)
    rr = 0.5 * t + 0.5
    acc = 0.0
    for r1, w1 in zip(rr, wq):
        shat, js, _ = oracle_mod.map_nu(r1, 0.0, 1.0, tau0 * S, S, a=0.0)
        _, _, jx = oracle_mod.r_to_x1x2(0.5, shat, S)
        acc += 0.5 * w1 * js * jx  # J_x does not depend on r_x, so that integral is 1
    exact = 1.0 - tau0 + tau0 * math.log(tau0)
    assert abs(acc - exact) < 1e-12


def test_kallen(oracle_mod):
    for x, y, z in [(100.0, 1.0, 4.0), (1e6, 173.0 ** 2, 173.0 ** 2), (50.0, 0.0, 0.0), (7.0, -3.0, 1.0)]:
        lit = (mp.mpf(x) - y - z) ** 2 - 4 * mp.mpf(y) * z
        assert rel(oracle_mod.kallen(x, y, z), lit) < 1e-14
    assert oracle_mod.kallen(4.0, 1.0, 1.0) == 0.0  # threshold
    assert oracle_mod.kallen(3.0, 1.0, 1.0) == 0.0  # below threshold, clamped
