"""Oracle pins for the integrands and the local multichannel weights against values the
mathematics fixes, with no use of the oracle's own formulas:

* the 2->4 W W integral (parton densities times two W propagators, Sec. 2.2.2 and the
  phase-space factorisation of Sec. 2.2) by an independent nested quadrature over
  (tau, y, s1, s2), against the oracle's Monte Carlo estimate;
* the SDE channel weights P_c (Sec. 2.1, products of propagator denominators) written out
  by hand for the six 2->5 channels and evaluated at 50 digits on hand-built momenta whose
  invariants are exact in double precision;
* the parton-density factor f(x1) f(x2) of the integrand at 50 digits;
* alpha_c = P_c / sum_j P_j summing to one over the channels for the same momenta;
* the Kallen function's branch for two space-like legs (every t-chain block uses it).
"""
import math

import mpmath as mp
import numpy as np
from scipy import integrate

from paper_2602_06895_gb300 import workloads as W

mp.mp.dps = 50


# ---------------------------------------------------------------- nested quadrature of the 2->4 integral
# I = int dx1 dx2 f(x1) f(x2) int dPhi_4 BW(s1) BW(s2), with dx1 dx2 = dtau dy (x1,2 = sqrt(tau) e^(+-y)),
# shat = tau S and, by the factorisation dPhi_n = dPhi_(n-1) dPhi_2 ds/(2 pi) with massless two-body
# volumes 1/(8 pi):  Phi_4 = int ds1/(2 pi) ds2/(2 pi) sqrt(lambda(shat, s1, s2)) / (8 pi shat) / (8 pi)^2.
# f(x1) f(x2) = tau^a (1 + tau - 2 sqrt(tau) cosh y)^b for f(x) = x^a (1-x)^b.
_S = W.S_LHC
_M, _G = W.M_W, W.G_W
_M2, _MG = _M * _M, _M * _G
_A, _B = W.PDF_ALPHA, W.PDF_BETA
_CS = np.array([1.0, 5.0, 25.0])
_WIN = _CS[-1] * _MG
# panel breakpoints in s: around the W peak, then geometric above it
_PEAK_BP = np.concatenate([_M2 - _CS[::-1] * _MG, [_M2], _M2 + _CS * _MG, (_M2 + _WIN) * 4.0 ** np.arange(1, 13)])


def _gl01(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def _bw(s):
    return 1.0 / ((s - _M2) ** 2 + _MG ** 2)


def _panels(lo, hi, bps, n):
    """Nodes s and weights BW(s) ds of Gauss-Legendre rules on [lo, hi] (arrays), cut at the
    breakpoints into panels.  A panel below the peak window is mapped by s = t^2 (square-root
    behaviour at s = 0), one inside by s = M^2 + M G tan(t) (flat in t), one above by s = e^t;
    every panel then by t = ta + (tb - ta)(2v - v^2), which absorbs a square-root end point."""
    lo = np.asarray(lo, float)
    hi = np.asarray(hi, float)
    bp = np.clip(bps, lo[..., None], hi[..., None])
    edges = np.sort(np.concatenate([lo[..., None], bp, hi[..., None]], -1), -1)
    p, q = edges[..., :-1, None], edges[..., 1:, None]
    v, wv = _gl01(n)
    u, du = 2 * v - v * v, 2 * (1 - v) * wv
    mid = 0.5 * (p + q)
    inside = np.abs(mid - _M2) < _WIN
    below = mid <= _M2 - _WIN
    tp, tq = np.sqrt(p), np.sqrt(q)
    t = tp + (tq - tp) * u
    s_lo, w_lo = t * t, 2 * t * (tq - tp) * du * _bw(t * t)
    ap, aq = np.arctan((p - _M2) / _MG), np.arctan((q - _M2) / _MG)
    s_pk, w_pk = _M2 + _MG * np.tan(ap + (aq - ap) * u), (aq - ap) * du / _MG
    lp, lq = np.log(np.maximum(p, _M2)), np.log(np.maximum(q, _M2))
    s_hi = np.exp(lp + (lq - lp) * u)
    w_hi = s_hi * (lq - lp) * du * _bw(s_hi)
    s = np.where(inside, s_pk, np.where(below, s_lo, s_hi))
    w = np.where(inside, w_pk, np.where(below, w_lo, w_hi))
    return s.reshape(s.shape[:-2] + (-1,)), w.reshape(w.shape[:-2] + (-1,))


def _phase_space_bw(shat, n=16):
    """int ds1/(2pi) ds2/(2pi) BW(s1) BW(s2) sqrt(lambda)/(8 pi shat)/(8 pi)^2 over
    sqrt(s1) + sqrt(s2) <= sqrt(shat).  The s1 panels are also cut where the upper end of the
    s2 range, (sqrt(shat) - sqrt(s1))^2, crosses the s2 peak window."""
    rs = math.sqrt(shat)
    x = _PEAK_BP[(_PEAK_BP > 0) & (_PEAK_BP < shat)]
    s1, w1 = _panels(np.array(0.0), np.array(shat), np.concatenate([_PEAK_BP, (rs - np.sqrt(x)) ** 2]), n)
    s_minus, s_plus = (rs - np.sqrt(s1)) ** 2, (rs + np.sqrt(s1)) ** 2
    s2, w2 = _panels(np.zeros_like(s1), s_minus, np.broadcast_to(_PEAK_BP, s1.shape + _PEAK_BP.shape), n)
    lam = np.maximum(s_minus[..., None] - s2, 0.0) * (s_plus[..., None] - s2)  # lambda = (s2 - s-)(s2 - s+)
    inner = np.sum(w2 * np.sqrt(lam), -1)
    return np.sum(w1 * inner) / (2 * math.pi) ** 2 / (8 * math.pi) ** 2 / (8 * math.pi * shat)


def _rapidity_integral(tau, n=40):
    """int_{-Y}^{Y} dy (1 + tau - 2 sqrt(tau) cosh y)^b, Y = -ln(tau)/2."""
    Y = -0.5 * math.log(tau)
    x, w = np.polynomial.legendre.leggauss(n)
    return Y * np.sum(w * (1 + tau - 2 * math.sqrt(tau) * np.cosh(Y * x)) ** _B)


def _rapidity_closed_form(tau):
    """The same for b = 3 from int cosh^k over [-Y, Y]: 2Y, 2 sinh Y, Y + sinh(2Y)/2,
    sinh(3Y)/6 + 3 sinh(Y)/2."""
    Y = mp.mpf(-0.5) * mp.log(tau)
    b, g = 1 + mp.mpf(tau), 2 * mp.sqrt(tau)
    c0, c1 = 2 * Y, 2 * mp.sinh(Y)
    c2, c3 = Y + mp.sinh(2 * Y) / 2, mp.sinh(3 * Y) / 6 + 3 * mp.sinh(Y) / 2
    return b ** 3 * c0 - 3 * b ** 2 * g * c1 + 3 * b * g ** 2 * c2 - g ** 3 * c3


def c2_integral_quadrature(n=16):
    """I = int d(ln tau) tau^(1+a) Y(tau) Phi_BW(tau S), adaptive in ln tau (cut at the
    single- and double-resonance thresholds), Gauss-Legendre panels inside."""
    f = lambda rho: math.exp(rho * (1 + _A)) * _rapidity_integral(math.exp(rho)) * _phase_space_bw(math.exp(rho) * _S, n)
    pts = sorted(math.log(x / _S) for x in [_M2, 4 * _M2, (2 * _M + 5 * _G) ** 2, (2 * _M - 5 * _G) ** 2,
                                            (_M + 25 * _G) ** 2])
    # below tau = 1e-12 the integrand falls like tau^(1.9) ln(1/tau): < 1e-12 of the total
    val, err = integrate.quad(f, math.log(1e-12), 0.0, points=pts, epsabs=0.0, epsrel=1e-9, limit=400)
    return val, err


def test_quadrature_building_blocks():
    """The quadrature's own checks: the rapidity integral against its closed form; the
    two-invariant integral converged in the rule order; far below the W peak it is the closed-form
    massless four-body volume times the two (then constant) propagators."""
    for tau in (1e-6, 1e-4, 0.01, 0.3):
        assert abs(_rapidity_integral(tau) / float(_rapidity_closed_form(tau)) - 1) < 1e-12
    for shat in (100.0 ** 2, 161.0 ** 2, 300.0 ** 2, 3000.0 ** 2):
        a, b = _phase_space_bw(shat, 16), _phase_space_bw(shat, 28)
        assert abs(a / b - 1) < 1e-7, shat
    # far below the peak both propagators equal 1/(M^4 + M^2 G^2); the rest is then the closed-form
    # massless four-body volume (2 pi)^-8 (pi/2)^3 shat^2 / (3! 2!), i.e. int sqrt(lambda) ds1 ds2 =
    # shat^3 / 12.  At shat = 1e-4 GeV^2 the propagators vary by 3e-8 across the range.
    shat = 1e-4
    want = (shat ** 3 / 12) / (2 * math.pi) ** 2 / (8 * math.pi) ** 3 / shat * _bw(0.0) ** 2
    assert abs(_phase_space_bw(shat, 24) / want - 1) < 1e-6
    vol4 = (2 * math.pi) ** -8 * (math.pi / 2) ** 3 * shat ** 2 / (6 * 2)
    assert abs(want / _bw(0.0) ** 2 / vol4 - 1) < 1e-14


def test_c2_integral_by_nested_quadrature(oracle_mod):
    """The oracle's Monte Carlo estimate of the 2->4 W W integral (no VEGAS, 8e6 Philox
    events) lies within 4 sigma of the nested quadrature, which is converged to far below 1e-6."""
    ch = W.ww_hadronic(vegas_dims=0)
    exact, err = c2_integral_quadrature()
    assert err < 1e-9 * exact
    o = oracle_mod.generate(ch, 1002, 0, 8_000_000, keep_momenta=False)
    w = o["w"]
    mean, sig = w.mean(), w.std() / math.sqrt(w.size)
    assert sig / mean < 2e-3
    assert abs(mean - exact) < 4 * sig, (mean, exact, sig)


# ---------------------------------------------------------------- SDE weights on hand-built momenta
# Five massless momenta from Pythagorean quadruples (components in units of 10 GeV), summing to
# p_a + p_b with p_a = (360,0,0,360), p_b = (110,0,0,-110): every component, sum and invariant
# below is an integer, exact in double precision.
_P = [(130, 30, 40, 120), (70, -20, -30, 60), (90, -10, -40, -80), (90, -40, 40, 70), (90, 40, -10, 80)]
_PA, _PB = (360, 0, 0, 360), (110, 0, 0, -110)


def _hand_momenta():
    return np.array([[_PA, _PB] + _P], dtype=np.float64)


def _m(q):
    return q[0] ** 2 - q[1] ** 2 - q[2] ** 2 - q[3] ** 2


def _add(*ps):
    return tuple(sum(mp.mpf(p[k]) for p in ps) for k in range(4))


def _sub(a, *ps):
    return tuple(mp.mpf(a[k]) - sum(mp.mpf(p[k]) for p in ps) for k in range(4))


def _bwlit(s, M, G):
    M, G = mp.mpf(M), mp.mpf(G)
    return 1 / ((s - M * M) ** 2 + M * M * G * G)


def _tlit(t):
    return 1 / (t - mp.mpf(W.M_W) ** 2) ** 2  # t-channel propagator mass 80.4 GeV


def _p_literal(c):
    """P_c of the six 2->5 channels, written out: resonant s-channel propagators of the channel's
    tree and the t-channel propagators q_k = p_a - (legs 1..k of the chain)."""
    p1, p2, p3, p4, p5 = _P
    s12, s34 = _m(_add(p1, p2)), _m(_add(p3, p4))
    if c == 0:
        return (_tlit(_m(_sub(_PA, p1))) * _tlit(_m(_sub(_PA, p1, p2))) * _tlit(_m(_sub(_PA, p1, p2, p3)))
                * _tlit(_m(_sub(_PA, p1, p2, p3, p4))))
    if c in (1, 2):
        M, G = (W.M_Z, W.G_Z) if c == 1 else (W.M_H, W.G_H)
        return (_bwlit(s12, M, G) * _tlit(_m(_sub(_PA, p1, p2))) * _tlit(_m(_sub(_PA, p1, p2, p3)))
                * _tlit(_m(_sub(_PA, p1, p2, p3, p4))))
    if c == 3:
        return (_bwlit(s12, W.M_T, W.G_T) * _bwlit(s34, W.M_Z, W.G_Z) * _tlit(_m(_sub(_PA, p1, p2)))
                * _tlit(_m(_sub(_PA, p1, p2, p3, p4))))
    if c == 4:
        return _bwlit(s12, W.M_Z, W.G_Z) * _bwlit(s34, W.M_T, W.G_T)
    if c == 5:
        return (_bwlit(s12, W.M_Z, W.G_Z) * _bwlit(s34, W.M_H, W.G_H) * _tlit(_m(_sub(_PA, p1, p2)))
                * _tlit(_m(_sub(_PA, p1, p2, p3, p4))))
    raise ValueError(c)


def test_hand_built_momenta_conserve():
    tot = _add(*_P)
    assert tot == _add(_PA, _PB)
    for p in _P:
        assert _m(p) == 0


def test_sde_weights_literal_on_hand_built_momenta(oracle_mod):
    chans = W.multichannel_2to5()
    mom = _hand_momenta()
    lit = [_p_literal(c) for c in range(6)]
    for c in range(6):
        got = oracle_mod.sde_weights(chans, c, mom)[0]
        assert abs(mp.mpf(got) / lit[c] - 1) < 1e-14, (c, got, lit[c])
    # alpha_c = P_c / sum_j P_j at 50 digits against the oracle's propagator products
    tot = sum(lit)
    P = np.array([oracle_mod.sde_weights(chans, c, mom)[0] for c in range(6)])
    for c in range(6):
        assert abs(mp.mpf(P[c] / P.sum()) / (lit[c] / tot) - 1) < 1e-14


def _pdf_lit(x):
    x = mp.mpf(x)
    return x ** mp.mpf(_A) * (1 - x) ** mp.mpf(_B)


def test_integrand_pdf_factor_literal(oracle_mod):
    """f = f(x1) f(x2) P_own for the 2->4 workload and f = f(x1) f(x2) (P_own + sum_{j != c} P_j(p))
    for a 2->5 channel, with f(x) = x^-1.1 (1-x)^3 at 50 digits on the oracle's own x1, x2,
    P_own and momenta; the SDE weight is alpha = P_own over that sum."""
    ch = W.ww_hadronic(vegas_dims=0)
    r = W.uniform_r(811, 400, oracle_mod.dims(ch))
    o = oracle_mod.forward(ch, r, aux=True)
    for e in range(0, 400, 7):
        x1, x2 = o["x"][e]
        a = o["aux"][e]
        want = _pdf_lit(x1) * _pdf_lit(x2) * mp.mpf(a[oracle_mod.AUX["p_own"]])
        assert abs(mp.mpf(a[oracle_mod.AUX["f"]]) / want - 1) < 1e-14
    chans = W.multichannel_2to5()
    for c in (1, 5):
        r = W.uniform_r(812 + c, 300, 13)
        o = oracle_mod.forward(chans[c], r, channels=chans, chan=c, aux=True)
        others = sum(oracle_mod.sde_weights(chans, j, o["mom"]) for j in range(6) if j != c)
        for e in range(0, 300, 5):
            if o["w"][e] == 0.0:
                continue
            x1, x2 = o["x"][e]
            a = o["aux"][e]
            tot = mp.mpf(a[oracle_mod.AUX["p_own"]]) + mp.mpf(others[e])
            assert abs(mp.mpf(a[oracle_mod.AUX["f"]]) / (_pdf_lit(x1) * _pdf_lit(x2) * tot) - 1) < 1e-14
            assert abs(mp.mpf(o["alpha"][e]) - mp.mpf(a[oracle_mod.AUX["p_own"]]) / tot) < 1e-15


def test_alpha_sums_to_one_over_channels(oracle_mod):
    """For the momenta of events of each 2->5 channel: the six alpha_j(p) = P_j(p)/sum_k P_k(p) sum
    to one to 1e-15, and the channel's own alpha (its P from the sampled invariants) agrees with
    alpha_c(p) within the propagator product's rounding."""
    chans = W.multichannel_2to5()
    for c in range(6):
        r = W.uniform_r(900 + c, 3000, 13)
        o = oracle_mod.forward(chans[c], r, channels=chans, chan=c, aux=True)
        keep = o["w"] != 0
        P = np.array([oracle_mod.sde_weights(chans, j, o["mom"]) for j in range(6)])[:, keep]
        al = P / P.sum(axis=0)
        assert np.max(np.abs(al.sum(axis=0) - 1.0)) <= 1e-15
        a_own = o["alpha"][keep]
        rel_p = np.abs(o["aux"][keep, oracle_mod.AUX["p_own"]] / P[c] - 1.0)
        # |d alpha| <= alpha (1 - alpha) |dP/P| (to first order), plus the divisions' rounding
        bound = al[c] * (1 - al[c]) * rel_p * 1.01 + 4e-16
        assert np.all(np.abs(a_own - al[c]) <= bound)
        assert np.median(np.abs(a_own - al[c])) < 1e-14


def test_kallen_two_spacelike_legs(oracle_mod):
    """lambda(x, y, z) with y, z < 0 (the t-chain blocks' incoming legs), with one space-like leg,
    and symmetric cases, against the literal x^2 + y^2 + z^2 - 2xy - 2xz - 2yz at 50 digits."""
    cases = [(100.0, -1.0, -4.0), (1e6, -3.0e4, -2.9e4), (8317.44, -1239.0, -1e-9), (1e-3, -5e4, -5e4),
             (6464.16, -2.0e5, -7.0), (2.5e7, -1e3, 0.0), (400.0, -50.0, 30.0), (1.0e4, 0.0, -1.0e4)]
    for x, y, z in cases:
        X, Y, Z = mp.mpf(x), mp.mpf(y), mp.mpf(z)
        lit = X * X + Y * Y + Z * Z - 2 * X * Y - 2 * X * Z - 2 * Y * Z
        assert lit > 0
        assert abs(mp.mpf(oracle_mod.kallen(x, y, z)) / lit - 1) < 1e-14, (x, y, z)
        assert oracle_mod.kallen(x, z, y) == oracle_mod.kallen(x, y, z)
