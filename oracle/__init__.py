"""FP64 CPU oracle of the phase-space hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path:
the arithmetic lives in ``ps_oracle.c`` (plain C, IEEE double, no FMA
contraction); this file only compiles it on demand, lays out its structures
and marshals numpy arrays.

Inputs are the plain channel dictionaries of the workload module (topology,
masses, widths, exponents) and seeded random points.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ps_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_PROBE = os.path.join(_HERE, "rounding_probe.h")
_RLIB = os.path.join(_HERE, "liboracle_rounding.so")
_FLIB = os.path.join(_HERE, "liboracle_fma.so")
_FRLIB = os.path.join(_HERE, "liboracle_fma_rounding.so")
_COUNT_H = os.path.join(_HERE, "op_count.h")
_CLIB = os.path.join(_HERE, "liboracle_count.so")
_lock = threading.Lock()
_lib = None
_rlib = None
_flib = None
_frlib = None
_clib = None

MAXN, MAXK, MAXP, MAXC, NAUX = 32, 10, 16, 32, 10
AUX = {"shat": 0, "w_ps": 1, "f": 2, "jac_vegas": 3, "p_own": 4, "cut": 5, "fail": 6, "p_own_momenta": 7, "cond": 8, "cond_p": 9}


def build(force=False):
    """Compile ps_oracle.c into liboracle.so (gcc, -O2 -ffp-contract=off, OpenMP), the
    rounding-probe copy liboracle_rounding.so (rounding_probe.h force-included, no OpenMP), and
    liboracle_fma.so with multiply-adds contracted wherever the compiler may (-ffp-contract=fast;
    on machines with a fused multiply-add instruction, e.g. aarch64, that is a second, equally
    valid rounding of the same formulas), liboracle_fma_rounding.so (both: contracted and with
    the rounding probe), and liboracle_count.so, compiled as C++ with op_count.h
    force-included: the same arithmetic, with every operation counted by class."""
    src_time = max(os.path.getmtime(_SRC), os.path.getmtime(_PROBE))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
               "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    if force or not os.path.exists(_RLIB) or os.path.getmtime(_RLIB) < src_time:
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-include", _PROBE,
               "-o", _RLIB + ".tmp", _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(_RLIB + ".tmp", _RLIB)
    if force or not os.path.exists(_FLIB) or os.path.getmtime(_FLIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-ffp-contract=fast", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
               "-o", _FLIB + ".tmp", _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(_FLIB + ".tmp", _FLIB)
    if force or not os.path.exists(_FRLIB) or os.path.getmtime(_FRLIB) < src_time:
        cmd = ["gcc", "-O2", "-ffp-contract=fast", "-fno-fast-math", "-fPIC", "-shared", "-include", _PROBE,
               "-o", _FRLIB + ".tmp", _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(_FRLIB + ".tmp", _FRLIB)
    ctime = max(os.path.getmtime(_SRC), os.path.getmtime(_COUNT_H))
    if force or not os.path.exists(_CLIB) or os.path.getmtime(_CLIB) < ctime:
        cmd = ["g++", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-x", "c++",
               "-DORC_BOOKKEEPING=0", "-include", _COUNT_H, "-o", _CLIB + ".tmp", _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(_CLIB + ".tmp", _CLIB)
    return _LIB


class Node(C.Structure):
    _fields_ = [("kind", C.c_int32), ("nchild", C.c_int32), ("child", C.c_int32 * MAXK),
                ("leaf", C.c_int32), ("sde", C.c_int32), ("mass", C.c_double),
                ("M", C.c_double), ("G", C.c_double), ("nu", C.c_double)]


class Channel(C.Structure):
    _fields_ = [("n", C.c_int32), ("hadronic", C.c_int32), ("n_nodes", C.c_int32), ("n_sorder", C.c_int32),
                ("sorder", C.c_int32 * MAXN), ("tside", C.c_int32 * MAXK), ("integrand", C.c_int32),
                ("vegas_dims", C.c_int32), ("vegas_bins", C.c_int32), ("partonic", C.c_int32),
                ("sqrt_s", C.c_double), ("S", C.c_double), ("a", C.c_double),
                ("shat_M", C.c_double), ("shat_G", C.c_double), ("shat_nu", C.c_double),
                ("t_nu", C.c_double), ("ts_nu", C.c_double), ("Mt", C.c_double),
                ("pdf_a", C.c_double), ("pdf_b", C.c_double), ("node", Node * MAXN)]


class Prop(C.Structure):
    _fields_ = [("kind", C.c_int32), ("mask", C.c_int32), ("M", C.c_double), ("G", C.c_double)]


class Sde(C.Structure):
    _fields_ = [("n_ch", C.c_int32), ("n_prop", C.c_int32 * MAXC), ("prop", (Prop * MAXP) * MAXC)]


_D = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def _setup(L):
    L.orc_philox4x32_10.argtypes = [C.POINTER(C.c_uint32)] * 3
    L.orc_bits_to_unit.restype = C.c_double
    L.orc_bits_to_unit.argtypes = [C.c_uint64]
    L.orc_random_batch.argtypes = [C.c_uint64, C.c_uint32, C.c_uint64, C.c_int64, C.c_int, _D, C.c_int]
    L.orc_kallen.restype = C.c_double
    L.orc_kallen.argtypes = [C.c_double] * 3
    L.orc_map_nu.argtypes = [C.c_double] * 6 + [C.POINTER(C.c_double)] * 2
    L.orc_map_bw.argtypes = [C.c_double] * 5 + [C.POINTER(C.c_double)] * 2
    L.orc_inv_nu.restype = C.c_double
    L.orc_inv_nu.argtypes = [C.c_double] * 6
    L.orc_inv_bw.restype = C.c_double
    L.orc_inv_bw.argtypes = [C.c_double] * 5
    L.orc_r_to_x1x2.argtypes = [C.c_double] * 3 + [C.POINTER(C.c_double)] * 3
    L.orc_two_body_decay.restype = C.c_double
    L.orc_two_body_decay.argtypes = [C.c_double] * 5 + [C.c_void_p, _D, _D]
    L.orc_t_min_max.argtypes = [C.c_double] * 5 + [C.POINTER(C.c_double)] * 2
    L.orc_two_to_two.restype = C.c_double
    L.orc_two_to_two.argtypes = [C.c_double, _D, _D] + [C.c_double] * 6 + [_D, _D]
    L.orc_vegas_map.restype = C.c_double
    L.orc_vegas_map.argtypes = [C.c_double, _D, C.c_int, C.POINTER(C.c_double)]
    L.orc_vegas_inv.restype = C.c_double
    L.orc_vegas_inv.argtypes = [C.c_double, _D, C.c_int]
    L.orc_vegas_accumulate.argtypes = [_D, C.c_int, _D, C.c_int64, C.c_int, C.c_int, _D]
    L.orc_vegas_rebin.argtypes = [_D, _D, _D, C.c_int, C.c_double]
    L.orc_channel_dims.restype = C.c_int
    L.orc_channel_dims.argtypes = [C.POINTER(Channel)]
    L.orc_forward_batch.argtypes = [C.POINTER(Channel), C.POINTER(Sde), C.c_int, C.c_void_p, C.c_int64,
                                    _D, _D, _D, _D, _D, C.c_void_p, C.c_int]
    L.orc_generate_batch.argtypes = [C.POINTER(Channel), C.POINTER(Sde), C.c_int, C.c_void_p, C.c_uint64,
                                     C.c_uint64, C.c_int64, C.c_void_p, C.c_void_p, _D, C.c_void_p,
                                     C.c_int]
    L.orc_inverse_batch.argtypes = [C.POINTER(Channel), C.c_void_p, C.c_int64, _D, _D, _D, C.c_int]
    L.orc_stats.argtypes = [_D, C.c_int64, _D]
    L.orc_sde_weights.argtypes = [C.POINTER(Sde), C.c_int, C.c_int64, C.c_int, _D, _D]
    L.orc_max_threads.restype = C.c_int
    assert L.orc_sizeof_channel() == C.sizeof(Channel)
    assert L.orc_sizeof_sde() == C.sizeof(Sde)
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _setup(C.CDLL(_LIB))
    return _lib


def rounding_lib():
    """The rounding-probe copy of the oracle (see rounding_probe.h)."""
    global _rlib
    with _lock:
        if _rlib is None:
            build()
            L = _setup(C.CDLL(_RLIB))
            L.orc_rounding_seed.argtypes = [C.c_uint64]
            _rlib = L
    return _rlib


def fma_lib():
    """The oracle compiled with contracted multiply-adds (see build)."""
    global _flib
    with _lock:
        if _flib is None:
            build()
            _flib = _setup(C.CDLL(_FLIB))
    return _flib


def count_lib():
    """The operation-counting copy of the oracle (see op_count.h)."""
    global _clib
    with _lock:
        if _clib is None:
            build()
            L = _setup(C.CDLL(_CLIB))
            L.orc_count_classes.restype = C.c_int
            L.orc_count_get.argtypes = [C.POINTER(C.c_ulonglong)]
            _clib = L
    return _clib


OP_CLASSES = ("add", "mul", "div", "sqrt", "exp", "expm1", "log", "log1p", "pow", "atan", "atan2", "tan", "sin",
              "cos", "cmp", "other")


def op_counts(ch, r, grid=None, channels=None, chan=0):
    """Operations of the forward map per event, by class (op_count.h), averaged over the points r
    [B, d]: the method's arithmetic as the oracle performs it (condition-number bookkeeping
    excluded).  Returns (counts per event as a dict, the forward result)."""
    L = count_lib()
    assert L.orc_count_classes() == len(OP_CLASSES)
    L.orc_count_reset()
    res = _forward(L, ch, r, grid, channels, chan, 1, False)
    buf = (C.c_ulonglong * len(OP_CLASSES))()
    L.orc_count_get(buf)
    B = r.shape[0]
    return {k: buf[i] / B for i, k in enumerate(OP_CLASSES)}, res


def fma_rounding_lib():
    """The oracle compiled with contracted multiply-adds and the rounding probe (see build)."""
    global _frlib
    with _lock:
        if _frlib is None:
            build()
            L = _setup(C.CDLL(_FRLIB))
            L.orc_rounding_seed.argtypes = [C.c_uint64]
            _frlib = L
    return _frlib


def max_threads():
    return lib().orc_max_threads()


# --------------------------------------------------------------------------
# Channel encoding
# --------------------------------------------------------------------------
_INTEGRAND = {"none": 0, "one_plus_cos2": 1, "pdf_props": 2, "pdf_sde": 3, "pdf_sde_uniform": 4}
_KIND = {"leaf": 0, "decay": 1, "tchain": 2}


def encode_channel(ch):
    c = Channel()
    c.n = ch["n"]
    c.hadronic = 1 if ch["hadronic"] else 0
    nodes = ch["nodes"]
    c.n_nodes = len(nodes)
    for j, nd in enumerate(nodes):
        o = c.node[j]
        o.kind = _KIND[nd["kind"]]
        kids = nd.get("children", [])
        o.nchild = len(kids)
        for k, kid in enumerate(kids):
            o.child[k] = kid
        o.leaf = nd.get("leaf", -1)
        o.sde = 1 if nd.get("sde", False) else 0
        o.mass = nd.get("mass", 0.0)
        o.M = nd.get("M", 0.0)
        o.G = nd.get("G", 0.0)
        o.nu = nd.get("nu", 0.8)
    c.n_sorder = len(ch["sorder"])
    for i, j in enumerate(ch["sorder"]):
        c.sorder[i] = j
    for i, sd in enumerate(ch["tside"]):
        c.tside[i + 1] = sd
    c.integrand = _INTEGRAND[ch["integrand"]]
    c.vegas_dims = ch["vegas_dims"]
    c.vegas_bins = ch["vegas_bins"]
    c.partonic = 1 if ch.get("partonic", False) else 0
    c.sqrt_s = ch["sqrt_s"]
    c.S = ch["S"]
    c.a = ch["a"]
    c.shat_M = ch["shat"]["M"]
    c.shat_G = ch["shat"]["G"]
    c.shat_nu = ch["shat"]["nu"]
    c.t_nu = ch["t_nu"]
    c.ts_nu = ch["ts_nu"]
    c.Mt = ch["Mt"]
    c.pdf_a, c.pdf_b = ch["pdf"]
    return c


def _leaves(nodes, j):
    nd = nodes[j]
    if nd["kind"] == "leaf":
        return 1 << nd["leaf"]
    m = 0
    for k in nd["children"]:
        m |= _leaves(nodes, k)
    return m


def sde_props(ch):
    """Propagators of one channel for the SDE weights (Sec. 2.1): every resonant
    s-channel node (mask of the leaves below it) and every t-channel propagator
    q_k = p_a - (legs 1..k of the chain), k = 1..kappa, with mass Mt."""
    nodes = ch["nodes"]
    props = []
    for j, nd in enumerate(nodes):
        if nd["kind"] == "decay" and nd.get("sde", False) and j != 0:
            props.append((0, _leaves(nodes, j), nd["M"], nd["G"]))
    if nodes[0]["kind"] == "tchain":
        legs = nodes[0]["children"]
        m = 0
        for k in range(len(legs) - 1):
            m |= _leaves(nodes, legs[k])
            props.append((1, m, ch["Mt"], 0.0))
    return props


def encode_sde(channels):
    s = Sde()
    s.n_ch = len(channels)
    for c, ch in enumerate(channels):
        props = sde_props(ch)
        s.n_prop[c] = len(props)
        for k, (kind, mask, M, G) in enumerate(props):
            p = s.prop[c][k]
            p.kind, p.mask, p.M, p.G = kind, mask, M, G
    return s


def dims(ch):
    c = ch if isinstance(ch, Channel) else encode_channel(ch)
    return lib().orc_channel_dims(C.byref(c))


def _grid_arg(ch, grid):
    if ch["vegas_dims"] == 0:
        return None, None
    g = np.ascontiguousarray(grid, dtype=np.float64)
    assert g.shape == (ch["vegas_dims"], ch["vegas_bins"] + 1)
    return g, g.ctypes.data_as(C.c_void_p)


def _threads(threads):
    return int(threads) if threads else max_threads()


def forward(ch, r, grid=None, channels=None, chan=0, threads=None, aux=False):
    """Forward map of a batch: r [B, d] -> dict(mom [B, n+2, 4], x [B, 2], w [B], alpha [B], aux)."""
    return _forward(lib(), ch, r, grid, channels, chan, threads, aux)


def forward_fma(ch, r, grid=None, channels=None, chan=0, threads=None):
    """The forward map of the oracle compiled with contracted multiply-adds."""
    return _forward(fma_lib(), ch, r, grid, channels, chan, threads, False)


def forward_fma_perturbed(ch, r, seed, grid=None, channels=None, chan=0):
    """One run of the oracle compiled with contracted multiply-adds and with every elementary-
    function result moved by a random whole number of ulps in [-2, 2] (rounding_probe.h): a
    second FP64 evaluation that differs from the plain oracle the way another machine's
    compiler and libm can."""
    L = fma_rounding_lib()
    L.orc_rounding_seed(seed)
    return _forward(L, ch, r, grid, channels, chan, 1, False)


def rounding_spread(ch, r, grid=None, channels=None, chan=0, runs=8, base=None):
    """Rounding sensitivity of the forward map by stochastic arithmetic (see rounding_probe.h):
    the oracle re-run `runs` times with every elementary-function result moved by a random
    whole number of ulps in [-2, 2].  Per event: "w" the largest relative change of a nonzero
    weight, "alpha" that of the multichannel weight, "mom" the largest change of a momentum
    component over the event's largest energy, "flip" whether some run changed w == 0."""
    if base is None:
        base = forward(ch, r, grid, channels, chan)
    L = rounding_lib()
    B = base["w"].shape[0]
    scale = np.max(np.abs(base["mom"][:, :, 0]), axis=1)
    scale = np.where(scale > 0, scale, 1.0)
    nz = base["w"] != 0
    out = {"w": np.zeros(B), "alpha": np.zeros(B), "mom": np.zeros(B), "flip": np.zeros(B, bool)}
    for k in range(runs):
        L.orc_rounding_seed(k + 1)
        o = _forward(L, ch, r, grid, channels, chan, 1, False)
        both = nz & (o["w"] != 0)
        out["flip"] |= (o["w"] != 0) != nz
        rel = np.zeros(B)
        rel[both] = np.abs(o["w"][both] / base["w"][both] - 1.0)
        out["w"] = np.maximum(out["w"], rel)
        ra = np.zeros(B)
        ab = both & (base["alpha"] != 0)
        ra[ab] = np.abs(o["alpha"][ab] / base["alpha"][ab] - 1.0)
        out["alpha"] = np.maximum(out["alpha"], ra)
        dm = np.max(np.abs(o["mom"] - base["mom"]), axis=(1, 2)) / scale
        out["mom"] = np.maximum(out["mom"], np.where(both, dm, 0.0))
    return out


def _forward(L, ch, r, grid, channels, chan, threads, aux):
    c = encode_channel(ch)
    sde = encode_sde(channels if channels is not None else [ch])
    r = np.ascontiguousarray(r, dtype=np.float64)
    B, d = r.shape
    assert d == dims(c), (d, dims(c))
    n = ch["n"]
    mom = np.zeros((B, n + 2, 4))
    x = np.zeros((B, 2))
    w = np.zeros(B)
    alpha = np.zeros(B)
    auxa = np.zeros((B, NAUX)) if aux else None
    g, gp = _grid_arg(ch, grid)
    L.orc_forward_batch(C.byref(c), C.byref(sde), chan, gp, B, r, mom, x, w, alpha,
                        auxa.ctypes.data_as(C.c_void_p) if aux else None, _threads(threads))
    out = {"mom": mom, "x": x, "w": w, "alpha": alpha}
    if aux:
        out["aux"] = auxa
    return out


def generate(ch, seed, ev0, B, grid=None, channels=None, chan=0, threads=None, keep_momenta=True):
    """Philox-driven batch (the random point of event ev0 + e is drawn in place)."""
    L = lib()
    c = encode_channel(ch)
    sde = encode_sde(channels if channels is not None else [ch])
    n = ch["n"]
    mom = np.zeros((B, n + 2, 4)) if keep_momenta else None
    x = np.zeros((B, 2)) if keep_momenta else None
    w = np.zeros(B)
    alpha = np.zeros(B) if keep_momenta else None
    g, gp = _grid_arg(ch, grid)
    ptr = lambda a: a.ctypes.data_as(C.c_void_p) if a is not None else None
    L.orc_generate_batch(C.byref(c), C.byref(sde), chan, gp, seed, ev0, B, ptr(mom), ptr(x), w, ptr(alpha),
                         _threads(threads))
    return {"mom": mom, "x": x, "w": w, "alpha": alpha}


def random(seed, chan, ev0, B, d, threads=None):
    r = np.zeros((B, d))
    lib().orc_random_batch(seed, chan, ev0, B, d, r, _threads(threads))
    return r


def inverse(ch, mom, x, grid=None, threads=None):
    L = lib()
    c = encode_channel(ch)
    mom = np.ascontiguousarray(mom, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    B = mom.shape[0]
    r = np.zeros((B, dims(c)))
    g, gp = _grid_arg(ch, grid)
    L.orc_inverse_batch(C.byref(c), gp, B, mom, x, r, _threads(threads))
    return r


def sde_weights(channels, j, mom):
    """P_j(p) of channel j of `channels` (the SDE propagator product) for momenta [B, n+2, 4]."""
    sde = encode_sde(channels)
    mom = np.ascontiguousarray(mom, dtype=np.float64)
    out = np.zeros(mom.shape[0])
    lib().orc_sde_weights(C.byref(sde), j, mom.shape[0], mom.shape[1] - 2, mom, out)
    return out


def global_weights(channels, alphas, mom, x, grids=None, threads=None):
    """Global multichannel weights (Kleiss-Pittau, Eq. multi-channel-standard) of events given by
    lab momenta [B, n+2, 4] and x [B, 2]:  w = f / sum_j alpha_j g_j,  g_j = 1/J_j(G_j^-1(p)) with
    J_j the phase-space weight of channel j (integrand "none") at its inverse point, and
    f = pdf(x1) pdf(x2) sum_j P_j(p) (the integrand whose SDE split the channels' own weights use).
    Returns (w, J [M, B], P [M, B], r list)."""
    M = len(channels)
    grids = grids if grids is not None else [None] * M
    J, P, rs = [], [], []
    for j, ch in enumerate(channels):
        r = inverse(ch, mom, x, grids[j], threads)
        dens = dict(ch)
        dens["integrand"] = "none"
        J.append(forward(dens, r, grids[j], threads=threads)["w"])
        P.append(sde_weights(channels, j, mom))
        rs.append(r)
    J, P = np.array(J), np.array(P)
    ch0 = channels[0]
    f = P.sum(axis=0)
    if ch0["hadronic"]:
        a, b = ch0["pdf"]
        f = f * x[:, 0] ** a * (1 - x[:, 0]) ** b * x[:, 1] ** a * (1 - x[:, 1]) ** b
    al = np.asarray(alphas, dtype=np.float64)[:, None]
    inv = np.where(J > 0, 1.0 / np.where(J > 0, J, 1.0), 0.0)
    g = np.sum(al * inv, axis=0)
    w = np.where(g > 0, f / np.where(g > 0, g, 1.0), 0.0)
    return w, J, P, rs


def stats(w):
    out = np.zeros(5)
    w = np.ascontiguousarray(w, dtype=np.float64)
    lib().orc_stats(w, w.shape[0], out)
    return {"n": out[0], "n_nonzero": out[1], "sum_w": out[2], "sum_w2": out[3], "max_w": out[4]}


# --------------------------------------------------------------------------
# Single building blocks (for pins)
# --------------------------------------------------------------------------
def philox(ctr, key):
    c = (C.c_uint32 * 4)(*ctr)
    k = (C.c_uint32 * 2)(*key)
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return list(o)


def bits_to_unit(bits):
    return lib().orc_bits_to_unit(bits)


def kallen(x, y, z):
    return lib().orc_kallen(x, y, z)


def map_nu(r, m, nu, xmin, xmax, a=1e-4):
    x, j = C.c_double(), C.c_double()
    st = lib().orc_map_nu(r, m, nu, xmin, xmax, a, C.byref(x), C.byref(j))
    return x.value, j.value, st


def map_bw(r, M, G, xmin, xmax):
    x, j = C.c_double(), C.c_double()
    st = lib().orc_map_bw(r, M, G, xmin, xmax, C.byref(x), C.byref(j))
    return x.value, j.value, st


def inv_nu(x, m, nu, xmin, xmax, a=1e-4):
    return lib().orc_inv_nu(x, m, nu, xmin, xmax, a)


def inv_bw(x, M, G, xmin, xmax):
    return lib().orc_inv_bw(x, M, G, xmin, xmax)


def r_to_x1x2(r, shat, S):
    a, b, j = C.c_double(), C.c_double(), C.c_double()
    lib().orc_r_to_x1x2(r, shat, S, C.byref(a), C.byref(b), C.byref(j))
    return a.value, b.value, j.value


def two_body_decay(rphi, rth, s0, m1, m2, p0=None):
    p1 = np.zeros(4)
    p2 = np.zeros(4)
    p0a = None if p0 is None else np.ascontiguousarray(p0, dtype=np.float64)
    jac = lib().orc_two_body_decay(rphi, rth, s0, m1, m2,
                                   None if p0a is None else p0a.ctypes.data_as(C.c_void_p), p1, p2)
    return p1, p2, jac


def t_min_max(s, mA2, mB2, m1, m2):
    a, b = C.c_double(), C.c_double()
    lib().orc_t_min_max(s, mA2, mB2, m1, m2, C.byref(a), C.byref(b))
    return a.value, b.value


def two_to_two(rphi, pA, pB, tabs, m1, m2, s, mA2, mB2):
    p1 = np.zeros(4)
    p2 = np.zeros(4)
    jac = lib().orc_two_to_two(rphi, np.ascontiguousarray(pA, dtype=np.float64),
                               np.ascontiguousarray(pB, dtype=np.float64), tabs, m1, m2, s, mA2, mB2, p1, p2)
    return p1, p2, jac


def vegas_map(r, edges):
    e = np.ascontiguousarray(edges, dtype=np.float64)
    j = C.c_double(1.0)
    v = lib().orc_vegas_map(r, e, e.shape[0] - 1, C.byref(j))
    return v, j.value


def vegas_inv(rp, edges):
    e = np.ascontiguousarray(edges, dtype=np.float64)
    return lib().orc_vegas_inv(rp, e, e.shape[0] - 1)


def vegas_accumulate(r, w, dv, N, hist=None):
    r = np.ascontiguousarray(r, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    hist = np.zeros((dv, N)) if hist is None else hist
    lib().orc_vegas_accumulate(r, r.shape[1], w, r.shape[0], dv, N, hist)
    return hist


def vegas_rebin(hist, edges, alpha=1.5):
    hist = np.ascontiguousarray(hist, dtype=np.float64)
    edges = np.ascontiguousarray(edges, dtype=np.float64)
    out = np.zeros_like(edges)
    for j in range(edges.shape[0]):
        o = np.zeros(edges.shape[1])
        lib().orc_vegas_rebin(np.ascontiguousarray(hist[j]), np.ascontiguousarray(edges[j]), o,
                              edges.shape[1] - 1, alpha)
        out[j] = o
    return out
