"""Synthetic workloads: channel topologies and seeded inputs.

This module holds only *descriptions* -- which particles, propagators and
building blocks make up each channel, with their masses, widths and map
exponents -- and seeded random inputs.  It contains none of the phase-space
arithmetic; both the CUDA path (through the graph builder) and the FP64
oracle read these plain dictionaries.

Channel dictionary
------------------
``n``          final-state multiplicity
``hadronic``   True: the PDF convolution of Sec. 2.2.2 (shat map, r_to_x1x2,
               boost_beam); False: fixed partonic energy ``sqrt_s``
``S``          hadronic beam invariant (sqrt(S) = 13 TeV)
``a``          auxiliary shift m^2 = -a for massless maps (Sec. 2.2.1)
``shat``       map of shat: ``{"M", "G", "nu"}`` (Breit-Wigner if G > 0)
``t_nu``       exponent of the |t| power-law map (Eq. 2_to_2_mapping)
``ts_nu``      exponent for the t-chain invariants s_i (Sec. 2.2.8)
``Mt``         t-channel propagator mass used in the multichannel weights
``pdf``        (alpha, beta) of the synthetic parton density x^alpha (1-x)^beta
``integrand``  "none" | "one_plus_cos2" | "pdf_props" | "pdf_sde"
``vegas_dims`` number of leading random dimensions mapped by VEGAS
``nodes``      topology tree, node 0 = root (the shat invariant):
               {"kind": "leaf", "leaf": i, "mass": m}
               {"kind": "decay", "children": [c1, c2], "M", "G", "nu", "sde"}
               {"kind": "tchain", "children": [legs from leg A to leg B]}
``sorder``     decay nodes (excluding the root) in s-invariant sampling order
``tside``      t-chain: for steps 1..kappa-1, 0 = take the leg next to A, 1 = next to B
"""
from __future__ import annotations

import copy

import numpy as np

SQRT_S_LHC = 13000.0
S_LHC = SQRT_S_LHC * SQRT_S_LHC
A_SHIFT = 1.0e-4      # GeV^2, auxiliary negative mass^2 of massless maps
NU_DEFAULT = 0.8      # default power-law exponent (Sec. 2.2.1)
M_W, G_W = 80.4, 2.1
M_Z, G_Z = 91.2, 2.5
M_H, G_H = 125.0, 0.004
M_T, G_T = 173.0, 1.4
PDF_ALPHA, PDF_BETA = -1.1, 3.0


class _Tree:
    """Tiny helper that turns nested tuples into the flat node list."""

    def __init__(self):
        self.nodes = []

    def add(self, spec):
        kind = spec[0]
        idx = len(self.nodes)
        self.nodes.append(None)
        if kind == "leaf":
            _, leaf, mass = spec
            self.nodes[idx] = {"kind": "leaf", "leaf": leaf, "mass": float(mass)}
        elif kind == "decay":
            _, M, G, nu, sde, c1, c2 = spec
            kids = [self.add(c1), self.add(c2)]
            self.nodes[idx] = {"kind": "decay", "children": kids, "M": float(M), "G": float(G),
                               "nu": float(nu), "sde": bool(sde)}
        elif kind == "tchain":
            kids = [self.add(c) for c in spec[1]]
            self.nodes[idx] = {"kind": "tchain", "children": kids}
        else:
            raise ValueError(kind)
        return idx


def leaf(i, m=0.0):
    return ("leaf", i, m)


def decay(M, G, c1, c2, nu=NU_DEFAULT, sde=True):
    """s-channel 1->2 node; Breit-Wigner if G > 0, else power law (exponent nu)."""
    return ("decay", M, G, nu, sde, c1, c2)


def tchain(*legs):
    return ("tchain", list(legs))


def _preorder_decays(nodes, j=0, out=None):
    out = [] if out is None else out
    nd = nodes[j]
    if nd["kind"] == "decay" and j != 0:
        out.append(j)
    for c in nd.get("children", []):
        _preorder_decays(nodes, c, out)
    return out


def make_channel(root, n, *, hadronic=True, sqrt_s=None, shat=None, integrand="none",
                 vegas_dims=0, vegas_bins=64, t_nu=NU_DEFAULT, ts_nu=NU_DEFAULT, Mt=M_W,
                 sorder=None, tside=None, a=A_SHIFT, name=""):
    tr = _Tree()
    tr.add(root)
    nodes = tr.nodes
    if nodes[0]["kind"] == "decay":
        nodes[0]["sde"] = False
    if sorder is None:
        sorder = _preorder_decays(nodes)
    kappa = len(nodes[0]["children"]) - 1 if nodes[0]["kind"] == "tchain" else 0
    if tside is None:
        tside = [0] * max(kappa - 1, 0)
    return {
        "name": name, "n": n, "hadronic": bool(hadronic),
        "sqrt_s": float(sqrt_s) if sqrt_s is not None else 0.0,
        "S": S_LHC, "a": a,
        "shat": dict(shat) if shat is not None else {"M": 0.0, "G": 0.0, "nu": 1.0},
        "t_nu": t_nu, "ts_nu": ts_nu, "Mt": Mt, "pdf": (PDF_ALPHA, PDF_BETA),
        "integrand": integrand, "vegas_dims": vegas_dims, "vegas_bins": vegas_bins,
        "nodes": nodes, "sorder": list(sorder), "tside": list(tside),
    }


def n_random_dims(ch):
    """3n-2 for hadronic channels, 3n-4 at fixed energy (Sec. 2.2)."""
    return 3 * ch["n"] - (2 if ch["hadronic"] else 4)


# --------------------------------------------------------------------------
# The configurations
# --------------------------------------------------------------------------
def two_body_fixed(sqrt_s=1000.0, integrand="one_plus_cos2"):
    """Massless 2->2 at fixed sqrt(s) = 1000 GeV: one two_body_decay of the
    partonic system at rest, (phi, cos theta) from r in [0,1]^2."""
    return make_channel(decay(0.0, 0.0, leaf(0), leaf(1)), 2, hadronic=False, sqrt_s=sqrt_s,
                        integrand=integrand, name="2to2_fixed")


def ww_hadronic(vegas_dims=8):
    """Hadronic 2->4 at sqrt(S) = 13 TeV: shat with 1/tau sampling (nu = 1 log map
    with the auxiliary shift, range [0, S]), shat -> W W, each W a Breit-Wigner
    (80.4, 2.1) decaying to two massless particles; integrand = f(x1) f(x2) x the
    two W propagators; VEGAS on the first 8 of the 10 dimensions."""
    root = decay(0.0, 0.0, decay(M_W, G_W, leaf(0), leaf(1)), decay(M_W, G_W, leaf(2), leaf(3)))
    return make_channel(root, 4, hadronic=True, integrand="pdf_props", vegas_dims=vegas_dims,
                        name="ww_2to4")


def multichannel_2to5():
    """Six 2->5 channels with t-chains and resonances (all final states massless)."""
    Z = lambda a, b: decay(M_Z, G_Z, leaf(a), leaf(b))
    H = lambda a, b: decay(M_H, G_H, leaf(a), leaf(b))
    T = lambda a, b: decay(M_T, G_T, leaf(a), leaf(b))
    chans = [
        make_channel(tchain(leaf(0), leaf(1), leaf(2), leaf(3), leaf(4)), 5, integrand="pdf_sde",
                     name="ch0_t4"),
        make_channel(tchain(Z(0, 1), leaf(2), leaf(3), leaf(4)), 5, integrand="pdf_sde", name="ch1_Z_t3"),
        make_channel(tchain(H(0, 1), leaf(2), leaf(3), leaf(4)), 5, integrand="pdf_sde", name="ch2_H_t3",
                     tside=[1, 0]),
        make_channel(tchain(T(0, 1), Z(2, 3), leaf(4)), 5, integrand="pdf_sde", name="ch3_TZ_t2"),
        make_channel(decay(0.0, 0.0, Z(0, 1), decay(0.0, 0.0, T(2, 3), leaf(4), sde=False)), 5,
                     integrand="pdf_sde", name="ch4_s"),
        make_channel(tchain(Z(0, 1), H(2, 3), leaf(4)), 5, integrand="pdf_sde", name="ch5_ZH_t2"),
    ]
    return chans


MULTICHANNEL_EVENTS = [100_000, 4_000_000, 4_000_000, 4_000_000, 4_000_000, 3_900_000]

C5_MASSES = [0.0] * 6 + [M_T, M_T]   # 2->8: six massless and two top-mass final-state particles
C5_EVENTS = 100_000_000               # streamed in chunks of C5_CHUNK
C5_CHUNK = 1 << 22


def channels_2to8(n_channels=24, seed=1005):
    """Channels of the hadronic 2->8 process (six massless particles, two of mass 173 GeV), mixing
    t-chains and pure s-channel trees, drawn deterministically from `seed`: every third channel is
    one binary s-channel tree of all eight particles; the others are t-chains of 3-6 clusters,
    each cluster of two or more particles a binary decay tree.  An internal node is a resonance
    (W, Z, H or top, Breit-Wigner, in the SDE weights) with probability 1/2, else a massless
    power-law node; the t-chain legs are taken from side A or B at random.  Integrand: PDFs times
    the SDE channel sum, as in the 2->5 workload."""
    rng = np.random.default_rng(seed)
    res = [(M_W, G_W), (M_Z, G_Z), (M_H, G_H), (M_T, G_T)]

    def tree(parts):
        if len(parts) == 1:
            return leaf(int(parts[0]), C5_MASSES[int(parts[0])])
        cut = int(rng.integers(1, len(parts)))
        left, right = tree(parts[:cut]), tree(parts[cut:])
        if rng.random() < 0.5:
            M, G = res[int(rng.integers(len(res)))]
            return decay(M, G, left, right)
        return decay(0.0, 0.0, left, right, sde=False)

    chans = []
    for c in range(n_channels):
        legs = [int(x) for x in rng.permutation(8)]
        if c % 3 == 2:
            root = tree(legs)
            root = ("decay", 0.0, 0.0, NU_DEFAULT, False, root[5], root[6]) if root[0] == "decay" else root
            tside = None
        else:
            m = int(rng.integers(3, 7))
            cuts = sorted(int(x) for x in rng.choice(np.arange(1, 8), m - 1, replace=False))
            groups = [legs[a:b] for a, b in zip([0] + cuts, cuts + [8])]
            root = tchain(*[tree(gr) for gr in groups])
            tside = [int(x) for x in rng.integers(0, 2, m - 2)]
        chans.append(make_channel(root, 8, integrand="pdf_sde", tside=tside, name=f"c5_{c:02d}"))
    return chans


def volume_topologies(n=4, sqrt_s=1000.0, nu=0.3):
    """Massless 2->n at fixed energy with every invariant on the power law with
    exponent nu (Sec. 4.1): pure t-chain, mixed t/s, pure s."""
    out = []
    legs = [leaf(i) for i in range(n)]
    out.append(make_channel(tchain(*legs), n, hadronic=False, sqrt_s=sqrt_s, t_nu=nu, ts_nu=nu,
                            name=f"pure_t_{n}"))
    if n == 4:
        mixed = tchain(decay(0.0, 0.0, leaf(0), leaf(1), nu=nu, sde=False),
                       decay(0.0, 0.0, leaf(2), leaf(3), nu=nu, sde=False))
        pure_s = decay(0.0, 0.0, decay(0.0, 0.0, leaf(0), leaf(1), nu=nu, sde=False),
                       decay(0.0, 0.0, leaf(2), leaf(3), nu=nu, sde=False))
    elif n == 3:
        mixed = tchain(decay(0.0, 0.0, leaf(0), leaf(1), nu=nu, sde=False), leaf(2))
        pure_s = decay(0.0, 0.0, decay(0.0, 0.0, leaf(0), leaf(1), nu=nu, sde=False), leaf(2))
    else:
        raise ValueError(n)
    out.append(make_channel(mixed, n, hadronic=False, sqrt_s=sqrt_s, t_nu=nu, ts_nu=nu, name=f"mixed_{n}"))
    out.append(make_channel(pure_s, n, hadronic=False, sqrt_s=sqrt_s, t_nu=nu, ts_nu=nu, name=f"pure_s_{n}"))
    return out


def with_masses(ch, masses):
    """Copy of a channel with the given final-state masses on its leaves."""
    ch = copy.deepcopy(ch)
    for nd in ch["nodes"]:
        if nd["kind"] == "leaf":
            nd["mass"] = float(masses[nd["leaf"]])
    return ch


# --------------------------------------------------------------------------
# Seeded inputs
# --------------------------------------------------------------------------
def uniform_r(seed, B, d, edge_fraction=0.0):
    """Seeded uniform points in (0,1)^d, shape [B, d] (float64).  With
    edge_fraction > 0 that share of the coordinates is pushed to within 1e-9 of
    0 or 1, to exercise the edges of the maps."""
    rng = np.random.default_rng(seed)
    r = rng.random((B, d))
    r = np.clip(r, 2.0 ** -53, 1.0 - 2.0 ** -53)
    if edge_fraction > 0.0:
        m = rng.random((B, d)) < edge_fraction
        side = rng.random((B, d)) < 0.5
        tiny = rng.random((B, d)) * 1e-9 + 2.0 ** -53
        r = np.where(m & side, tiny, r)
        r = np.where(m & ~side, 1.0 - tiny, r)
    return r


def vegas_grid_random(seed, dims, bins):
    """Seeded non-uniform VEGAS edges [dims][bins+1] with e_0 = 0, e_N = 1."""
    rng = np.random.default_rng(seed)
    w = rng.random((dims, bins)) + 0.05
    e = np.zeros((dims, bins + 1))
    e[:, 1:] = np.cumsum(w, axis=1)
    e /= e[:, -1:]
    e[:, -1] = 1.0
    return e


def vegas_grid_uniform(dims, bins):
    e = np.tile(np.arange(bins + 1, dtype=np.float64) / bins, (dims, 1))
    return e
