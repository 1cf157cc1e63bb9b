"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.

Tolerances (stated per quantity; the derivation is in the design notes):
  momenta   |p_gpu - p_orc| <= max(1e-12, 32 eps kappa_p) * (largest energy of the event), per
            component; kappa_p is the oracle's rounding amplification: kappa of a decay or block at
            threshold, |t|_max/(|t|_max - |t|) for backward 2->2 scattering (1 + cos(theta) from
            |t|_max - |t|) -- both reach the later legs of a t-chain -- and gamma^2 = E0^2/s of a
            boost into the rest frame of a composite momentum (its components and its sampled
            invariant agree only to eps E0^2) -- the small-s, small-t tail of the paper's Sec. 4.1
  x1, x2    relative 1e-12
  weight    relative max(1e-12, 32 eps kappa): kappa is the oracle's per-event condition number
            (a sampled range width sqrt(s_r)/(m_max - m_min), or a decay/block at threshold
            s/(s - (m1+m2)^2)); two correct FP64 evaluations cannot agree better than eps kappa
            there.  For ~98% of events the 1e-12 floor applies.  Zero weights agree exactly.
  alpha     relative 1e-12, or the conditioning bound of a propagator evaluated from
            momenta (see _alpha_tolerance)
  integers  (cut decisions, counts, VEGAS bin indices, Philox bits) bit-exact
  spread    the analytic kappa assumes inputs good to an ulp; nested sliver ranges compound the
            libm differences of earlier invariants (a range spanning many decades gives its top
            end ~|exponent| ulps, which the next sliver range amplifies).  The oracle's own
            rounding sensitivity is therefore also measured by stochastic arithmetic
            (oracle.rounding_spread: 8 re-runs with every elementary-function result moved by up
            to 2 ulps -- CUDA's double functions are within 1-2 ulps of the exact value, glibc's
            within about 1) and every per-event bound above is at least 4x that spread; a zero
            weight may differ where a perturbed run of the oracle also changes it.
In addition, at least 99% of the events whose random numbers are not pushed to within 1e-8 of
0 or 1 meet the bounds without their safety factors -- max(1e-12, 4 eps kappa, spread) on
weights and momenta: the bulk must agree as closely as two roundings of the oracle do, and
only a tail may use the factor 32 and the factor 4 on the spread.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2602_06895_gb300 import ps
from paper_2602_06895_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RTOL = 1e-12
EPS = 2.0 ** -52


def weight_tol(orc, spread=None):
    t = np.maximum(RTOL, 32.0 * EPS * orc["aux"][:, O.AUX["cond"]])
    return t if spread is None else np.maximum(t, 4.0 * spread["w"])


def momentum_tol(orc, spread=None):
    t = np.maximum(RTOL, 32.0 * EPS * orc["aux"][:, O.AUX["cond_p"]])
    return t if spread is None else np.maximum(t, 4.0 * spread["mom"])


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2602_06895_gb300 import build

    build.build()
    return torch


def run_map(torch, channels, which, r, grid=None, block=128, jit=False):
    """Explicit-input map of channel `which` on the GPU; r [B, d] numpy."""
    prog = ps.program_for(channels, block_threads=block, jit=jit)
    ch = channels[which]
    if grid is not None:
        prog.set_vegas(which, grid)
    B = r.shape[0]
    n_mom = ch["n"] + 2
    out, ws = prog.alloc([B if c == which else 0 for c in range(len(channels))], n_mom, x=ch["hadronic"],
                         alpha=ch["integrand"] == "pdf_sde")
    rt = torch.from_numpy(np.ascontiguousarray(r.T)).to("cuda")
    prog.map(which, rt, out, ws)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res["mom"] = res["momenta"][:, :B].reshape(n_mom, 4, B).transpose(2, 0, 1)
    res["w"] = res["weight"][:B]
    if "x1" in res:
        res["x"] = np.stack([res["x1"][:B], res["x2"][:B]], axis=1)
    if "alpha" in res:
        res["alpha"] = res["alpha"][:B]
    res["stats"] = prog.stats()[which]
    res["status"] = prog.status()
    return res


def compare(gpu, orc, ch, label, alpha_tol=None, r=None, spread=None):
    mom_g, mom_o = gpu["mom"], orc["mom"]
    scale = np.max(np.abs(mom_o[:, :, 0]), axis=1)
    # zero weights (cuts, empty ranges) are integer outcomes and must agree -- except at an exact
    # threshold, where the weight itself is undetermined (its bound reaches 1, or a perturbed
    # rounding of the oracle changes it too)
    bad = np.flatnonzero((gpu["w"] == 0) != (orc["w"] == 0))
    n_threshold = 0
    if "aux" in orc:
        undetermined = weight_tol(orc, spread) >= 1.0
        if spread is not None:
            undetermined |= spread["flip"]
        n_threshold = int(np.sum(undetermined[bad]))
        bad = bad[~undetermined[bad]]
    assert bad.size == 0, (label, "zero weights differ", bad[:5].tolist(), gpu["w"][bad[:5]].tolist(),
                           orc["w"][bad[:5]].tolist(), orc["aux"][bad[:5]].tolist() if "aux" in orc else None)
    ok = (orc["w"] != 0) & (gpu["w"] != 0)
    dm = np.max(np.abs(mom_g - mom_o), axis=(1, 2))
    ptol = momentum_tol(orc, spread)[ok] if "aux" in orc else RTOL
    # the bulk: the per-event bounds without their safety factors (spread x1, kappa x4)
    bulk_w, bulk_p, need = RTOL, RTOL, 0.95
    if "aux" in orc:
        bulk_w = np.maximum(RTOL, 4.0 * EPS * orc["aux"][ok, O.AUX["cond"]])
        bulk_p = np.maximum(RTOL, 4.0 * EPS * orc["aux"][ok, O.AUX["cond_p"]])
        need = 0.99
        if spread is not None:
            bulk_w = np.maximum(bulk_w, spread["w"][ok])
            bulk_p = np.maximum(bulk_p, spread["mom"][ok])
    bulk_ok = (dm[ok] <= bulk_p * scale[ok]) & (np.abs(gpu["w"][ok] / orc["w"][ok] - 1.0) <= bulk_w)
    interior = np.ones(ok.sum(), bool) if r is None else np.all((r[ok] > 1e-8) & (r[ok] < 1 - 1e-8), axis=1)
    frac = float(bulk_ok[interior].mean()) if interior.any() else 1.0
    assert frac >= need, (label, "fraction of interior events within the bulk bar", frac)
    ratio = dm[ok] / (ptol * scale[ok])
    worst = int(np.flatnonzero(ok)[np.argmax(ratio)])
    assert np.all(ratio <= 1.0), (label, "momenta", "worst event", worst, "rel err", dm[worst] / scale[worst],
                                  "bound ratio", float(ratio.max()), int(np.sum(dm[ok] > RTOL * scale[ok])))
    if ch["hadronic"]:
        rx = np.abs(gpu["x"] / orc["x"] - 1.0)
        assert np.all(rx[ok] <= RTOL), (label, "x", rx[ok].max())
    rw = np.abs(gpu["w"][ok] / orc["w"][ok] - 1.0)
    tol = weight_tol(orc, spread)[ok]
    assert np.all(rw <= tol), (label, "weight", "worst event", int(np.flatnonzero(ok)[np.argmax(rw / tol)]),
                               float(np.max(rw / tol)), rw.max(), int(np.sum(rw > RTOL)))
    if alpha_tol is not None:
        ra = np.abs(gpu["alpha"][ok] - orc["alpha"][ok])
        bound = alpha_tol[ok] * np.maximum(orc["alpha"][ok], 1e-300) + 1e-300
        k = int(np.argmax(ra / bound))
        assert np.all(ra <= bound), (label, "alpha", "worst", int(np.flatnonzero(ok)[k]), float(orc["alpha"][ok][k]),
                                     float(gpu["alpha"][ok][k]), float((ra / bound)[k]),
                                     float(orc["aux"][ok][k, O.AUX["cond_p"]]) if "aux" in orc else None)
    return n_threshold


def parity_channels():
    out = [("2to2_fixed", [W.two_body_fixed()], 0, None),
           ("2to2_fixed_none", [W.two_body_fixed(integrand="none")], 0, None),
           ("ww_2to4", [W.ww_hadronic()], 0, W.vegas_grid_random(11, 8, 64))]
    for t in W.volume_topologies(3) + W.volume_topologies(4):
        out.append((t["name"], [t], 0, None))
        m = W.with_masses(t, [173.0, 173.0] + [0.0] * (t["n"] - 2))
        out.append((t["name"] + "_massive", [m], 0, None))
    multi = W.multichannel_2to5()
    for i in range(len(multi)):
        out.append((multi[i]["name"], multi, i, None))
    c5 = W.channels_2to8()
    for i in range(len(c5)):
        out.append((c5[i]["name"], c5, i, None))
    return out


def _alpha_tolerance(orc, spread=None):
    # alpha_c = P_c / sum_j P_j with the other channels' P_j from momenta.  A propagator
    # 1/((s-M^2)^2 + M^2 G^2) evaluated from momenta inherits the rounding of s = (sum p)^2:
    # the momenta agree to 32 eps kappa_p E (E the event's energy scale), so s to ~4 of that
    # times E, and P_j moves by that over M G near its peak -- at worst the Higgs, M G = 0.5 GeV^2.
    # alpha moves by at most (1 - alpha) times the relative change of the other channels' sum.
    a = orc["alpha"]
    e = np.max(np.abs(orc["mom"][:, :, 0]), axis=1)
    kp = np.maximum(1.0, orc["aux"][:, O.AUX["cond_p"]])
    rel_s = 4.0 * 32.0 * EPS * kp * e * e / 0.5
    t = np.maximum(RTOL, np.minimum(1.0, rel_s) * (1.0 - a))
    return t if spread is None else np.maximum(t, 4.0 * spread["alpha"])


def _flat_agreement(a, orc, interior):
    """Per event (both weights nonzero, random numbers inside [1e-8, 1-1e-8]): whether every
    momentum component agrees with the oracle within 1e-12 of the event's largest energy and the
    weight within 1e-12 relative -- the flat bar, with no condition number."""
    ok = (a["w"] != 0) & (orc["w"] != 0) & interior
    scale = np.max(np.abs(orc["mom"][:, :, 0]), axis=1)
    dm = np.max(np.abs(a["mom"] - orc["mom"]), axis=(1, 2))
    rw = np.abs(a["w"] / np.where(orc["w"] != 0, orc["w"], 1.0) - 1.0)
    return ok, (dm <= RTOL * scale) & (rw <= RTOL)


# The flat 1e-12 bar against a second FP64 evaluation of the same formulas: the oracle compiled
# with contracted multiply-adds (as the GPU evaluates them) and with every elementary-function
# result moved by a random whole number of ulps in [-2, 2] (CUDA's double functions are within
# 1-2 ulps, glibc's within about 1).  The GPU may miss the flat bar on at most twice as many
# events as that evaluation does (mean of two seeds), plus 0.5 % of the events; and on at most
# 8 percentage points more events than the contracted oracle alone, where the host compiler
# contracts at all.  Measured on the GB300 over these workloads when the bounds were set: the
# ratio of misses at most 1.74 (one 2->8 channel; 1.2 or less elsewhere), the excess over the
# contracted oracle at most 7.1 points.  (A Breit-Wigner tangent of 3-5 ulps, tried later, put
# one 2->8 channel 12 points below the contracted oracle; these bounds caught it.)
FLAT_MISS_RATIO, FLAT_MISS_SLACK, FLAT_FMA_MARGIN = 2.0, 0.005, 0.08


@pytest.mark.parametrize("case", parity_channels(), ids=lambda c: c[0])
def test_explicit_input_parity(torch_cuda, case):
    name, chans, which, grid = case
    ch = chans[which]
    d = O.dims(ch)
    # 4999 events: 39 full tiles of 128 and a ragged tail; 2% of coordinates near 0 or 1
    r = W.uniform_r(4242 + which, 4999, d, edge_fraction=0.02)
    gpu = run_map(torch_cuda, chans, which, r, grid=grid)
    orc = O.forward(ch, r, grid=grid, channels=chans, chan=which, aux=True)
    spread = O.rounding_spread(ch, r, grid=grid, channels=chans, chan=which, base=orc)
    at = _alpha_tolerance(orc, spread) if ch["integrand"] == "pdf_sde" else None
    n_thr = compare(gpu, orc, ch, name, alpha_tol=at, r=r, spread=spread)
    # the flat-bar fraction against the second FP64 evaluation and the contracted oracle
    interior = np.all((r > 1e-8) & (r < 1 - 1e-8), axis=1)
    ok_g, flat_g = _flat_agreement(gpu, orc, interior)
    miss_ref = []
    for seed in (1, 2):
        ok_p, flat_p = _flat_agreement(O.forward_fma_perturbed(ch, r, seed, grid=grid, channels=chans, chan=which),
                                       orc, interior)
        m = ok_p & ok_g
        miss_ref.append(1.0 - float(flat_p[m].mean()))
    miss_gpu = 1.0 - float(flat_g[ok_g].mean())
    assert miss_gpu <= FLAT_MISS_RATIO * np.mean(miss_ref) + FLAT_MISS_SLACK, (name, miss_gpu, miss_ref)
    fma = O.forward_fma(ch, r, grid=grid, channels=chans, chan=which)
    if not np.array_equal(fma["w"], orc["w"]):  # the host compiler contracted multiply-adds
        ok_f, flat_f = _flat_agreement(fma, orc, interior)
        m = ok_f & ok_g
        assert float(flat_g[m].mean()) >= float(flat_f[m].mean()) - FLAT_FMA_MARGIN, (name, "vs contracted oracle")
    st = O.stats(orc["w"])
    s = gpu["stats"]
    assert s["n"] == st["n"] and abs(s["n_nonzero"] - st["n_nonzero"]) <= n_thr
    for k in ("sum_w", "sum_w2", "max_w"):
        assert abs(s[k] - st[k]) <= max(RTOL, float(np.max(weight_tol(orc, spread)))) * abs(st[k]), (name, k)


@pytest.mark.parametrize("B", [0, 1, 31, 33, 127, 128, 129, 1000])
def test_ragged_sizes(torch_cuda, B):
    ch = W.ww_hadronic()
    grid = W.vegas_grid_random(12, 8, 64)
    r = W.uniform_r(77 + B, max(B, 1), 10)[:B]
    if B == 0:
        prog = ps.program_for([ch])
        out, ws = prog.alloc([1], 6)
        rt = torch_cuda.zeros((10, 1), dtype=torch_cuda.float64, device="cuda")[:, :0]
        prog.map(0, rt.contiguous() if rt.numel() else torch_cuda.zeros((10, 1), dtype=torch_cuda.float64,
                                                                          device="cuda")[:, :0], out, ws)
        torch_cuda.cuda.synchronize()
        assert prog.stats()[0]["n"] == 0.0 and prog.stats()[0]["sum_w"] == 0.0
        return
    gpu = run_map(torch_cuda, [ch], 0, r, grid=grid)
    orc = O.forward(ch, r, grid=grid, aux=True)
    compare(gpu, orc, ch, f"B={B}")


@pytest.mark.parametrize("block", [32, 64, 256])
def test_block_sizes(torch_cuda, block):
    ch = W.multichannel_2to5()
    r = W.uniform_r(90 + block, 777, 13)
    gpu = run_map(torch_cuda, ch, 3, r, block=block)
    orc = O.forward(ch[3], r, channels=ch, chan=3, aux=True)
    compare(gpu, orc, ch[3], f"block={block}", alpha_tol=_alpha_tolerance(orc))


def test_philox_bits_exact(torch_cuda):
    """The in-kernel Philox4x32-10 stream is bit-identical to the oracle's."""
    d = 13
    for j in (0, 1, 6, 12):
        g = ps.Graph.create(d)
        (v,) = g.add("REDUCE_PRODUCT", [j], 1)
        g.set_outputs([v], [ps.ROLE_WEIGHT])
        prog = ps.Program([g])
        B = 3000
        w = torch_cuda.empty(B, dtype=torch_cuda.float64, device="cuda")
        ws = torch_cuda.empty(prog.workspace_size([B]) // 8 + 32, dtype=torch_cuda.float64, device="cuda")
        prog.generate([B], 0x1234_5678_9ABC_DEF0, {"weight": w}, ws, event_offset=(1 << 32) - 1000)
        torch_cuda.cuda.synchronize()
        ref = O.random(0x1234_5678_9ABC_DEF0, 0, (1 << 32) - 1000, B, d)[:, j]
        assert np.array_equal(w.cpu().numpy().view(np.uint64), ref.view(np.uint64)), j


def test_generate_parity_single_channel(torch_cuda):
    ch = W.ww_hadronic()
    grid = W.vegas_grid_random(13, 8, 64)
    prog = ps.program_for([ch])
    prog.set_vegas(0, grid)
    B = 20_011
    out, ws = prog.alloc([B], 6)
    prog.generate([B], 1002, out, ws, event_offset=5)
    torch_cuda.cuda.synchronize()
    orc = O.forward(ch, O.random(1002, 0, 5, B, 10), grid=grid, aux=True)
    gpu = {"mom": out["momenta"].cpu().numpy().reshape(6, 4, B).transpose(2, 0, 1),
           "x": np.stack([out["x1"].cpu().numpy(), out["x2"].cpu().numpy()], axis=1),
           "w": out["weight"].cpu().numpy()}
    compare(gpu, orc, ch, "generate")


def test_generate_parity_multichannel(torch_cuda):
    chans = W.multichannel_2to5()
    counts = [257, 1000, 3, 0, 640, 1501]
    prog = ps.program_for(chans)
    out, ws = prog.alloc(counts, 7, alpha=True)
    prog.generate(counts, 1003, out, ws)
    torch_cuda.cuda.synchronize()
    tot = sum(counts)
    mom = out["momenta"].cpu().numpy().reshape(7, 4, tot).transpose(2, 0, 1)
    stats = prog.stats()
    col = 0
    for c, n in enumerate(counts):
        if n:
            orc = O.forward(chans[c], O.random(1003, c, 0, n, 13), channels=chans, chan=c, aux=True)
            sl = slice(col, col + n)
            gpu = {"mom": mom[sl], "w": out["weight"].cpu().numpy()[sl],
                   "x": np.stack([out["x1"].cpu().numpy()[sl], out["x2"].cpu().numpy()[sl]], axis=1),
                   "alpha": out["alpha"].cpu().numpy()[sl]}
            compare(gpu, orc, chans[c], chans[c]["name"], alpha_tol=_alpha_tolerance(orc))
            st = O.stats(orc["w"])
            assert stats[c]["n_nonzero"] == st["n_nonzero"]
            assert abs(stats[c]["sum_w"] - st["sum_w"]) <= RTOL * st["sum_w"]
        else:
            assert stats[c]["n"] == 0 and stats[c]["sum_w"] == 0
        col += n


def test_determinism_and_partition_invariance(torch_cuda):
    ch = W.ww_hadronic()
    prog = ps.program_for([ch])
    N = 10_000
    a, ws = prog.alloc([N], 6)
    prog.generate([N], 7, a, ws)
    b, _ = prog.alloc([N], 6)
    prog.generate([N], 7, b, ws)
    h1, _ = prog.alloc([N // 2], 6)
    h2, _ = prog.alloc([N - N // 2], 6)
    prog.generate([N // 2], 7, h1, ws, event_offset=0)
    prog.generate([N - N // 2], 7, h2, ws, event_offset=N // 2)
    torch_cuda.cuda.synchronize()
    for k in ("momenta", "weight", "x1"):
        assert torch_cuda.equal(a[k], b[k])
    joined = torch_cuda.cat([h1["weight"], h2["weight"]])
    assert torch_cuda.equal(a["weight"], joined)


def test_vegas_training_histogram_and_rebin(torch_cuda):
    ch = W.ww_hadronic()
    grid = W.vegas_grid_random(21, 8, 64)
    prog = ps.program_for([ch])
    prog.set_vegas(0, grid)
    prog.vegas_training(True)
    B = 50_000
    out, ws = prog.alloc([B], 6)
    prog.generate([B], 31, out, ws)
    torch_cuda.cuda.synchronize()
    hist = prog.vegas_histogram(0, 8)
    r = O.random(31, 0, 0, B, 10)
    orc = O.forward(ch, r, grid=grid)
    ref = O.vegas_accumulate(r, orc["w"], 8, 64)
    nz = ref > 0
    assert np.array_equal(hist > 0, nz)
    assert np.all(np.abs(hist[nz] / ref[nz] - 1.0) <= 1e-12)
    prog.vegas_adapt(0, alpha=1.5)
    new = prog.get_vegas(0, 8)
    ref_new = O.vegas_rebin(ref, grid, alpha=1.5)
    assert np.max(np.abs(new - ref_new)) <= 1e-12
    assert np.all(prog.vegas_histogram(0, 8) == 0.0)


def test_vegas_adaptation_bit_reproducible(torch_cuda):
    """VEGAS training sums the histogram in a fixed order: three adaptation rounds give the same
    grid bit for bit when repeated, also with another block size and as a compiled program, and
    a multichannel histogram does not depend on the launch shape either."""
    ch = W.ww_hadronic()

    def adapt(block, jit):
        prog = ps.program_for([ch], block_threads=block, jit=jit)
        prog.vegas_training(True)
        B = 300_001
        out, ws = prog.alloc([B], 6)
        hists = []
        for it in range(3):
            prog.generate([B], 90 + it, out, ws)
            torch_cuda.cuda.synchronize()
            hists.append(prog.vegas_histogram(0, 8))
            prog.vegas_adapt(0, alpha=1.5)
        return prog.get_vegas(0, 8), hists

    g0, h0 = adapt(128, False)
    for block, jit in ((128, False), (64, False), (256, True)):
        g, h = adapt(block, jit)
        assert np.array_equal(g, g0), (block, jit)
        for a, b in zip(h, h0):
            assert np.array_equal(a, b), (block, jit)
    chans = W.multichannel_2to5()
    vch = [dict(c, vegas_dims=6) for c in chans]
    counts = [1000, 20_000, 0, 7_777, 130, 50_000]
    res = []
    for block, cps in ((128, 0), (64, 3)):
        prog = ps.program_for(vch, block_threads=block, ctas_per_sm=cps)
        prog.vegas_training(True)
        out, ws = prog.alloc(counts, 7, alpha=True)
        prog.generate(counts, 5, out, ws)
        torch_cuda.cuda.synchronize()
        res.append([prog.vegas_histogram(c, 6) for c in range(6)])
    for a, b in zip(*res):
        assert np.array_equal(a, b)
    assert np.all(res[0][2] == 0) and np.all(res[0][1] > 0)


def test_full_size_sampled(torch_cuda):
    """1e7 events of the 2->4 W W workload in the benchmark's launch configuration:
    sampled events against the oracle one by one, and the channel sums against a full
    oracle pass."""
    ch = W.ww_hadronic()
    grid = W.vegas_grid_random(41, 8, 64)
    prog = ps.program_for([ch])
    prog.set_vegas(0, grid)
    N = 10_000_000
    out, ws = prog.alloc([N], 6)
    prog.generate([N], 1002, out, ws)
    torch_cuda.cuda.synchronize()
    rng = np.random.default_rng(5)
    idx = np.sort(rng.choice(N, 3000, replace=False))
    idx = np.concatenate([idx, [0, 1, N - 2, N - 1]])
    w = out["weight"].cpu().numpy()
    mom = out["momenta"][:, idx].cpu().numpy().reshape(6, 4, idx.size).transpose(2, 0, 1)
    x = np.stack([out["x1"][idx].cpu().numpy(), out["x2"][idx].cpu().numpy()], axis=1)
    r = np.vstack([O.random(1002, 0, int(i), 1, 10) for i in idx])
    orc = O.forward(ch, r, grid=grid, aux=True)
    compare({"mom": mom, "x": x, "w": w[idx]}, orc, ch, "full-size")
    full = O.generate(ch, 1002, 0, N, grid=grid, keep_momenta=False)
    s = prog.stats()[0]
    assert s["n_nonzero"] == np.count_nonzero(full["w"])
    # channel sums against the exactly rounded sums of the oracle's weights; the allowance is
    # the sum of the per-event weight bounds, estimated on the sampled events (x3)
    est = float(np.sum(weight_tol(orc) * orc["w"]) / np.sum(orc["w"]))
    s1 = math.fsum(full["w"])
    s2 = math.fsum(full["w"] * full["w"])
    assert abs(s["sum_w"] - s1) <= (RTOL + 3 * est) * s1, (s["sum_w"] / s1 - 1, est)
    assert abs(s["sum_w2"] - s2) <= (RTOL + 6 * est) * s2, (s["sum_w2"] / s2 - 1, est)
    k = int(np.argmax(full["w"]))
    orc_k = O.forward(ch, O.random(1002, 0, k, 1, 10), grid=grid, aux=True)
    assert abs(s["max_w"] / full["w"][k] - 1.0) <= weight_tol(orc_k)[0]
    assert np.array_equal(w == 0, full["w"] == 0)
    assert prog.status()["nonfinite"] == 0
    assert prog.status()["cut"] == 0  # the stable forms leave cut_unphysical nothing to cut


def _multichannel_full_size(torch, chans, counts, seed, offset, block, ctas, per_channel, label):
    """One CUDA-graph launch of a multichannel program in the benchmark's configuration; sampled
    events of every channel against the oracle one by one (their Philox draws recomputed by the
    oracle), with the rounding-spread bounds."""
    prog = ps.program_for(chans, block_threads=block, ctas_per_sm=ctas)
    n_mom = chans[0]["n"] + 2
    out, ws = prog.alloc(counts, n_mom, alpha=True)
    ex = prog.exec_create(counts, out, ws)
    ex.launch(seed, offset)
    torch.cuda.synchronize()
    st = prog.stats()
    assert [s["n"] for s in st] == counts
    assert prog.status()["nonfinite"] == 0
    assert prog.status()["cut"] == 0  # the stable forms leave cut_unphysical nothing to cut
    rng = np.random.default_rng(seed)
    col = 0
    for c, n in enumerate(counts):
        ch = chans[c]
        d = O.dims(ch)
        loc = np.sort(rng.choice(n, min(per_channel, n), replace=False))
        loc = np.unique(np.concatenate([loc, [0, n - 1]]))
        cols = torch.from_numpy(col + loc).cuda()
        mom = out["momenta"][:, cols].cpu().numpy().reshape(n_mom, 4, loc.size).transpose(2, 0, 1)
        gpu = {"mom": mom, "w": out["weight"][cols].cpu().numpy(), "alpha": out["alpha"][cols].cpu().numpy(),
               "x": np.stack([out["x1"][cols].cpu().numpy(), out["x2"][cols].cpu().numpy()], axis=1)}
        r = np.vstack([O.random(seed, c, offset + int(j), 1, d) for j in loc])
        orc = O.forward(ch, r, channels=chans, chan=c, aux=True)
        sp = O.rounding_spread(ch, r, channels=chans, chan=c, base=orc)
        compare(gpu, orc, ch, f"{label} {ch['name']}", alpha_tol=_alpha_tolerance(orc, sp), spread=sp)
        col += n


def test_full_size_multichannel_2to5(torch_cuda):
    """2e7 events in six 2->5 channels with the benchmark's uneven counts, one persistent launch
    replayed from its CUDA graph (128 threads x 3 CTAs per SM, the autotuner's choice)."""
    _multichannel_full_size(torch_cuda, W.multichannel_2to5(), list(W.MULTICHANNEL_EVENTS), 1003, 0, 128, 3, 400,
                            "2->5 full size")


def test_full_size_streamed_chunk_2to8(torch_cuda):
    """One 2^22-event chunk of the streamed 2->8 workload (24 channels, the chunk of the third
    step of the stream) in the benchmark's launch configuration (64 threads x 4 CTAs per SM)."""
    chans = W.channels_2to8()
    chunk = W.C5_CHUNK
    counts = [chunk // 24 + (1 if c < chunk % 24 else 0) for c in range(24)]
    _multichannel_full_size(torch_cuda, chans, counts, 1005, 2 * chunk, 64, 4, 120, "2->8 chunk")


def test_azimuth_table_matches_quad_precision(torch_cuda):
    """The FP64 kernels' cos and sin of 2 pi r (a 256-point table and Taylor series of the
    remaining angle) agree with a quad- or extended-precision evaluation to 6 ulps of 1,
    over [0, 1] including the table points, the ends and their neighbours."""
    torch = torch_cuda
    rng = np.random.default_rng(42)
    grid = np.arange(257) / 256.0
    r = np.concatenate([rng.random(1 << 18), grid, np.nextafter(grid[1:], 0), np.nextafter(grid[:-1], 1),
                        [0.0, 1.0, 0.5, 0.25, 0.75, 1e-300, 5e-324]])
    rt = torch.from_numpy(r).cuda()
    out = torch.empty(2 * r.size, dtype=torch.float64, device="cuda")
    ps.mixed_helper("sincos_turn", rt, out)
    o = out.cpu().numpy().reshape(-1, 2)
    rl = r.astype(np.longdouble)
    pi = np.longdouble("3.14159265358979323846264338327950288")
    cl, sl = np.cos(2 * pi * rl), np.sin(2 * pi * rl)
    err = np.maximum(np.abs(o[:, 0] - cl), np.abs(o[:, 1] - sl)).astype(np.float64)
    assert err.max() < 6 * np.finfo(np.float64).eps, err.max()
    # outside [0, 1] the sincospi fallback
    rs = torch.tensor([-0.25, 1.5, -0.0], dtype=torch.float64, device="cuda")
    o2 = torch.empty(6, dtype=torch.float64, device="cuda")
    ps.mixed_helper("sincos_turn", rs, o2)
    o2 = o2.cpu().numpy().reshape(-1, 2)
    assert np.allclose(o2, [[0.0, -1.0], [-1.0, 0.0], [1.0, 0.0]], atol=1e-15)


def test_bw_tangent_matches_quad_precision(torch_cuda):
    """The FP64 Breit-Wigner map's tangent (a double-double table at k pi/512 and the Taylor
    series of the remainder) against a quad- or extended-precision tan over [-pi/4, pi/4], the
    table points and their neighbours: within 2 ulps of the result everywhere, and the correctly
    rounded double for at least 97 % of the arguments (as CUDA's and the host's tan nearly are)."""
    torch = torch_cuda
    rng = np.random.default_rng(43)
    q = np.pi / 4
    pts = np.arange(129) * (np.pi / 512)
    pts = pts[pts <= q]
    x = np.concatenate([rng.uniform(-q, q, 1 << 18), rng.uniform(-1e-3, 1e-3, 1 << 14), pts, -pts,
                        np.nextafter(pts[1:], 0), np.nextafter(pts[:-1], 1), [0.0, -0.0, 1e-300, -5e-324, q, -q]])
    xt = torch.from_numpy(x).cuda()
    out = torch.empty_like(xt)
    ps.mixed_helper("tan_quarter", xt, out)
    t = out.cpu().numpy()
    ref = np.tan(x.astype(np.longdouble))
    refd = ref.astype(np.float64)
    ulp = np.spacing(np.abs(refd))
    err = (np.abs(t.astype(np.longdouble) - ref) / ulp).astype(np.float64)
    assert np.all(np.isfinite(t)) and err.max() <= 2.0, err.max()
    assert np.mean(t == refd) >= 0.97, np.mean(t == refd)
    assert np.all(np.signbit(t) == np.signbit(x))
