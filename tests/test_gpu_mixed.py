"""Mixed precision (FP32 bulk, FP64 islands) against the FP64 oracle, per output.

The stated error of each output on the 2->4 W W workload (measured on 4999 interior points:
medians 3e-7 momenta, 7e-7 x, 5e-6 weight; asserted with margin):
  momenta  |p_mixed - p_orc| / (largest energy of the event):  99.9% < 5e-6, all < 1e-4
  x1, x2   relative:                                          99.9% < 5e-6, all < 1e-5
  weight   relative:                                          99% < 5e-4, 99.9% < 5e-3, all < 5e-2
(the weight tail is the (1-x)^3 factor of the parton density amplifying x's FP32 rounding as
x -> 1).  t-chains lose more: a boost into the rest frame of a light cluster amplifies FP32
rounding by gamma^2, so the 2->5 channels are held to median 1e-6 / 99% 3e-3 on momenta --
FP64 is the path for them.  The integral of 1e7 Philox events agrees with the FP64 path on the
same events to 1e-5 relative, far inside the 0.5% Monte Carlo error target.
2->8 channels (SDE weights of all 24 channels in FP32): momenta median 1.3-2.1e-7, 99% < 3.3e-6;
weights median 2.5e-6 to 5e-5, 99% < 1.7e-2 (the worst-conditioned channel has a far tail);
alpha within 1e-6 absolute at the median; integrals of 2^20 events within 1.5e-6 of FP64.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2602_06895_gb300 import ps
from paper_2602_06895_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2602_06895_gb300 import build

    build.build()
    return torch


def per_output_errors(torch, chans, which, r, grid=None):
    ch = chans[which]
    prog = ps.program_for(chans, precision="mixed")
    if grid is not None:
        prog.set_vegas(which, grid)
    B, n = r.shape[0], ch["n"] + 2
    out, ws = prog.alloc([B if c == which else 0 for c in range(len(chans))], n, x=ch["hadronic"],
                         alpha=ch["integrand"] == "pdf_sde")
    prog.map(which, torch.from_numpy(np.ascontiguousarray(r.T)).cuda(), out, ws)
    torch.cuda.synchronize()
    orc = O.forward(ch, r, grid=grid, channels=chans, chan=which)
    ok = (orc["w"] != 0) & (out["weight"][:B].cpu().numpy() != 0)
    mom = out["momenta"][:, :B].double().cpu().numpy().reshape(n, 4, B).transpose(2, 0, 1)
    scale = np.max(np.abs(orc["mom"][:, :, 0]), axis=1)
    em = np.max(np.abs(mom - orc["mom"]), axis=(1, 2))[ok] / scale[ok]
    ew = np.abs(out["weight"][:B].cpu().numpy()[ok] / orc["w"][ok] - 1.0)
    res = {"momenta": em, "weight": ew}
    if ch["hadronic"]:
        x = np.stack([out["x1"][:B].double().cpu().numpy(), out["x2"][:B].double().cpu().numpy()], axis=1)
        res["x"] = np.max(np.abs(x / orc["x"] - 1.0), axis=1)[ok]
    return res


def describe(e):
    return {k: (float(np.median(v)), float(np.percentile(v, 99)), float(np.percentile(v, 99.9)), float(v.max()))
            for k, v in e.items()}


def test_mixed_per_output_error_ww(torch_cuda):
    grid = W.vegas_grid_random(11, 8, 64)
    r = W.uniform_r(515, 4999, 10)
    e = per_output_errors(torch_cuda, [W.ww_hadronic()], 0, r, grid)
    d = describe(e)
    print("mixed 2->4 W W per-output error (median, p99, p99.9, max):", d)
    assert np.percentile(e["momenta"], 99.9) < 5e-6 and e["momenta"].max() < 1e-4, d
    assert np.percentile(e["x"], 99.9) < 5e-6 and e["x"].max() < 1e-5, d
    assert np.percentile(e["weight"], 99) < 5e-4 and np.percentile(e["weight"], 99.9) < 5e-3, d
    assert e["weight"].max() < 5e-2, d


@pytest.mark.parametrize("which", range(6))
def test_mixed_per_output_error_multichannel(torch_cuda, which):
    chans = W.multichannel_2to5()
    r = W.uniform_r(600 + which, 2000, 13)
    e = per_output_errors(torch_cuda, chans, which, r)
    d = describe(e)
    print(chans[which]["name"], "mixed per-output error:", d)
    assert np.median(e["momenta"]) < 1e-6 and np.percentile(e["momenta"], 99) < 3e-3, d
    assert np.median(e["weight"]) < 1e-5 and np.percentile(e["weight"], 99) < 5e-3, d


def test_mixed_integral_matches_fp64(torch_cuda):
    ch = W.ww_hadronic()
    grid = W.vegas_grid_random(41, 8, 64)
    N = 10_000_000
    sums = {}
    for prec in ("f64", "mixed"):
        prog = ps.program_for([ch], precision=prec)
        prog.set_vegas(0, grid)
        out, ws = prog.alloc([N], 6)
        prog.generate([N], 1002, out, ws)
        sums[prec] = prog.stats()[0]
    a, b = sums["mixed"], sums["f64"]
    rel = abs(a["sum_w"] / b["sum_w"] - 1.0)
    mc = math.sqrt(b["sum_w2"] / b["n"] - (b["sum_w"] / b["n"]) ** 2) / math.sqrt(b["n"]) / (b["sum_w"] / b["n"])
    print("integral: mixed/f64 - 1 =", rel, " MC relative error of one step =", mc)
    assert rel < 1e-5 and rel < 0.01 * mc
    assert abs(a["n_nonzero"] - b["n_nonzero"]) <= 1e-6 * N


def _alpha_errors(torch, chans, which, r):
    ch = chans[which]
    prog = ps.program_for(chans, precision="mixed")
    B, n = r.shape[0], ch["n"] + 2
    out, ws = prog.alloc([B if c == which else 0 for c in range(len(chans))], n, alpha=True)
    prog.map(which, torch.from_numpy(np.ascontiguousarray(r.T)).cuda(), out, ws)
    torch.cuda.synchronize()
    orc = O.forward(ch, r, channels=chans, chan=which)
    ok = (orc["w"] != 0) & (out["weight"][:B].cpu().numpy() != 0)
    return np.abs(out["alpha"][:B].double().cpu().numpy()[ok] - orc["alpha"][ok])


@pytest.mark.parametrize("which", [0, 1, 2, 9, 17])
def test_mixed_per_output_error_2to8(torch_cuda, which):
    """2->8 channels (t-chains and s-channel trees, two top-mass particles, SDE weights of all 24
    channels evaluated in FP32): per-output errors of the mixed form against the FP64 oracle."""
    chans = W.channels_2to8()
    r = W.uniform_r(700 + which, 3000, W.n_random_dims(chans[which]))
    e = per_output_errors(torch_cuda, chans, which, r)
    e["alpha_abs"] = _alpha_errors(torch_cuda, chans, which, r)
    d = describe(e)
    print(chans[which]["name"], "mixed per-output error:", d)
    assert np.median(e["momenta"]) < 1e-5 and np.percentile(e["momenta"], 99) < 1e-2, d
    assert np.median(e["weight"]) < 1e-4 and np.percentile(e["weight"], 99) < 5e-2, d
    assert np.median(e["alpha_abs"]) < 1e-4, d


def test_mixed_integral_matches_fp64_2to8(torch_cuda):
    """The 24-channel 2->8 program, mixed against FP64 on the same 2^20 Philox events: the summed
    channel integrals agree far inside the Monte Carlo error.  The mixed form zeroes a few more
    events than FP64 (measured: at most 5 of 43690 in a channel, 1.1e-4): FP32 rounding at a
    threshold empties a sampled range, or makes a value non-finite so that cut_unphysical drops
    the event."""
    chans = W.channels_2to8()
    counts = [(1 << 20) // 24] * 24
    sums = {}
    for prec in ("f64", "mixed"):
        prog = ps.program_for(chans, precision=prec, block_threads=64)
        out, ws = prog.alloc(counts, 10, alpha=True)
        prog.generate(counts, 1005, out, ws)
        sums[prec] = prog.stats()
    I = {p: sum(s["sum_w"] / s["n"] for s in st) for p, st in sums.items()}
    var = sum((s["sum_w2"] / s["n"] - (s["sum_w"] / s["n"]) ** 2) / s["n"] for s in sums["f64"])
    rel = abs(I["mixed"] / I["f64"] - 1.0)
    mc = math.sqrt(var) / I["f64"]
    print("2->8 integral: mixed/f64 - 1 =", rel, " MC relative error =", mc)
    assert rel < 1e-4 and rel < 0.01 * mc
    for a, b in zip(sums["mixed"], sums["f64"]):
        assert abs(a["n_nonzero"] - b["n_nonzero"]) <= 5e-4 * b["n"]


# ---------------------------------------------------------------- the helpers at the islands' edges
# The mixed kernels convert between FP32 and FP64 on the integer ALU and seed their FP64
# reciprocal and square root from float approximations.  The conversions must equal the
# hardware's IEEE 754 conversions bit for bit: float -> double over every one of the 2^32 float
# bit patterns, double -> float over random patterns of every exponent and, for each float
# cell, the two neighbours of its rounding boundary and the exact ties (normal and subnormal).
def _same_or_both_nan(torch, a, b):
    nan = torch.isnan(a)
    assert torch.equal(nan, torch.isnan(b))
    return torch.equal(a[~nan].view(torch.int64 if a.dtype == torch.float64 else torch.int32),
                       b[~nan].view(torch.int64 if b.dtype == torch.float64 else torch.int32))


def test_f2d_matches_hardware_on_every_float(torch_cuda):
    torch = torch_cuda
    chunk = 1 << 28
    out = torch.empty(chunk, dtype=torch.float64, device="cuda")
    for c in range(1 << 32 >> 28):
        bits = torch.arange(c * chunk, (c + 1) * chunk, dtype=torch.int64, device="cuda").to(torch.int32)
        x = bits.view(torch.float32)
        ps.mixed_helper("f2d", x, out)
        assert _same_or_both_nan(torch, out, x.double()), c
        del bits, x


def test_d2f_matches_hardware(torch_cuda):
    torch = torch_cuda
    g = torch.Generator(device="cuda").manual_seed(20260412)
    n = 1 << 26
    # random bit patterns (every exponent, both signs)
    hi = torch.randint(-(1 << 31), 1 << 31, (n,), generator=g, device="cuda", dtype=torch.int64)
    lo = torch.randint(0, 1 << 32, (n,), generator=g, device="cuda", dtype=torch.int64)
    x_rand = ((hi << 32) | lo).view(torch.float64)
    # exponents around the float range's ends (double exponents 860..910 and 1140..1160)
    e = torch.cat([torch.randint(860, 911, (n // 2,), generator=g, device="cuda"),
                   torch.randint(1140, 1161, (n // 2,), generator=g, device="cuda")])
    x_edge = ((e << 52) | (lo & ((1 << 52) - 1)) | ((hi & 1) << 63)).view(torch.float64)
    # every float cell's rounding boundary: the double of a float plus k double ulps around
    # half a float ulp (normal floats: 2^28 double ulps), and the exact subnormal ties
    f = torch.randint(0, 1 << 31, (n // 8,), generator=g, device="cuda", dtype=torch.int64).to(torch.int32)
    fb = f.view(torch.float32).double().view(torch.int64)
    ks = torch.tensor([0, 1, -1, (1 << 28) - 1, 1 << 28, (1 << 28) + 1, (1 << 29) - 1], device="cuda")
    x_cells = (fb[:, None] + ks[None, :]).reshape(-1).view(torch.float64)
    q = torch.randint(0, 1 << 23, (n // 8,), generator=g, device="cuda", dtype=torch.int64).double()
    x_ties = torch.cat([torch.ldexp(q + 0.5, torch.tensor(-149.0, device="cuda")),
                        torch.ldexp(q + 0.25, torch.tensor(-149.0, device="cuda")),
                        torch.ldexp(q + 0.75, torch.tensor(-149.0, device="cuda"))])
    special = torch.tensor([0.0, -0.0, float("inf"), -float("inf"), float("nan"), 3.4028234663852886e38,
                            3.4028235677973366e38, 3.4028235677973362e38, 1.1754943508222875e-38,
                            1.401298464324817e-45, 7.006492321624085e-46, 7.006492321624087e-46,
                            5e-324, -5e-324, 1e300, -1e-300], dtype=torch.float64, device="cuda")
    for x in (x_rand, x_edge, x_cells, x_ties, special):
        out = torch.empty(x.numel(), dtype=torch.float32, device="cuda")
        ps.mixed_helper("d2f", x, out)
        assert _same_or_both_nan(torch, out, x.float())


def test_sqrt64_rcp64_accuracy(torch_cuda):
    """One Newton step from a seed whose exponent is set on the integer ALU and whose fraction
    comes from a float instruction (error delta <= ~2.2e-7 from the truncation to 23 bits and
    the approximate instruction) leaves a relative error of 1.5 delta^2 for the square root and
    delta^2 for the reciprocal: below 1e-13 over the normal doubles (|ln x| < 700, far outside
    the float range on both sides)."""
    torch = torch_cuda
    g = torch.Generator(device="cuda").manual_seed(7)
    n = 1 << 24
    x = torch.exp(torch.empty(n, dtype=torch.float64, device="cuda").uniform_(-700.0, 700.0, generator=g))
    out = torch.empty_like(x)
    ps.mixed_helper("sqrt64", x, out)
    assert torch.max(torch.abs(out / torch.sqrt(x) - 1.0)).item() < 1e-13
    xs = torch.where(torch.rand(n, generator=g, device="cuda") < 0.5, x, -x)
    ps.mixed_helper("rcp64", xs, out)
    assert torch.max(torch.abs(out * xs - 1.0)).item() < 1e-13
    edge = torch.tensor([0.0, -0.0, -1.0, float("nan"), -float("inf")], dtype=torch.float64, device="cuda")
    o = torch.empty_like(edge)
    ps.mixed_helper("sqrt64", edge, o)
    assert torch.equal(o, torch.zeros_like(o))  # x <= 0 and NaN give 0


def test_mixed_keeps_every_fp64_event_multichannel(torch_cuda):
    """On 2e6 events of the six 2->5 channels the mixed and FP64 programs make the same cut
    decisions: no event is zeroed in one precision only.  This holds down to the near-threshold
    events (weights to 1e-70), whose FP64 islands take square roots and reciprocals of numbers
    outside the float range."""
    torch = torch_cuda
    chans = W.multichannel_2to5()
    counts = [c // 10 for c in W.MULTICHANNEL_EVENTS]
    w = {}
    for prec in ("f64", "mixed"):
        prog = ps.program_for(chans, block_threads=128, ctas_per_sm=3, precision=prec, jit=True)
        out, ws = prog.alloc(counts, 7, alpha=True)
        prog.generate(counts, 1003, out, ws)
        torch.cuda.synchronize()
        w[prec] = out["weight"].cpu().numpy()
    assert np.array_equal(w["f64"] == 0, w["mixed"] == 0)
    assert np.min(w["f64"][w["f64"] > 0]) < 1e-60  # the near-threshold events are in the sample
