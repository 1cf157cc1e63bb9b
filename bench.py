"""Benchmark: weighted events/s of the phase-space map on one GB300.

Workload: hadronic 2->4 at sqrt(S) = 13 TeV -- shat with 1/tau sampling, r_to_x1x2,
two Breit-Wigner W bosons (80.4, 2.1 GeV) decaying to massless pairs, the synthetic
parton density f(x) = x^-1.1 (1-x)^3, integrand f(x1) f(x2) x the two W propagators,
an 8-dimensional VEGAS grid with 64 bins per dimension adapted over 10 x 1e6 events
and then frozen, 1e7 events per step, FP64.

A step is one ps_generate call: in-kernel Philox4x32-10, VEGAS lookup, every map of the
channel, the Jacobian product, integrand, cut_unphysical, SoA stores of the event record
(6 momenta, x1, x2, w) and the per-channel reductions.  `value` is timed with CUDA
events on the launching stream with the outputs resident in HBM; `e2e` puts the whole event
record of every step into pinned host memory: the map kernel stores it there directly (the GPU
reaches the Grace memory over NVLink-C2C), timed on the host clock with the per-step read of the
channel sums; the copy-engine form (HBM, then a copy on a second stream) is reported beside it.

Every timed map runs the program compiled at creation (NVRTC, the slot file in registers;
programs of more than six channels compiled one unit per channel and linked); `--no-jit` runs
the interpreter kernel instead, and the main leg reports the interpreter's time beside it.
Compile times fall outside the timed regions.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--no-jit]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "weighted events/sec (1 GB300) and effective events/sec at fixed 0.5% integral error vs FP64 VEGAS"
UNIT = "events/s"
EVENTS = 10_000_000
SEED = 1002
VEGAS_ITERS, VEGAS_EVENTS = 10, 1_000_000
WORKLOAD = ("hadronic 2->4 W W at sqrt(S)=13 TeV: 1/tau shat map, r_to_x1x2, 2 Breit-Wigner W(80.4,2.1)->2 "
            "massless, f(x)=x^-1.1(1-x)^3, 8-dim VEGAS x 64 bins adapted 10x1e6 then frozen, 1e7 events/step, FP64")
# Algorithmic output bytes of one event: 6 momenta x 4 x 8 + x1 + x2 + w.
BYTES_PER_EVENT = 6 * 4 * 8 + 8 + 8 + 8
# FP64 floating-point operations executed per event by the map kernel (DFMA = 2, DADD/DMUL = 1):
# 2 x 438.2 + 140.6 + 233.7 from the ncu instruction counters of this kernel on this workload
# (profiles/ps_map_kernel_ww_2to4.md).
FP64_FLOP_PER_EVENT = 1250.7
# DRAM traffic per event from the same capture (read + write, 2e6-event launch), scaled to a launch.
DRAM_BYTES_PER_EVENT = 186.0
# FP64 peak of a GB300: 1.25 TFLOP/s nominal (152 SMs x 2 DFMA/clk x ~2.07 GHz) -- the ALU peak
# derived from the unit counts and clocks; no measured FP64 peak is provided.
FP64_PEAK_GFLOPS = 1250.0
# The binding resource is the FP64 pipe: 2 FP64 instructions per clock per SM, whether DFMA, DADD
# or DMUL, i.e. 152 x 2 x 2.07 GHz = 629.3 G instructions/s.  FP64 arithmetic instructions per
# event of the map kernel from the same ncu capture: DFMA + DADD + DMUL = 438.2 + 140.6 + 233.7.
FP64_INSTR_PER_EVENT = 812.5
FP64_PEAK_GINSTR = 152 * 2 * 2.07
# The same counters for the compiled program's kernel (ps_jit_map) on this workload, from its own
# ncu capture (profiles/ps_jit_map_ww_2to4.md): DFMA 405.6 + DADD 113.6 + DMUL 197.6 = 716.8 FP64
# arithmetic instructions (1122.4 flops) and 185.9 DRAM bytes per event; FP64 pipe 85.4 % active.
# Re-captured on the current build (the Kallen function of decays and 2->2 blocks taken from the
# masses, the per-tile statistics with six FP64 instructions per event, bins, maxima and sign
# tests on the integer ALU, one exponential for both parton densities, x2 = tau / x1, the decay
# daughters boosted with one dot product, the VEGAS bin widths staged with the grid, the
# collider's 1/S folded, the azimuths from a 256-point table and short Taylor series, the
# Breit-Wigner map's tangent from a double-double table and its regions without branches;
# profiles/fp64_pipe_probes.md): DFMA 331.9 + DADD 101.6 + DMUL 209.6 = 643.0 (974.9 flops),
# 676.7 FP64-pipe instructions in all (688.5 in warp-issue slots x 32: lanes 0.983 busy),
# 185.3 DRAM bytes per event, pipe active 0.845 of the elapsed cycles -- the FP64 issue probe's
# saturating loop reaches 0.84.
COMPILED_COUNTERS = {"instr": 643.0, "flops": 974.9, "dram": 185.3, "pipe": 0.845, "pipe_instr": 676.7}
INTERPRETER_COUNTERS = {"instr": FP64_INSTR_PER_EVENT, "flops": FP64_FLOP_PER_EVENT, "dram": DRAM_BYTES_PER_EVENT,
                        "pipe": 0.854}
# FP64 arithmetic instructions (DFMA + DADD + DMUL) per event of the 24-channel 2->8 workload, from
# the ncu captures of one 2^20-event launch: the compiled program on the current build
# (profiles/fp64_pipe_probes.md: 2451.3 + 1058.3 + 895.5); the interpreter's from an earlier build
# (profiles/ps_map_kernel_c5_2to8.md, before the mass-based Kallen function; an upper bound).
C5_FP64_INSTR_PER_EVENT = {"compiled": 4405.0, "interpreter": 6559.0}
# The same for the compiled six-channel 2->5 program, from one 2e6-event launch in the benchmark's
# channel proportions (profiles/fp64_pipe_probes.md): DFMA 998.1 + DADD 287.0 + DMUL 409.8.
C3_FP64_INSTR_PER_EVENT = 1694.9
# FP64-pipe instructions in all (arithmetic and conversions) per event of the compiled mixed-precision
# programs (profiles/fp64_pipe_probes.md): the FP64 pipe's share of the mixed form (with the
# conversions on the integer ALU, 0.55-0.75 of its cycles: no longer the only bound).
# Launch shapes (threads per CTA, CTAs per SM) the autotuner tries for compiled programs: the
# CTA count caps the registers (65536 / (threads x CTAs)); the large CTAs keep more warps on the
# same stretch of a long straight-line program, which the instruction cache rewards.
JIT_SHAPES = ((128, 2), (128, 3), (128, 4), (256, 1), (256, 2), (256, 3), (512, 1))
MIXED_FP64_PIPE_PER_EVENT = {"2to4": 61.0, "2to5": 312.6, "2to8": 434.6}
# FP64-pipe instructions per call of CUDA's double functions on the GB300, from the ncu counters of
# ps_fp64_probe's function loops less the empty loop (profiles/fp64_pipe_probes.md); an add or a
# multiply is one.  They convert the oracle's operation counts into the pipe's work.
FP64_PIPE_PER_CALL = {"add": 1.0, "mul": 1.0, "div": 5.0, "sqrt": 8.0, "exp": 15.0, "expm1": 19.0, "log": 28.0,
                      "log1p": 28.3, "pow": 83.0, "atan": 27.9, "atan2": 34.3, "tan": 28.8, "sin": 18.0,
                      "cos": 18.0}
# The measured FP64 issue rate of this run (fp64_peak), once taken; the derived figure otherwise.
_FP64_PEAK = {"value": None, "source": None}


def fp64_peak(ps, torch, local, reps=5):
    """The FP64 pipe's issue rate, measured: ps_fp64_probe's DFMA loop (eight independent chains
    per thread, 8 CTAs of 256 threads per SM, ~56 ms per launch) timed with CUDA events on the
    launching stream, median of `reps`; DADD and DMUL once each beside it."""
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    blocks, iters = sms * 8, 12000
    sink = torch.empty(blocks * 256, dtype=torch.float64, device=f"cuda:{local}")
    stream = torch.cuda.current_stream()
    n = 8.0 * iters * blocks * 256
    res = {"sm_count": sms, "blocks": blocks, "iters": iters}
    for kind, k in (("dfma", reps), ("dadd", 1), ("dmul", 1)):
        ps.fp64_probe(kind, blocks, iters, sink, stream)
        ts = []
        for _ in range(k):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ps.fp64_probe(kind, blocks, iters, sink, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        res[kind + "_ginstr_per_s"] = n / (statistics.median(ts) / 1e3) / 1e9
    _FP64_PEAK["value"] = res["dfma_ginstr_per_s"]
    _FP64_PEAK["source"] = (f"measured: DFMA issue loop (ps_fp64_probe), {sms} SMs x 8 CTAs x 256 threads, "
                            f"median of {reps} launches of {n:.3g} instructions")
    res["derived_ginstr_per_s"] = FP64_PEAK_GINSTR
    return res


def fp64_pipe_roofline(instr_per_event, events_per_s, flops_per_event=None):
    """The FP64-pipe roofline object of a kernel: its FP64 arithmetic instructions per event (from
    ncu) times its events per second (per GPU) against the FP64 issue peak measured in this run
    (fp64_peak; the derived 629.3 G/s if it was not taken); with flops per event also the flop form
    against 1.25 TFLOP/s.  Unknown counters give null fields."""
    achieved = None if instr_per_event is None else instr_per_event * events_per_s / 1e9
    peak = _FP64_PEAK["value"] or FP64_PEAK_GINSTR
    r = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "G FP64-pipe instructions/s",
         "frac": None if achieved is None else achieved / peak,
         "peak_source": _FP64_PEAK["source"] or "derived: 152 SMs x 2 FP64 instructions/clk x 2.07 GHz",
         "frac_of_derived_peak": None if achieved is None else achieved / FP64_PEAK_GINSTR}
    if flops_per_event is not None or instr_per_event is not None:
        gflops = None if flops_per_event is None else flops_per_event * events_per_s / 1e9
        r["flops"] = {"achieved": gflops, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
                      "frac": None if gflops is None else gflops / FP64_PEAK_GFLOPS,
                      "peak_source": "derived: 1.25 TFLOP/s FP64 (152 SMs x 2 DFMA/clk x 2.07 GHz)"}
    return r


def _r(x, nd=4):
    return None if x is None else float(f"{x:.{nd}g}")


def summary(line):
    """The headline figures of every leg in one short object, placed last in the JSON line so that
    a reader of the line's tail sees all of them."""
    g = lambda d, *ks: None if d is None else (g(d.get(ks[0]), *ks[1:]) if len(ks) > 1 else d.get(ks[0]))
    rf = line["roofline"]
    out = {"fp64_2to4": {"events_per_s": _r(line["value"]), "fp64_pipe_frac": _r(rf["frac"], 3),
                         "frac_of_derived_peak": _r(rf["frac_of_derived_peak"], 3), "e2e": _r(g(line, "e2e", "value")),
                         "interpreter": _r(g(line, "interpreter", "value"))},
           "fp64_peak_ginstr_per_s": _r(g(rf, "fp64_peak", "dfma_ginstr_per_s")),
           "sm_count": g(rf, "fp64_peak", "sm_count"),
           "method_pipe_equiv_per_event": _r(g(rf, "method", "fp64_pipe_equivalent_per_event")),
           "mixed_2to4": {"events_per_s": _r(g(line, "mixed_precision", "value")),
                          "speedup": _r(g(line, "mixed_precision", "speedup_vs_fp64"), 3),
                          "fp64_pipe_frac": _r(g(line, "mixed_precision", "fp64_pipe", "frac"), 3)},
           "multichannel_2to5": {"fp64": _r(g(line, "multichannel", "value")),
                                 "fp64_pipe_frac": _r(g(line, "multichannel", "roofline", "frac"), 3),
                                 "mixed": _r(g(line, "multichannel", "mixed_precision", "value"))},
           "streamed_2to8": {"fp64": _r(g(line, "streamed_2to8", "value")),
                             "fp64_pipe_frac": _r(g(line, "streamed_2to8", "roofline", "frac"), 3),
                             "e2e": _r(g(line, "streamed_2to8", "e2e", "value")),
                             "mixed": _r(g(line, "streamed_2to8", "mixed_precision", "value"))},
           "neff_per_s_over_fp64_vegas_2to8": {
               "mixed_vegas": _r(g(line, "importance_2to8", "mixed_n_eff_per_s_over_vegas_fp64"), 3),
               "flows_mixed_map": _r(g(line, "importance_2to8", "flow_mixed_map_n_eff_per_s_over_vegas_fp64"), 3),
               "flows_fp64_map": _r(g(line, "importance_2to8", "flow_n_eff_per_s_over_vegas_fp64"), 3)},
           "flow_2to4": {"ess_fraction": _r(g(line, "flow", "ess_fraction_flow"), 4),
                         "ess_fraction_vegas": _r(g(line, "flow", "ess_fraction_vegas"), 4),
                         "ess_per_s_over_vegas": None if g(line, "flow", "ess_per_s_flow") is None else
                         _r(line["flow"]["ess_per_s_flow"] / line["flow"]["ess_per_s_vegas"], 3),
                         "mixed_map_ess_per_s_over_vegas": _r(g(line, "flow", "mixed_map", "ess_per_s_over_fp64_vegas"), 3),
                         "sample_ms": _r(g(line, "flow", "sample_ms"), 3),
                         "train_ms_per_step": _r(g(line, "flow", "train_ms_per_step"), 3),
                         "train_steps": g(line, "flow", "train_steps")},
           "unweighting_events_per_s": _r(g(line, "unweighting", "events_per_s")),
           "global_multichannel_events_per_s": _r(g(line, "global_multichannel", "events_per_s")),
           "cpu_oracle_events_per_s": _r(g(line, "cpu_baseline", "value")),
           "cpu_cores": g(line, "cpu_baseline", "cores")}
    return out


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--events", type=int, default=EVENTS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-multichannel", action="store_true")
    ap.add_argument("--no-flow", action="store_true")
    ap.add_argument("--no-unweight", action="store_true")
    ap.add_argument("--no-global", action="store_true")
    ap.add_argument("--no-streamed", action="store_true")
    ap.add_argument("--no-c5-importance", action="store_true")
    ap.add_argument("--no-jit", action="store_true",
                    help="run every map on the interpreter instead of compiled programs")
    ap.add_argument("--stream-events", type=int, default=None, help="streamed leg: total events (default 1e8)")
    ap.add_argument("--stream-chunk", type=int, default=None, help="streamed leg: events per chunk (default 2^22)")
    ap.add_argument("--stream-config", default=None, help="streamed leg: 'threads,ctas_per_sm' instead of autotuning")
    ap.add_argument("--stream-precision", default="f64", choices=["f64", "mixed"])
    ap.add_argument("--flow-steps", type=int, default=20000,
                    help="flow training steps of 2^16 events (the learned-proposal workload trains 2e4)")
    ap.add_argument("--flow-infer-events", type=int, default=EVENTS)
    ap.add_argument("--leg", default="all", choices=["all", "flow", "unweight", "global", "streamed", "c5_importance"],
                    help="run one secondary leg alone (for profiling); prints its object only")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"ps_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if p[5 + k].lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(events, grid, seconds_target=12.0):
    """The FP64 oracle as it stands, on all host cores, on a bounded sample of the workload:
    consecutive 1e7-event steps (full event record kept) until about `seconds_target` of wall time."""
    import oracle as O
    from paper_2602_06895_gb300 import workloads as W

    ch = W.ww_hadronic()
    threads = O.max_threads()
    O.generate(ch, SEED, 0, 100_000, grid=grid, keep_momenta=True, threads=threads)  # warm-up
    t0 = time.perf_counter()
    O.generate(ch, SEED, 0, 1_000_000, grid=grid, keep_momenta=True, threads=threads)
    rate = 1_000_000 / max(time.perf_counter() - t0, 1e-6)
    steps = max(1, int(round(seconds_target * rate / events)))
    t0 = time.perf_counter()
    for k in range(steps):
        O.generate(ch, SEED, k * events, events, grid=grid, keep_momenta=True, threads=threads)
    dt = time.perf_counter() - t0
    n = steps * events
    t1 = time.perf_counter()
    O.generate(ch, SEED, 0, 200_000, grid=grid, keep_momenta=True, threads=1)
    single = 200_000 / (time.perf_counter() - t1)
    # the method's operations per event, counted by class in the oracle's own arithmetic (its
    # operation-counting build), on 2e4 events of the same stream; with the FP64-pipe cost of each
    # class on the GPU, the pipe work a literal evaluation of those operations would take
    ops, _ = O.op_counts(ch, O.random(SEED, 0, 0, 20_000, O.dims(ch)), grid=grid)
    pipe = sum(ops[k] * FP64_PIPE_PER_CALL[k] for k in FP64_PIPE_PER_CALL)
    return {"value": n / dt, "unit": UNIT, "cores": threads, "kind": "oracle", "single_core_value": single,
            "method_ops_per_event": {k: round(v, 2) for k, v in ops.items()},
            "method_fp64_pipe_equivalent_per_event": pipe,
            "sample": f"{steps} consecutive steps of {events} events (seed {SEED}, events 0..{n - 1}) of the "
                      f"workload, full event record kept, {dt:.2f} s wall ({dt * threads:.0f} core-s) on "
                      f"{threads} OpenMP threads"}


def adapted_grid(ps, W, torch):
    """VEGAS adaptation on the GPU (untimed): 10 iterations of 1e6 events, alpha = 1.5."""
    ch = W.ww_hadronic()
    prog = ps.program_for([ch])
    prog.vegas_training(True)
    out, ws = prog.alloc([VEGAS_EVENTS], 6)
    for it in range(VEGAS_ITERS):
        prog.generate([VEGAS_EVENTS], 7_000_000 + it, out, ws)
        prog.vegas_adapt(0, alpha=1.5)
    torch.cuda.synchronize()
    return prog.get_vegas(0, 8)


def timed(torch, fn, reps, stream):
    """Mean CUDA-event time (ms) of fn() over reps calls after one warm-up call."""
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def vegas_all_dims_leg(ps, W, torch, stream, local, jit, reps=3):
    """The 2->4 workload with VEGAS on all 10 random dimensions instead of 8: the two angles of the
    second W decay, on which the integrand does not depend, are mapped too.  Adapted like the
    8-dim grid (10 x 1e6 events, alpha 1.5), then 1e7 events per step; the ESS fraction shows what
    the two extra dimensions change."""
    ch = W.ww_hadronic(vegas_dims=10)
    prog = ps.program_for([ch], device=local)
    prog.vegas_training(True)
    out, ws = prog.alloc([VEGAS_EVENTS], 6, device=local)
    for it in range(VEGAS_ITERS):
        prog.generate([VEGAS_EVENTS], 7_000_000 + it, out, ws)
        prog.vegas_adapt(0, alpha=1.5)
    grid = prog.get_vegas(0, 10)
    del prog, out, ws
    tprog = ps.program_for([ch], device=local, jit=jit)
    tprog.set_vegas(0, grid)
    out, ws = tprog.alloc([EVENTS], 6, device=local)
    ms = timed(torch, lambda: tprog.generate([EVENTS], SEED, out, ws), reps, stream)
    st = tprog.stats()[0]
    ess = st["sum_w"] ** 2 / st["sum_w2"]
    return {"workload": "the main workload with VEGAS on all 10 dimensions (10 x 64 bins)", "events": EVENTS,
            "ms_per_step": ms, "events_per_s": EVENTS / (ms / 1e3), "ess_fraction": ess / EVENTS,
            "effective_events_per_s": ess / (ms / 1e3), "integral": st["sum_w"] / st["n"]}


def c1_leg(ps, W, torch, stream, local, events=100_000, reps=20):
    """2->2 at fixed sqrt(s) = 1000 GeV (two_body_decay of p0 = (1000, 0, 0, 0)): the phase-space
    volume (every weight is 1/(8 pi)) and the integral of 1 + cos^2(theta) (closed form 1/(6 pi)),
    1e5 events per launch (the size is launch-bound: the rate is that of a 1e5-event batch)."""
    res = {}
    for name, integrand, exact in (("volume", "none", 1.0 / (8.0 * math.pi)),
                                   ("one_plus_cos2", "one_plus_cos2", 1.0 / (6.0 * math.pi))):
        ch = W.two_body_fixed(integrand=integrand)
        prog = ps.program_for([ch], device=local)
        out, ws = prog.alloc([events], 4, x=False)
        ms = timed(torch, lambda: prog.generate([events], 1001, out, ws), reps, stream)
        st = prog.stats()[0]
        mean = st["sum_w"] / st["n"]
        sigma = math.sqrt(max(st["sum_w2"] / st["n"] - mean * mean, 0.0) / st["n"])
        res[name] = {"integral": mean, "sigma": sigma, "exact": exact, "rel_diff": mean / exact - 1.0,
                     "pulls": (mean - exact) / sigma if sigma > 1e-12 * mean else None,
                     "events_per_s": events / (ms / 1e3), "ms_per_launch": ms}
    res["workload"] = "2->2 massless at sqrt(s) = 1000 GeV, 1e5 events per launch (seed 1001)"
    return res


def streamed_leg(ps, W, torch, stream, rank, world, local, precision="f64", best=None, host_copy=False,
                 total=None, chunk=None, jit=False, zero_copy=False):
    """The 2->8 workload (six massless partons and two 173 GeV particles, 24 channels, SDE weights
    in-kernel) streamed: 1e8 events in chunks of 2^22, each chunk one persistent launch for all 24
    channels (CUDA graph, tiles and schedule from the autotuner) into one of two output buffers, its
    per-channel sums added on the device (streaming statistics, read once at the end).  With
    host_copy the record of each chunk also goes to pinned host memory on a second stream while
    the next chunk is generated; with zero_copy the map kernel writes the records straight into
    pinned host memory (the GPU reaches it over NVLink-C2C), with no copy.  With jit the program is
    compiled (one unit per channel, compiled in parallel and linked; the compile time is reported,
    outside the timed region)."""
    import numpy as np

    from paper_2602_06895_gb300 import distributed as D

    chans = W.channels_2to8()
    nc = len(chans)
    chunk = chunk or W.C5_CHUNK
    total = total or W.C5_EVENTS
    split = lambda n: [n // nc + (1 if c < n % nc else 0) for c in range(nc)]
    n_full, tail = divmod(total, chunk)
    table = None
    t_compile = time.perf_counter()
    if best is None:
        best, table = ps.autotune(chans, split(chunk // 4), precision=precision,
                                  blocks=(64, 128, 256), ctas=(1, 2, 3, 4), reps=2, device=local, jit=jit,
                                  pairs=JIT_SHAPES if jit else None)
    prog = ps.program_for(chans, device=local, precision=precision, jit=jit, **best)
    t_compile = time.perf_counter() - t_compile
    n_mom = chans[0]["n"] + 2
    bufs = [prog.alloc(split(chunk), n_mom, alpha=True, device=local) for _ in range(2)]
    if zero_copy:  # the output tensors in pinned host memory, the workspaces on the device
        bufs = [({k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for k, v in o.items()}, w)
                for o, w in bufs]
    execs = [prog.exec_create(split(chunk), o, w) for o, w in bufs]
    plan = [(execs[k % 2], k % 2, chunk) for k in range(n_full)]
    if tail:
        b = n_full % 2
        plan.append((prog.exec_create(split(tail), *bufs[b]), b, tail))
    seed = 1005
    # warm-up: one chunk per buffer
    for b in range(2):
        execs[b].launch(seed, D.step_offset(rank, world, chunk, len(plan) + b), stream)
    torch.cuda.synchronize()

    copy_stream = host = None
    if host_copy:
        copy_stream = torch.cuda.Stream(device=local)
        host = [{k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for k, v in o.items()} for o, _ in bufs]
    copied = [torch.cuda.Event() for _ in range(2)]
    d2h = 0
    prog.stats_accumulate(True, stream)  # per-channel sums of all chunks add up on the device
    l0 = ps.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e0.record(stream)
    for k, (ex, b, n) in enumerate(plan):
        if host_copy and k >= 2:
            stream.wait_event(copied[b])  # the copy of the chunk that last used this buffer is done
        ex.launch(seed, D.step_offset(rank, world, chunk, k), stream)
        if zero_copy:
            d2h += sum((v[:, :n] if v.dim() == 2 else v[:n]).numel() * v.element_size() for v in bufs[b][0].values())
        if host_copy:
            gen = torch.cuda.Event()
            gen.record(stream)
            copy_stream.wait_event(gen)
            with torch.cuda.stream(copy_stream):
                for key, v in bufs[b][0].items():
                    cols = v[:, :n] if v.dim() == 2 else v[:n]
                    dst = host[b][key][:, :n] if v.dim() == 2 else host[b][key][:n]
                    dst.copy_(cols, non_blocking=True)
                    d2h += cols.numel() * cols.element_size()
            copied[b].record(copy_stream)
    st = prog.stats(stream)  # the running per-channel sums of all chunks, read once
    e1.record(stream)
    if host_copy:
        copy_stream.synchronize()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    ms = e0.elapsed_time(e1)
    prog.stats_accumulate(False, stream)
    acc = np.array([(sc["n"], sc["n_nonzero"], sc["sum_w"], sc["sum_w2"]) for sc in st])
    max_w = max(sc["max_w"] for sc in st)
    launches = ps.launch_count() - l0
    if world > 1:
        t = torch.tensor([ms, wall], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms, wall = float(t[0]), float(t[1])
        a = torch.tensor(acc, device="cuda")
        torch.distributed.all_reduce(a)
        acc = a.cpu().numpy()
    n_ev = acc[:, 0].sum()
    # equal counts per channel: the integral is nc x the mean pooled weight, Kish ESS of the pool
    integral = nc * acc[:, 2].sum() / n_ev
    ess = acc[:, 2].sum() ** 2 / acc[:, 3].sum()
    var_mean = (acc[:, 3].sum() / n_ev - (acc[:, 2].sum() / n_ev) ** 2) / n_ev
    res = {"workload": "2->8 at sqrt(S)=13 TeV: 6 massless + 2 x 173 GeV, 24 channels (t-chains of 3-6 "
                       "clusters with W/Z/H/top resonances, s-channel trees), SDE multichannel weights "
                       "in-kernel, f(x)=x^-1.1(1-x)^3, uniform r (no VEGAS)",
           "events": int(n_ev), "chunk": chunk, "chunks": len(plan), "precision": precision,
           "value": world * total / (ms / 1e3), "unit": "streamed events/s", "ms_total": ms,
           "wall_s": wall, "map_launches_per_chunk": 1, "gpu_launches": int(launches), "cuda_graph": True,
           "autotuned": best, "integral": integral, "rel_err": math.sqrt(var_mean) * nc / integral,
           "ess": ess, "effective_events_per_s": ess / (ms / 1e3), "max_w": max_w,
           "nonzero_fraction": acc[:, 1].sum() / n_ev,
           "kernel": "compiled program (24 channel units, NVRTC in parallel, nvJitLink)" if jit else "interpreter",
           "setup_s": t_compile}
    if precision == "f64":  # the FP64 pipe's roofline, from this workload's ncu instruction counts
        instr = C5_FP64_INSTR_PER_EVENT["compiled" if jit else "interpreter"]
        res["roofline"] = fp64_pipe_roofline(instr, res["value"] / world)
        res["roofline"]["fp64_instr_per_event"] = instr
    elif jit:  # the mixed form: every FP64-pipe instruction (islands and conversions)
        res["roofline"] = fp64_pipe_roofline(MIXED_FP64_PIPE_PER_EVENT["2to8"], res["value"] / world)
        res["roofline"]["fp64_pipe_instr_per_event"] = MIXED_FP64_PIPE_PER_EVENT["2to8"]
    if table is not None:
        res["autotune_candidates"] = len(table)
    if host_copy or zero_copy:
        res["e2e"] = {"value": world * total / wall, "unit": "streamed events/s", "h2d_bytes_per_chunk": 16,
                      "d2h_bytes_per_chunk": int(d2h / len(plan)) + 40 * nc,
                      "note": ("the map kernel writes every chunk's event record straight into pinned host "
                               "memory (zero-copy over NVLink-C2C), two buffers; timed on the host clock"
                               if zero_copy else
                               "event records of every chunk copied to pinned host memory on a second stream, "
                               "double-buffered; timed on the host clock")}
    del execs, plan, bufs
    return res


def c5_importance_leg(ps, W, torch, stream, local, vegas_iters=10, vegas_events=1 << 21, flow_steps=150,
                      flow_batch=1 << 14, eval_events=1 << 22, jit=False):
    """Importance sampling on the 2->8 workload (24 channels, d = 22): uniform r, a VEGAS grid per
    channel (22 dims x 64 bins, adapted in one multichannel launch per iteration), the same grids
    in the mixed-precision program, and one RQ-spline flow per channel trained on top of its grid.

    Each sampler first draws eval_events events with equal counts per channel (pilot), then
    eval_events events with the variance-optimal counts n_c ~ sigma_c of its own pilot (the
    multichannel estimate I = sum_c mean_c has Var = sum_c sigma_c^2 / n_c).  Figure of merit:
    N_eff = I^2 / Var (unit-weight-equivalent events) per second of generation; the integrals
    must agree.  The median per-channel Kish ESS fraction shows the sampler quality alone.  With jit
    every timed program is a compiled one (the VEGAS adaptation and the flow training, untimed, run
    on the interpreter)."""
    import numpy as np

    chans = W.channels_2to8()
    nc, d = len(chans), W.n_random_dims(chans[0])
    n_mom = chans[0]["n"] + 2
    equal = [eval_events // nc + (1 if c < eval_events % nc else 0) for c in range(nc)]
    res = {"workload": "2->8, 24 channels (the streamed workload), " + str(eval_events) + " events per sampler"}

    def optimal(stats):
        sig = np.array([math.sqrt(max(s2 / n - (s1 / n) ** 2, 0.0)) if n else 0.0 for n, s1, s2 in stats])
        share = np.maximum(sig / max(sig.sum(), 1e-300), 0.002)  # every channel keeps a few events
        n = np.floor(share / share.sum() * eval_events).astype(np.int64)
        n[np.argmax(n)] += eval_events - int(n.sum())
        return [int(x) for x in n]

    def measure(name, run):
        """run(counts) -> per-channel (n, sum w, sum w^2) of the events it drew (after the timing)."""
        pilot = run(equal, timed_run=False)
        counts = optimal(pilot)
        run(counts, timed_run=False)  # warm-up at the final counts
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = run(counts, timed_run=True, events=(e0, e1))
        ms = e0.elapsed_time(e1)
        mean = [s1 / n for n, s1, _ in st]
        var = sum((s2 / n - (s1 / n) ** 2) / n for n, s1, s2 in st)
        I = sum(mean)
        neff = I * I / var
        kish = [s1 * s1 / s2 / n for n, s1, s2 in st if s2 > 0]
        res[name] = {"ms": ms, "events_per_s": eval_events / (ms / 1e3), "integral": I,
                     "rel_err": math.sqrt(var) / I, "n_eff": neff, "n_eff_fraction": neff / eval_events,
                     "n_eff_per_s": neff / (ms / 1e3), "events_for_0.5pct": var / (I * 0.005) ** 2 * eval_events,
                     "median_channel_kish_ess_fraction": float(np.median(kish)),
                     "pilot_kish_ess_fraction_equal_counts": sum(x[1] for x in pilot) ** 2 /
                     sum(x[2] for x in pilot) / eval_events}
        return res[name]

    def program_runner(prog, out_ws, seed):
        def run(counts, timed_run, events=None):
            # one generate call draws every channel's events into one record
            if "full" not in out_ws or out_ws["full"][0] != counts:
                out_ws["full"] = (counts, prog.alloc(counts, n_mom, alpha=True, device=local))
            out, ws = out_ws["full"][1]
            prog.generate(counts, seed, out, ws)
            if events is not None:
                events[1].record(stream)
            return [(sc["n"], sc["sum_w"], sc["sum_w2"]) for sc in prog.stats(stream)]
        return run

    # compiled programs: the shapes the streamed leg's autotuner picks on this workload (FP64: 2 CTAs
    # of 128 threads per SM at up to 255 registers; mixed: 4 CTAs, registers capped at 128)
    opts = {"block_threads": 128, "ctas_per_sm": 2, "jit": True} if jit else {"block_threads": 64, "ctas_per_sm": 3}
    opts_m = dict(opts, ctas_per_sm=4) if jit else opts
    res["kernel"] = "compiled programs" if jit else "interpreter"
    prog_u = ps.program_for(chans, device=local, **opts)
    measure("uniform_fp64", program_runner(prog_u, {}, 51))
    del prog_u

    # VEGAS per channel, adapted on the GPU (untimed)
    vchans = [dict(ch, vegas_dims=d) for ch in chans]
    prog_v = ps.program_for(vchans, device=local, block_threads=64, ctas_per_sm=3)
    vc = [vegas_events // nc] * nc
    out_v, ws_v = prog_v.alloc(vc, n_mom, alpha=True, device=local)
    prog_v.vegas_training(True)
    for it in range(vegas_iters):
        prog_v.generate(vc, 61 + it, out_v, ws_v)
        for c in range(nc):
            prog_v.vegas_adapt(c, alpha=1.5)
    prog_v.vegas_training(False)
    grids = [prog_v.get_vegas(c, d) for c in range(nc)]
    del out_v, ws_v
    prog_vt = prog_v
    if jit:
        prog_vt = ps.program_for(vchans, device=local, **opts)
        for c in range(nc):
            prog_vt.set_vegas(c, grids[c])
    vegas = measure("vegas_fp64", program_runner(prog_vt, {}, 52))
    res["vegas_fp64"]["adaptation"] = f"{vegas_iters} iterations x {vegas_events} events, alpha 1.5"

    prog_m = ps.program_for(vchans, device=local, precision="mixed", **opts_m)
    for c in range(nc):
        prog_m.set_vegas(c, grids[c])
    measure("vegas_mixed", program_runner(prog_m, {}, 52))

    # one flow per channel on top of its VEGAS grid, trained on the method's own weights
    flows = [ps.Flow(d, FLOW_LAYERS, FLOW_BINS, FLOW_HIDDEN, max_batch=flow_batch, init_seed=3000 + c)
             for c in range(nc)]
    r = torch.empty((d, flow_batch), dtype=torch.float64, device="cuda")
    ld = torch.empty(flow_batch, dtype=torch.float64, device="cuda")
    out_t, ws_t = prog_v.alloc([flow_batch] + [0] * (nc - 1), n_mom, alpha=True, device=local)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(flow_steps):
        for c in range(nc):
            flows[c].sample(flow_batch, 4000 + c, r, ld, event_offset=k * flow_batch)
            prog_v.map(c, r, out_t, ws_t)
            flows[c].train_step(out_t["weight"], 1e-3)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    del out_t, ws_t, r, ld

    def flow_runner(prog):
        buf = {}

        def run_f(counts, timed_run, events=None):
            nmax = max(counts)
            if buf.get("n") != nmax:
                buf.clear()
                buf["n"] = nmax
                buf["r"] = torch.empty((d, nmax), dtype=torch.float64, device="cuda")
                buf["ld"] = torch.empty(nmax, dtype=torch.float64, device="cuda")
                buf["o"] = prog.alloc([nmax] + [0] * (nc - 1), n_mom, alpha=True, device=local)
                buf["w"] = torch.empty(eval_events, dtype=torch.float64, device="cuda")
            ri, ldi, (oi, wsi), wf = buf["r"], buf["ld"], buf["o"], buf["w"]
            col = 0
            for c in range(nc):
                n = counts[c]
                flows[c].generate(n, 5000 + c, ri[:, :n], ldi[:n])
                prog.map(c, ri[:, :n], oi, wsi)
                flows[c].weights(oi["weight"][:n], ldi[:n], wf[col:col + n])
                col += n
            if events is not None:
                events[1].record(stream)
            out, col = [], 0
            for c in range(nc):
                w = wf[col:col + counts[c]]
                out.append((counts[c], float(w.sum()), float((w * w).sum())))
                col += counts[c]
            return out
        return run_f

    flow = measure("flow_on_vegas", flow_runner(prog_vt))
    res["flow_on_vegas"]["training"] = {"steps_per_channel": flow_steps, "batch": flow_batch, "seconds": train_s,
                                        "flows": nc, "layers": FLOW_LAYERS, "bins": FLOW_BINS,
                                        "hidden": FLOW_HIDDEN, "lr": 1e-3, "map": "fp64"}
    flow_m = measure("flow_on_vegas_mixed_map", flow_runner(prog_m))
    res["flow_on_vegas_mixed_map"]["note"] = "the same trained flows; events mapped by the mixed-precision program"
    res["flow_n_eff_per_s_over_vegas_fp64"] = flow["n_eff_per_s"] / vegas["n_eff_per_s"]
    res["flow_mixed_map_n_eff_per_s_over_vegas_fp64"] = flow_m["n_eff_per_s"] / vegas["n_eff_per_s"]
    res["mixed_n_eff_per_s_over_vegas_fp64"] = res["vegas_mixed"]["n_eff_per_s"] / vegas["n_eff_per_s"]
    del flows, prog_m, prog_vt
    return res

FLOW_LAYERS, FLOW_BINS, FLOW_HIDDEN, FLOW_BATCH = 6, 16, 128, 1 << 16


def flow_leg(args, ps, W, torch, grid, vegas_ess_per_event, vegas_ms_per_event, stream):
    """The learned proposal on C2's integrand: a 6-layer RQ-spline coupling flow (16 bins, MLP
    2 x 128, BF16 tensor-core GEMMs) trained on the method's own weights in batches of 2^16 on top
    of the adapted VEGAS grid, then 1e7 events drawn from it (sample -> explicit-input map -> flow
    weights), against VEGAS alone on the same integrand."""
    ch = W.ww_hadronic()
    d = W.n_random_dims(ch)
    prog = ps.program_for([ch], jit=True)  # the compiled FP64 map, as in the VEGAS main leg
    prog.set_vegas(0, grid)
    fl = ps.Flow(d, FLOW_LAYERS, FLOW_BINS, FLOW_HIDDEN, max_batch=FLOW_BATCH, init_seed=1004)
    B = FLOW_BATCH
    r = torch.empty((d, B), dtype=torch.float64, device="cuda")
    ld = torch.empty(B, dtype=torch.float64, device="cuda")
    out, ws = prog.alloc([B], 6)
    step = [0]

    def train_step():
        fl.sample(B, 1004, r, ld, event_offset=step[0] * B)
        prog.map(0, r, out, ws)
        fl.train_step(out["weight"], 1e-3)
        step[0] += 1

    for _ in range(max(args.flow_steps - 10, 0)):
        train_step()
    train_ms = timed(torch, train_step, min(9, max(args.flow_steps - 1, 1)), stream)
    loss, _ = fl.loss()
    N = args.flow_infer_events
    ri = torch.empty((d, N), dtype=torch.float64, device="cuda")
    ldi = torch.empty(N, dtype=torch.float64, device="cuda")
    oi, wsi = prog.alloc([N], 6)
    wi = torch.empty(N, dtype=torch.float64, device="cuda")

    def infer():
        fl.generate(N, 2004, ri, ldi)
        prog.map(0, ri, oi, wsi)
        fl.weights(oi["weight"], ldi, wi)

    sample_ms = timed(torch, lambda: fl.generate(N, 2004, ri, ldi), 2, stream)
    infer_ms = timed(torch, infer, 2, stream)
    w = wi
    s1, s2 = float(w.sum()), float((w * w).sum())
    ess = s1 * s1 / s2
    # the same flow with the mixed-precision compiled map (FP32 bulk, FP64 islands)
    mprog = ps.program_for([ch], jit=True, precision="mixed")
    mprog.set_vegas(0, grid)
    mo, mws = mprog.alloc([N], 6)
    wm = torch.empty(N, dtype=torch.float64, device="cuda")

    def infer_mixed():
        fl.generate(N, 2004, ri, ldi)
        mprog.map(0, ri, mo, mws)
        fl.weights(mo["weight"], ldi, wm)

    infer_mixed_ms = timed(torch, infer_mixed, 2, stream)
    m1, m2 = float(wm.sum()), float((wm * wm).sum())
    ess_m = m1 * m1 / m2
    del mo, mws, mprog
    # forward GEMM FLOPs per event: 2 (16 H + H^2 + H P_l) per layer, P_l = n_B (3K + 1) padded
    flops = 0.0
    for l in range(FLOW_LAYERS):
        nb = len(fl.mask(l))
        P = (nb * (3 * FLOW_BINS + 1) + 15) // 16 * 16
        flops += 2.0 * (16 * FLOW_HIDDEN + FLOW_HIDDEN * FLOW_HIDDEN + FLOW_HIDDEN * P)
    return {"workload": "C2 integrand, flow refining the adapted VEGAS grid: 6 coupling layers, 16 bins, "
                        f"MLP 2 x 128, BF16 operands / FP32 accumulation, batches of 2^16, {args.flow_steps} "
                        f"Adam steps (lr 1e-3), inference on {N} events",
            "train_ms_per_step": train_ms, "train_steps": args.flow_steps, "final_loss": loss,
            "inference_events": N, "sample_ms": sample_ms, "inference_ms": infer_ms,
            "ess_fraction_flow": ess / N, "ess_fraction_vegas": vegas_ess_per_event,
            "ess_per_s_flow": ess / (infer_ms / 1e3),
            "ess_per_s_vegas": vegas_ess_per_event / vegas_ms_per_event * 1e3,
            "integral_flow": s1 / N,
            "mixed_map": {"inference_ms": infer_mixed_ms, "ess_fraction": ess_m / N,
                          "ess_per_s": ess_m / (infer_mixed_ms / 1e3), "integral": m1 / N,
                          "ess_per_s_over_fp64_vegas": (ess_m / (infer_mixed_ms / 1e3)) /
                                                       (vegas_ess_per_event / vegas_ms_per_event * 1e3)},
            "tensor_gflop_per_event": flops / 1e9,
            "tensor_tflops_over_sample": flops * N / (sample_ms / 1e3) / 1e12,
            "sampling_path": "ps_flow_generate: one fused kernel per coupling layer",
            "note": "ESS = (sum w)^2 / sum w^2; ESS/s counts the whole generation time of each sampler "
                    "(no matrix element: the flow's gain per integrand call is ess_fraction_flow / "
                    "ess_fraction_vegas)"}


def unweight_leg(ps, torch, weights, stream):
    """Unweighting of one step's 1e7 C2 weights: maximum weight with 0.1% over-weight share of the
    cross section, then accept/reject and compaction."""
    N = weights.numel()
    uw = ps.Unweighter(N)
    idx = torch.empty(N, dtype=torch.int64, device="cuda")
    wo = torch.empty(N, dtype=torch.float64, device="cuda")
    mx_ms = timed(torch, lambda: uw.max_weight(weights, 1e-3), 5, stream)
    sel_ms = timed(torch, lambda: uw.select(weights, 1005, idx, wo), 5, stream)
    res = uw.result.cpu().tolist()
    na = int(uw.n_accepted.item())
    return {"events": N, "eps_overweight": 1e-3, "max_weight_ms": mx_ms, "select_ms": sel_ms,
            "events_per_s": N / ((mx_ms + sel_ms) / 1e3), "w_max": res[0], "n_over_w_max": int(res[3]),
            "unweighting_efficiency": na / N, "accepted": na}


def global_leg(ps, W, torch, stream):
    """Global (Kleiss-Pittau) multichannel weights for C3: events of one channel reweighted with
    the densities of all six channels (six GPU inverses, six density maps, one combination)."""
    import numpy as np

    chans = W.multichannel_2to5()
    dens = [dict(c, integrand="none") for c in chans]
    M = len(chans)
    N = 1_000_000
    prog = ps.program_for(chans)
    dprog = ps.program_for(dens)
    n_ev = [0, N, 0, 0, 0, 0]
    out, ws = prog.alloc(n_ev, 7, alpha=True)
    prog.generate(n_ev, 1006, out, ws)
    J = torch.empty((M, N), dtype=torch.float64, device="cuda")
    P = torch.empty((M, N), dtype=torch.float64, device="cuda")
    rs = [torch.empty((W.n_random_dims(c), N), dtype=torch.float64, device="cuda") for c in chans]
    outs = []
    for j in range(M):
        e = [0] * M
        e[j] = N
        outs.append(dprog.alloc(e, 7, x=True))
    w = torch.empty(N, dtype=torch.float64, device="cuda")
    alphas = np.full(M, 1.0 / M)

    def step():
        for j in range(M):
            ps.inverse_map(prog, j, chans[j], out["momenta"], out["x1"], out["x2"], rs[j], P[j])
            dprog.map(j, rs[j], outs[j][0], outs[j][1])
            J[j].copy_(outs[j][0]["weight"])
        ps.global_weights(J, alphas, w, P=P, x1=out["x1"], x2=out["x2"], pdf=chans[0]["pdf"])

    ms = timed(torch, step, 3, stream)
    inv_ms = timed(torch, lambda: ps.inverse_map(prog, 1, chans[1], out["momenta"], out["x1"], out["x2"], rs[1],
                                                 P[1]), 3, stream)
    return {"workload": "C3, 1e6 events of channel 1 reweighted with all six channel densities (alpha = 1/6)",
            "events_per_s": N / (ms / 1e3), "ms_per_1e6": ms, "inverse_ms_per_1e6_one_channel": inv_ms,
            "mean_w": float(w.mean())}


def run_reference(args, rank, world):
    """The reference arm: the oracle timed on the host cores (rank 0 only)."""
    if rank != 0:
        return
    import numpy as np

    import oracle as O
    from paper_2602_06895_gb300 import workloads as W

    ch = W.ww_hadronic()
    grid = W.vegas_grid_uniform(8, 64)
    threads = O.max_threads()
    sample = 2_000_000
    for _ in range(max(args.warmup, 0)):
        O.generate(ch, SEED, 0, sample // 10, grid=grid, threads=threads)
    t0 = time.perf_counter()
    for k in range(args.steps):
        O.generate(ch, SEED, k * sample, sample, grid=grid, threads=threads)
    dt = time.perf_counter() - t0
    value = args.steps * sample / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "events_per_step": sample,
                                            "note": "each step a bounded 2e6-event sample of the workload"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{args.steps} steps x {sample} events, uniform VEGAS grid"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import numpy as np
    import torch

    from paper_2602_06895_gb300 import build as B
    from paper_2602_06895_gb300 import distributed as D
    from paper_2602_06895_gb300 import ps
    from paper_2602_06895_gb300 import workloads as W

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    B.build()
    N = args.events

    grid = adapted_grid(ps, W, torch)
    if args.leg != "all":  # one secondary leg alone
        stream = torch.cuda.current_stream()
        ch = W.ww_hadronic()
        prog = ps.program_for([ch], device=local)
        prog.set_vegas(0, grid)
        out, ws = prog.alloc([N], 6, device=local)
        ms = timed(torch, lambda: prog.generate([N], SEED, out, ws), 1, stream)
        st = prog.stats()[0]
        ess = st["sum_w"] ** 2 / st["sum_w2"]
        if args.leg == "flow":
            res = flow_leg(args, ps, W, torch, grid, ess / N, ms / N, stream)
        elif args.leg == "streamed":
            cfg = None
            if args.stream_config:
                b, k = (int(x) for x in args.stream_config.split(","))
                cfg = {"block_threads": b, "ctas_per_sm": k}
            res = streamed_leg(ps, W, torch, stream, rank, world, local, precision=args.stream_precision, best=cfg,
                               jit=not args.no_jit,
                               total=args.stream_events, chunk=args.stream_chunk)
        elif args.leg == "c5_importance":
            res = c5_importance_leg(ps, W, torch, stream, local, jit=not args.no_jit)
        elif args.leg == "unweight":
            res = unweight_leg(ps, torch, out["weight"], stream)
        else:
            res = global_leg(ps, W, torch, stream)
        print(json.dumps({"leg": args.leg, args.leg: res}), flush=True)
        return
    ch = W.ww_hadronic()
    jit = not args.no_jit
    prog = ps.program_for([ch], device=local, jit=jit)  # compiled program (NVRTC) unless --no-jit
    prog.set_vegas(0, grid)
    out, ws = prog.alloc([N], 6, device=local)
    stream = torch.cuda.current_stream()
    off = lambda step: D.step_offset(rank, world, N, step)  # disjoint event ranges per rank and step

    # warm-up
    for k in range(args.warmup):
        prog.generate([N], SEED, out, ws, event_offset=off(k))
    torch.cuda.synchronize()

    # timed region: K steps, CUDA events on the launching stream, barrier + sync both sides
    sums = np.zeros(4)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    launches0 = ps.launch_count()
    ev[0].record(stream)
    for k in range(args.steps):
        prog.generate([N], SEED, out, ws, event_offset=off(args.warmup + k))
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    launches = ps.launch_count() - launches0
    clk = clocks.stop()
    step_ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    total_ms = ev[0].elapsed_time(ev[-1])
    st = prog.stats()[0]  # last step's statistics
    if world > 1:
        t = torch.tensor([total_ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
        st = D.combine_stats([st], device="cuda")[0]  # the one exchange: the global per-channel sums
    ms = total_ms / args.steps
    value = world * N * args.steps / (total_ms / 1e3)
    mean = st["sum_w"] / st["n"]
    var = st["sum_w2"] / st["n"] - mean * mean
    ess = st["sum_w"] ** 2 / st["sum_w2"]
    eff = ess / (ms / 1e3)  # effective (unit-weight-equivalent) events per second of the last step
    n_half_pct = var / (mean * mean * 0.005 ** 2)

    # the same steps on the interpreter kernel, for comparison (outside the timed region)
    interpreter = None
    if jit:
        iprog = ps.program_for([ch], device=local)
        iprog.set_vegas(0, grid)
        for k in range(args.warmup):
            iprog.generate([N], SEED, out, ws, event_offset=off(k))
        iev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        torch.cuda.synchronize()
        iev[0].record(stream)
        for k in range(args.steps):
            iprog.generate([N], SEED, out, ws, event_offset=off(args.warmup + k))
        iev[1].record(stream)
        torch.cuda.synchronize()
        ims = iev[0].elapsed_time(iev[1]) / args.steps
        interpreter = {"value": world * N / (ims / 1e3), "ms_per_step": ims, "kernel": "ps_map_kernel<0>"}
        del iprog

    # the FP64 pipe's measured issue rate: the denominator of every FP64 roofline below
    peak = fp64_peak(ps, torch, local)

    # end to end: same call with the event record in pinned host memory every step.  The headline
    # form writes it there from the map kernel (zero-copy: the GPU stores over NVLink-C2C into the
    # Grace memory); the copy-engine form (HBM, then cudaMemcpy on a second stream) is kept beside it.
    e2e = None
    if not args.no_e2e:
        zc = [{k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for k, v in out.items()} for _ in range(2)]
        zc_bytes = sum(v.numel() * v.element_size() for k, v in out.items() if k != "momenta") + \
            out["momenta"][:, :N].numel() * 8
        prog.generate([N], SEED, zc[0], ws, event_offset=off(0), stream=stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(args.steps):
            prog.generate([N], SEED, zc[k % 2], ws, event_offset=off(k), stream=stream)
            prog.stats(stream)  # per-channel sums to the host (synchronises the generation stream)
        torch.cuda.synchronize()
        dt_zc = time.perf_counter() - t0
        del zc
        # two output buffers: step k's record goes to pinned host memory on a second stream while
        # step k+1 is generated; every step also reads its per-channel sums back to the host
        outs = [out, prog.alloc([N], 6, device=local)[0]]
        host = [{k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for k, v in o.items()} for o in outs]
        d2h = sum(v.numel() * v.element_size() for k, v in out.items() if k != "momenta") + \
            out["momenta"][:, :N].numel() * 8
        copy_stream = torch.cuda.Stream(device=local)
        copied = [torch.cuda.Event(), torch.cuda.Event()]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(args.steps):
            b = k % 2
            if k >= 2:
                stream.wait_event(copied[b])  # the copy of step k-2 out of this buffer is done
            prog.generate([N], SEED, outs[b], ws, event_offset=off(k), stream=stream)
            gen = torch.cuda.Event()
            gen.record(stream)
            copy_stream.wait_event(gen)
            with torch.cuda.stream(copy_stream):
                for key, v in outs[b].items():
                    host[b][key].copy_(v, non_blocking=True)
            copied[b].record(copy_stream)
            prog.stats(stream)  # per-channel sums to the host (synchronises the generation stream)
        copy_stream.synchronize()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        e2e = {"value": world * N * args.steps / dt_zc, "unit": UNIT, "h2d_bytes_per_step": 16,
               "d2h_bytes_per_step": int(zc_bytes + 40),
               "copies": "the map kernel writes each step's record into pinned host memory (zero-copy over "
                         "NVLink-C2C, two buffers); the per-channel sums are read back every step",
               "copy_engine": {"value": world * N * args.steps / dt, "d2h_bytes_per_step": int(d2h + 40),
                               "copies": "each step's record from HBM to pinned host memory on a second "
                                         "stream (two buffers)"}}

    # mixed precision (FP32 bulk, FP64 islands) on the same events: same step, same grid
    mixed = None
    if not args.no_mixed:
        mprog = ps.program_for([ch], device=local, precision="mixed", jit=jit)
        mprog.set_vegas(0, grid)
        mout, mws = mprog.alloc([N], 6, device=local)
        for k in range(args.warmup):
            mprog.generate([N], SEED, mout, mws, event_offset=off(k))
        torch.cuda.synchronize()
        mev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        mev[0].record(stream)
        for k in range(args.steps):
            mprog.generate([N], SEED, mout, mws, event_offset=off(args.warmup + k))
            mev[k + 1].record(stream)
        torch.cuda.synchronize()
        mms = mev[0].elapsed_time(mev[-1]) / args.steps
        mst = mprog.stats()[0]
        # the last FP64 step and the last mixed step drew the same events
        mess = mst["sum_w"] ** 2 / mst["sum_w2"]
        mixed = {"value": world * N / (mms / 1e3), "ms_per_step": mms, "dtype": "f32 bulk + f64 islands",
                 "effective_events_per_s": mess / (mms / 1e3),
                 "integral_rel_diff_vs_fp64_same_events": mst["sum_w"] / st["sum_w"] - 1.0 if world == 1 else None,
                 "speedup_vs_fp64": ms / mms,
                 "bytes_per_event": 6 * 4 * 4 + 4 + 4 + 8,
                 "hbm_gbs": (6 * 4 * 4 + 4 + 4 + 8) * N / (mms / 1e3) / 1e9}
        if jit:  # the mixed form is bound by the FP64 pipe too (islands and conversions)
            mixed["fp64_pipe"] = fp64_pipe_roofline(MIXED_FP64_PIPE_PER_EVENT["2to4"], N / (mms / 1e3))
            mixed["fp64_pipe"]["counts"] = "every FP64-pipe instruction per event (arithmetic and conversions)"

    # multichannel 2->5: six channels of mixed topology, uneven counts (1e5 .. 4e6, 2e7 in all), one
    # persistent launch per step, tiles and schedule from the autotuner, replayed as a CUDA graph
    multi = None
    if not args.no_multichannel:
        chans = W.multichannel_2to5()
        counts = list(W.MULTICHANNEL_EVENTS)
        best, table = ps.autotune(chans, [c // 8 for c in counts], blocks=(64, 128, 256), ctas=(1, 2, 3, 4),
                                  reps=2, device=local, jit=jit, pairs=JIT_SHAPES + ((128, 5), (128, 6)) if jit else None)
        mprog = ps.program_for(chans, device=local, jit=jit, **best)
        mout, mws = mprog.alloc(counts, 7, alpha=True, device=local)
        ex = mprog.exec_create(counts, mout, mws)
        for k in range(args.warmup):
            ex.launch(1003, D.step_offset(rank, world, sum(counts), k))
        torch.cuda.synchronize()
        l0 = ps.launch_count()
        cev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        cev[0].record(stream)
        for k in range(args.steps):
            ex.launch(1003, D.step_offset(rank, world, sum(counts), args.warmup + k), stream)
            cev[k + 1].record(stream)
        torch.cuda.synchronize()
        cms = cev[0].elapsed_time(cev[-1]) / args.steps
        cst = mprog.stats()
        multi = {"workload": "2->5 massless at sqrt(S)=13 TeV, 6 channels (t-chains with Z/H/T resonances, "
                             "pure s), SDE multichannel weights in-kernel, events " + str(counts),
                 "value": world * sum(counts) / (cms / 1e3), "unit": UNIT, "ms_per_step": cms,
                 "precision": "fp64", "map_launches_per_step": 1, "compiled": jit,
                 "gpu_launches": int(ps.launch_count() - l0), "cuda_graph": True,
                 "autotuned": best,
                 "integral": sum(c["sum_w"] for c in cst) / 1.0,
                 "integral_mean": sum(c["sum_w"] / c["n"] for c in cst if c["n"]),
                 "integral_sigma": math.sqrt(sum((c["sum_w2"] / c["n"] - (c["sum_w"] / c["n"]) ** 2) / c["n"]
                                                 for c in cst if c["n"]))}
        # the FP64 pipe's roofline of the compiled program (instructions per event from its ncu capture)
        multi["roofline"] = fp64_pipe_roofline(C3_FP64_INSTR_PER_EVENT if jit else None, multi["value"] / world)
        multi["roofline"]["fp64_instr_per_event"] = C3_FP64_INSTR_PER_EVENT if jit else None
        # the mixed-precision form of the same step on the same events
        mbest, _ = ps.autotune(chans, [c // 8 for c in counts], precision="mixed", blocks=(64, 128, 256),
                               ctas=(1, 2, 3, 4), reps=2, device=local, jit=jit,
                               pairs=JIT_SHAPES + ((128, 5), (128, 6)) if jit else None)
        xprog = ps.program_for(chans, device=local, precision="mixed", jit=jit, **mbest)
        xout, xws = xprog.alloc(counts, 7, alpha=True, device=local)
        xex = xprog.exec_create(counts, xout, xws)
        for k in range(args.warmup):
            xex.launch(1003, D.step_offset(rank, world, sum(counts), k))
        torch.cuda.synchronize()
        xev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        xev[0].record(stream)
        for k in range(args.steps):
            xex.launch(1003, D.step_offset(rank, world, sum(counts), args.warmup + k), stream)
        xev[1].record(stream)
        torch.cuda.synchronize()
        xms = xev[0].elapsed_time(xev[1]) / args.steps
        xst = xprog.stats()  # the last step drew the same events as the last FP64 step
        multi["mixed_precision"] = {"value": world * sum(counts) / (xms / 1e3), "ms_per_step": xms,
                                    "fp64_pipe_frac": (MIXED_FP64_PIPE_PER_EVENT["2to5"] * sum(counts) / (xms / 1e3)
                                                       / 1e9 / (_FP64_PEAK["value"] or FP64_PEAK_GINSTR)) if jit else None,
                                    "speedup_vs_fp64": cms / xms, "autotuned": mbest,
                                    "integral_rel_diff_vs_fp64_same_events":
                                        sum(c["sum_w"] for c in xst) / multi["integral"] - 1.0}
        del xex, xprog, xout, xws

    # 2->8, 24 channels, 1e8 events streamed in 2^22-event chunks: FP64 (device-resident and with the
    # records copied to the host) and the mixed-precision form on the same events
    streamed = None
    if not args.no_streamed:
        streamed = streamed_leg(ps, W, torch, stream, rank, world, local, jit=jit)
        if not args.no_e2e:
            streamed["e2e"] = streamed_leg(ps, W, torch, stream, rank, world, local, best=streamed["autotuned"],
                                           zero_copy=True, jit=jit)["e2e"]
            streamed["e2e"]["copy_engine"] = streamed_leg(ps, W, torch, stream, rank, world, local,
                                                          best=streamed["autotuned"], host_copy=True,
                                                          jit=jit)["e2e"]["value"]
        sm = streamed_leg(ps, W, torch, stream, rank, world, local, precision="mixed", jit=jit)
        streamed["mixed_precision"] = {k: sm.get(k) for k in ("value", "ms_total", "integral", "rel_err", "ess",
                                                              "effective_events_per_s", "autotuned", "roofline")}
        streamed["mixed_precision"]["integral_rel_diff_vs_fp64_same_events"] = sm["integral"] / streamed["integral"] - 1
        streamed["mixed_precision"]["speedup_vs_fp64"] = streamed["ms_total"] / sm["ms_total"]

    c1 = c1_leg(ps, W, torch, stream, local) if rank == 0 else None
    dv10 = vegas_all_dims_leg(ps, W, torch, stream, local, jit) if rank == 0 else None

    c5imp = None
    if not args.no_c5_importance and rank == 0:
        c5imp = c5_importance_leg(ps, W, torch, stream, local, jit=jit)

    flow = None
    if not args.no_flow and rank == 0:
        flow = flow_leg(args, ps, W, torch, grid, ess / N, ms / N, stream)
    unweight = None
    if not args.no_unweight and rank == 0:
        prog.generate([N], SEED, out, ws)
        unweight = unweight_leg(ps, torch, out["weight"], stream)
    glob = None
    if not args.no_global and rank == 0:
        glob = global_leg(ps, W, torch, stream)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(N, grid)

    # the FP64-pipe roofline: FP64 arithmetic instructions issued per second against the pipe's
    # measured issue rate (a DADD or DMUL takes a slot exactly like a DFMA); the flop form beside it
    kc = COMPILED_COUNTERS if jit else INTERPRETER_COUNTERS
    roofline = fp64_pipe_roofline(kc["instr"], N / (ms / 1e3), flops_per_event=kc["flops"])
    roofline.update({"traffic": None if kc["dram"] is None else kc["dram"] * N,
                     "kernel": "ps_jit_map (compiled program)" if jit else "ps_map_kernel<0> (interpreter)",
                     "fp64_pipe_active_ncu": kc["pipe"], "hbm_gbs": BYTES_PER_EVENT * N / (ms / 1e3) / 1e9,
                     "fp64_peak": peak})
    if kc.get("pipe_instr"):  # every FP64-pipe instruction (conversions included) against the same peak
        roofline["pipe_instr_frac"] = kc["pipe_instr"] * N / (ms / 1e3) / 1e9 / roofline["peak"]
    if cpu is not None:  # the method's work beside the executed instructions
        meq = cpu["method_fp64_pipe_equivalent_per_event"]
        roofline["method"] = {"fp64_pipe_equivalent_per_event": meq, "executed_per_event": kc["instr"],
                              "executed_over_method": kc["instr"] / meq,
                              "note": "the oracle's operations per event (cpu_baseline.method_ops_per_event) at "
                                      "the GPU's FP64-pipe cost per operation class; the kernel issues fewer "
                                      "(contracted multiply-adds, shared reciprocals, log x handed to the "
                                      "densities, integer-ALU decisions)"}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "events_per_step": N, "global_events_per_step": world * N,
                       "parallelism": f"replicas x{world} (independent event ranges)",
                       "l2": "no flush: every step writes a 2.16 GB event record (> 129 MB L2)",
                       "precision": "fp64", "block_threads": 128,
                       "kernel": "compiled program (NVRTC, slots in registers)" if jit else "interpreter"},
            "interpreter": interpreter,
            "effective_events_per_s": eff, "integral": {"mean_w": mean, "rel_err_per_step": math.sqrt(var / st["n"]) / mean,
                                                        "ess_per_step": ess, "events_for_0.5pct": n_half_pct},
            "step_ms_min": min(step_ms), "step_ms_median": statistics.median(step_ms),
            "clocks": clk, "gpu_launches": int(launches), "e2e": e2e, "roofline": roofline,
            "cpu_baseline": cpu, "mixed_precision": mixed, "multichannel": multi, "streamed_2to8": streamed,
            "importance_2to8": c5imp, "fixed_2to2": c1, "vegas_all_10_dims": dv10, "flow": flow, "unweighting": unweight, "global_multichannel": glob}
    line["summary"] = summary(line)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
