"""The benchmark's reference arm (the oracle timed on the host cores) keeps the one-line JSON
contract without a GPU: the metric, unit and direction of the main arm, `impl`, a
`cpu_baseline` of kind "oracle" describing the run, and an `e2e` object with no host-device
bytes. Under several ranks only rank 0 runs and prints; the others exit without work. The FP64
roofline arithmetic of the main arm is checked on its measured counters."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None):
    env = dict(os.environ)
    env.update(extra_env or {})
    p = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    return [json.loads(line) for line in p.stdout.splitlines() if line.startswith("{")]


def test_reference_arm_prints_one_contract_line():
    lines = _run()
    assert len(lines) == 1
    d = lines[0]
    sys.path.insert(0, ROOT)
    import bench

    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == bench.WORKLOAD


def test_reference_arm_other_ranks_exit_without_work():
    assert _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}) == []


def test_fp64_pipe_roofline_arithmetic():
    """The roofline object of the main leg, from the measured counters of the compiled 2->4 kernel
    (716.8 FP64 instructions, 1122.4 flops per event) at 6.28e8 events/s: 0.715 of the issue
    peak (152 SMs x 2 per clock x 2.07 GHz) and 0.56 of 1.25 TFLOP/s."""
    sys.path.insert(0, ROOT)
    import bench

    r = bench.fp64_pipe_roofline(716.8, 6.28e8, flops_per_event=1122.4)
    assert r["bound"] == "alu" and abs(r["peak"] - 629.28) < 1e-9
    assert abs(r["achieved"] - 450.15) < 0.01 and abs(r["frac"] - 0.7153) < 1e-4
    assert abs(r["flops"]["frac"] - 0.5639) < 1e-4
    n = bench.fp64_pipe_roofline(None, 6.28e8)
    assert n["achieved"] is None and n["frac"] is None and "flops" not in n


def test_summary_fits_the_line_tail():
    """Every leg's headline figure is repeated in one short `summary` object: with every leg
    present it holds no missing value and stays under 1200 characters, so the last 1.5 kB of the
    JSON line (where it is placed) carries all of them."""
    sys.path.insert(0, ROOT)
    import bench

    v = 123456789.0123
    line = {"value": v, "roofline": {"frac": 0.95, "frac_of_derived_peak": 0.79,
                                     "fp64_peak": {"dfma_ginstr_per_s": 528.1, "sm_count": 152},
                                     "method": {"fp64_pipe_equivalent_per_event": 1572.4}},
            "e2e": {"value": v}, "interpreter": {"value": v},
            "mixed_precision": {"value": v, "speedup_vs_fp64": 8.27, "fp64_pipe": {"frac": 0.74}},
            "multichannel": {"value": v, "roofline": {"frac": 0.91}, "mixed_precision": {"value": v}},
            "streamed_2to8": {"value": v, "roofline": {"frac": 0.97}, "e2e": {"value": v},
                              "mixed_precision": {"value": v}},
            "importance_2to8": {"mixed_n_eff_per_s_over_vegas_fp64": 12.17,
                                "flow_mixed_map_n_eff_per_s_over_vegas_fp64": 2.227,
                                "flow_n_eff_per_s_over_vegas_fp64": 0.8676},
            "flow": {"ess_fraction_flow": 0.9911, "ess_fraction_vegas": 0.9027, "ess_per_s_flow": 3.4e8,
                     "ess_per_s_vegas": 7.0e8, "mixed_map": {"ess_per_s_over_fp64_vegas": 0.7919},
                     "sample_ms": 15.81, "train_ms_per_step": 1.866, "train_steps": 20000},
            "unweighting": {"events_per_s": v}, "global_multichannel": {"events_per_s": v},
            "cpu_baseline": {"value": v, "cores": 16}}
    s = bench.summary(line)

    def leaves(d):
        for x in d.values():
            yield from (leaves(x) if isinstance(x, dict) else [x])

    assert all(x is not None for x in leaves(s))
    assert len(json.dumps(s)) < 1200
