"""The FP64 Breit-Wigner map's tangent table (csrc/tan_table.h, the committed output of
csrc/gen_tan_table.py) against the tangent itself, evaluated independently at 50 digits:

* kTanHi[k] + kTanLo[k] equals tan(k pi/512) to 2^-104 relative (a double-double: hi the
  correctly rounded double, lo the rounded remainder), for k = 0..128;
* kTanSq1[k] is 1 + kTanHi[k]^2 rounded to double;
* kTanH1 + kTanH2 is pi/512 to 2^-80 relative (kTanH2, about 2^-31 of the step, carries its own
  double rounding: the reduced angle is then off by at most 128 x 2^-80 h, far below an ulp of
  the tangent it feeds), kTanH1 has at most 30 significant bits (so that k kTanH1 is exact for
  k <= 128) and kTanInvH is 512/pi rounded to double.

Table points are where the device's tangent is exact up to one rounding, so a wrong entry would
show at once as an error at its point; this pins the data without a GPU.
"""
import os
import re

import pytest

mp = pytest.importorskip("mpmath")

HERE = os.path.dirname(os.path.abspath(__file__))
HDR = os.path.join(os.path.dirname(HERE), "paper_2602_06895_gb300", "csrc", "tan_table.h")


def _parse():
    text = open(HDR).read()
    arrays = {}
    for name, body in re.findall(r"double (\w+)\[\d+\] = \{([^}]*)\}", text):
        arrays[name] = [float.fromhex(v.strip()) for v in body.split(",") if v.strip()]
    consts = {name: float.fromhex(v) for name, v in re.findall(r"(kTan\w+) = (-?0x[0-9a-fA-Fp.+-]+)", text)}
    n = int(re.search(r"kTanN = (\d+);", text).group(1))
    return n, arrays, consts


def test_tangent_table_values():
    mp.mp.dps = 50
    n, arr, c = _parse()
    assert n == 128 and all(len(arr[k]) == n + 1 for k in ("kTanHi", "kTanLo", "kTanSq1"))
    for k in range(n + 1):
        t = mp.tan(k * mp.pi / (4 * n))
        hi, lo = arr["kTanHi"][k], arr["kTanLo"][k]
        assert hi == float(t), k  # the correctly rounded double
        if k:
            assert abs((mp.mpf(hi) + mp.mpf(lo)) / t - 1) < mp.mpf(2) ** -104, k
        else:
            assert hi == 0.0 and lo == 0.0
        assert arr["kTanSq1"][k] == float(1 + mp.mpf(hi) ** 2), k
    assert arr["kTanHi"][n] == 1.0


def test_tangent_step_split():
    mp.mp.dps = 50
    n, _, c = _parse()
    h = mp.pi / (4 * n)
    h1, h2 = c["kTanH1"], c["kTanH2"]
    assert abs((mp.mpf(h1) + mp.mpf(h2)) / h - 1) < mp.mpf(2) ** -80
    m, e = mp.frexp(mp.mpf(h1))
    assert (m * 2 ** 30) == int(m * 2 ** 30)  # at most 30 significant bits
    for k in range(n + 1):  # k h1 exact in double
        assert float(k * mp.mpf(h1)) == k * h1
    assert c["kTanInvH"] == float(1 / h)


def test_header_is_the_generators_output():
    """The committed header is exactly what gen_tan_table.py writes (no hand edits)."""
    import importlib.util

    gen = os.path.join(os.path.dirname(HDR), "gen_tan_table.py")
    spec = importlib.util.spec_from_file_location("gen_tan_table", gen)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    assert mod.render() == open(HDR).read()
