"""Writes tan_table.h: the tangent at the points k h, h = pi / 512, k = 0..128, of [0, pi/4] as
double-double pairs (hi, lo), 1 + hi^2, and the Cody-Waite split of h, for the table tangent of
the FP64 Breit-Wigner map (map_device.cuh).  The values are computed at 60 significant digits
with mpmath and rounded to double; run once, the output is committed:

    python paper_2602_06895_gb300/csrc/gen_tan_table.py
"""
import math
import os

import mpmath as mp

N = 128  # intervals of [0, pi/4]


def render():
    """The text of tan_table.h."""
    mp.mp.dps = 60
    h = mp.pi / (4 * N)
    hi, lo, sk = [], [], []
    for k in range(N + 1):
        t = mp.tan(k * h)
        th = float(t)
        hi.append(th)
        lo.append(float(t - mp.mpf(th)))
        sk.append(float(1 + mp.mpf(th) ** 2))
    hd = float(h)
    m, e = math.frexp(hd)
    h1 = math.ldexp(round(m * 2 ** 30), e - 30)  # 30 significant bits: k h1 is exact for k <= 128
    h2 = float(h - mp.mpf(h1))

    def arr(name, v):
        body = ",\n    ".join(", ".join(x.hex() for x in v[i:i + 4]) for i in range(0, len(v), 4))
        return f"static __device__ double {name}[{N + 1}] = {{\n    {body}}};\n"

    out = ["// tan_table.h -- written by gen_tan_table.py (mpmath, 60 digits); do not edit.",
           "// tan(k h) = kTanHi[k] + kTanLo[k] and kTanSq1[k] = 1 + kTanHi[k]^2 at h = pi / 512,",
           "// k = 0..128; h = kTanH1 + kTanH2 with kTanH1 of 30 significant bits, kTanInvH = 1 / h.",
           "// The arrays are read-only global memory (each translation unit its own copy, read through",
           "// the read-only cache): indexed per thread, they would serialise in the constant bank.",
           "#pragma once", "",
           f"constexpr int kTanN = {N};",
           f"constexpr double kTanH1 = {h1.hex()}, kTanH2 = {h2.hex()}, kTanInvH = {float(1 / h).hex()};",
           arr("kTanHi", hi), arr("kTanLo", lo), arr("kTanSq1", sk)]
    return "\n".join(out)


def main():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tan_table.h")
    with open(path, "w") as f:
        f.write(render())


if __name__ == "__main__":
    main()
