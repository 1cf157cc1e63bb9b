"""Oracle pins: Philox4x32-10 against published known-answer vectors, the
bits -> (0,1) conversion and partition invariance of the counter-based stream."""
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def load_kat():
    rows = []
    with open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(t, 16) for t in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_philox_known_answers(oracle_mod):
    rows = load_kat()
    assert len(rows) == 3
    for ctr, key, want in rows:
        assert oracle_mod.philox(ctr, key) == want


def test_bits_to_unit_range_and_exactness(oracle_mod):
    assert oracle_mod.bits_to_unit(0) == 2.0 ** -53
    assert oracle_mod.bits_to_unit(2 ** 64 - 1) == 1.0 - 2.0 ** -53
    assert oracle_mod.bits_to_unit(1 << 63) == 0.5 + 2.0 ** -53
    # the low 12 bits are dropped
    assert oracle_mod.bits_to_unit((1 << 12) - 1) == 2.0 ** -53


def test_stream_is_partition_invariant(oracle_mod):
    full = oracle_mod.random(1234, 3, 1000, 257, 13)
    a = oracle_mod.random(1234, 3, 1000, 100, 13)
    b = oracle_mod.random(1234, 3, 1100, 157, 13)
    assert np.array_equal(full, np.vstack([a, b]))
    other = oracle_mod.random(1234, 4, 1000, 257, 13)
    assert not np.any(full == other)


def test_stream_uniformity(oracle_mod):
    r = oracle_mod.random(99, 0, 0, 200_000, 10).ravel()
    assert r.min() > 0.0 and r.max() < 1.0
    h, _ = np.histogram(r, bins=100, range=(0.0, 1.0))
    exp = r.size / 100
    chi2 = ((h - exp) ** 2 / exp).sum()
    assert chi2 < 100 + 5 * np.sqrt(200)  # 99 dof, ~5 sigma
    # Kolmogorov-Smirnov distance
    s = np.sort(r[:100_000])
    ks = np.max(np.abs(s - (np.arange(1, s.size + 1) - 0.5) / s.size))
    assert ks < 1.63 / np.sqrt(s.size) * 1.5
