"""Checkpoints of VEGAS grids and flow parameters (host only): exact round trips, the
little-endian layout, and rejection of damaged or mismatched files."""
import struct

import numpy as np
import pytest

from paper_2602_06895_gb300 import checkpoint as K
from paper_2602_06895_gb300 import workloads as W


def test_grids_round_trip_exactly(tmp_path):
    grids = [W.vegas_grid_random(3, 8, 64), None, W.vegas_grid_random(4, 22, 64), W.vegas_grid_uniform(2, 5)]
    p = tmp_path / "g.bin"
    K.save_grids(p, grids)
    back = K.load_grids(p)
    assert back[1] is None
    for a, b in zip(grids, back):
        if a is not None:
            assert b.dtype == np.float64 and np.array_equal(a, b)


def test_grid_file_layout_is_little_endian(tmp_path):
    g = W.vegas_grid_uniform(1, 2)  # one dimension, edges 0, 0.5, 1
    p = tmp_path / "g.bin"
    K.save_grids(p, [g])
    raw = p.read_bytes()
    assert raw[:8] == b"PSVEGAS1"
    assert struct.unpack("<III", raw[8:20]) == (1, 1, 2)
    assert struct.unpack("<3d", raw[20:44]) == (0.0, 0.5, 1.0) and len(raw) == 44


@pytest.mark.parametrize("damage", ["magic", "truncated", "trailing", "order"])
def test_damaged_grid_files_are_rejected(tmp_path, damage):
    p = tmp_path / "g.bin"
    K.save_grids(p, [W.vegas_grid_random(5, 3, 16)])
    raw = bytearray(p.read_bytes())
    if damage == "magic":
        raw[0] ^= 1
    elif damage == "truncated":
        raw = raw[:-8]
    elif damage == "trailing":
        raw += b"\0"
    else:  # swap two interior edges of the first row: no longer increasing
        a, b = 20 + 8, 20 + 16
        raw[a:a + 8], raw[b:b + 8] = raw[b:b + 8], raw[a:a + 8]
    p.write_bytes(bytes(raw))
    with pytest.raises(K.CheckpointError):
        K.load_grids(p)


def test_invalid_grids_are_not_written(tmp_path):
    g = W.vegas_grid_random(6, 2, 8)
    g[0, -1] = 0.999  # the last edge must be 1
    with pytest.raises(K.CheckpointError):
        K.save_grids(tmp_path / "g.bin", [g])


class _HostFlow:
    """Stands in for ps.Flow on the host: its shape and parameter vector."""

    def __init__(self, dims, n_layers, bins, hidden, n_params, seed):
        self.dims, self.n_layers, self.bins, self.hidden, self.n_params = dims, n_layers, bins, hidden, n_params
        self.p = np.random.default_rng(seed).standard_normal(n_params).astype(np.float32)

    def get_params(self):
        return self.p.copy()

    def set_params(self, p):
        self.p = np.array(p, dtype=np.float32)


def test_flow_round_trip_and_shape_check(tmp_path):
    a = _HostFlow(22, 6, 16, 128, 12345, 1)
    b = _HostFlow(22, 6, 16, 128, 12345, 2)
    p = tmp_path / "f.bin"
    K.save_flow(p, a)
    K.load_flow(p, b)
    assert np.array_equal(a.p, b.p)
    raw = p.read_bytes()
    assert raw[:8] == b"PSFLOW01" and struct.unpack("<IIIIQ", raw[8:32]) == (22, 6, 16, 128, 12345)
    with pytest.raises(K.CheckpointError):
        K.load_flow(p, _HostFlow(10, 6, 16, 128, 12345, 3))
    p.write_bytes(raw[:-4])
    with pytest.raises(K.CheckpointError):
        K.load_flow_params(p)
