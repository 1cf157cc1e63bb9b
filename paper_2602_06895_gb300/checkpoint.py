"""Checkpoints of what adaptation produces: VEGAS grids and flow parameters.

In the paper's validation runs the VEGAS grids are adapted and then frozen (section "Validation
and performance"), and its event generation keeps intermediate results for the final
combination and unweighting (section "Unweighting and file output", "Event generation"). With
the counter-based Philox generator, a run resumes from a checkpoint plus an event offset and
regenerates exactly the events it would have produced.

Formats (all little-endian, independent of the machine that wrote them):

* grids: ``b"PSVEGAS1"``, u32 channel count, then per channel u32 dims, u32 bins and
  dims x (bins + 1) f64 edges, row by row. A channel without VEGAS has dims = bins = 0. Every
  row must increase strictly from 0 to 1.
* flow: ``b"PSFLOW01"``, u32 dims, layers, bins, hidden, u64 parameter count, then the f32
  parameters in the order ``ps_flow_get_params`` gives them.
"""
from __future__ import annotations

import struct

import numpy as np

GRID_MAGIC = b"PSVEGAS1"
FLOW_MAGIC = b"PSFLOW01"


class CheckpointError(ValueError):
    pass


def _check_grid(a, c):
    if a.ndim != 2 or a.shape[1] < 2:
        raise CheckpointError(f"channel {c}: a grid is [dims][bins + 1] with bins >= 1")
    if not np.all(np.isfinite(a)) or np.any(a[:, 0] != 0.0) or np.any(a[:, -1] != 1.0) or \
            np.any(np.diff(a, axis=1) <= 0.0):
        raise CheckpointError(f"channel {c}: every row must increase strictly from 0 to 1")


def save_grids(path, grids):
    """Write one VEGAS grid per channel ([dims][bins + 1] edges, or None for no VEGAS)."""
    parts = [GRID_MAGIC, struct.pack("<I", len(grids))]
    for c, g in enumerate(grids):
        if g is None:
            parts.append(struct.pack("<II", 0, 0))
            continue
        a = np.asarray(g, dtype=np.float64)
        _check_grid(a, c)
        parts.append(struct.pack("<II", a.shape[0], a.shape[1] - 1))
        parts.append(a.astype("<f8").tobytes())
    with open(path, "wb") as f:
        f.write(b"".join(parts))


def load_grids(path):
    """The grids of a file written by save_grids (None for a channel without VEGAS)."""
    with open(path, "rb") as f:
        data = f.read()
    if data[:8] != GRID_MAGIC:
        raise CheckpointError("not a VEGAS grid checkpoint")
    pos = 8

    def take(n):
        nonlocal pos
        if pos + n > len(data):
            raise CheckpointError("truncated VEGAS grid checkpoint")
        b = data[pos:pos + n]
        pos += n
        return b

    (n_ch,) = struct.unpack("<I", take(4))
    grids = []
    for c in range(n_ch):
        dims, bins = struct.unpack("<II", take(8))
        if dims == 0:
            grids.append(None)
            continue
        a = np.frombuffer(take(8 * dims * (bins + 1)), dtype="<f8").reshape(dims, bins + 1).astype(np.float64)
        _check_grid(a, c)
        grids.append(a)
    if pos != len(data):
        raise CheckpointError("trailing bytes after the last grid")
    return grids


def save_program_grids(path, program, dims_per_channel, bins=64):
    """save_grids of a Program's current grids (dims_per_channel[c] = 0 for a channel without VEGAS)."""
    save_grids(path, [program.get_vegas(c, d, bins) if d else None for c, d in enumerate(dims_per_channel)])


def load_program_grids(path, program):
    """Upload the grids of a checkpoint into a Program (channels without VEGAS are skipped)."""
    for c, g in enumerate(load_grids(path)):
        if g is not None:
            program.set_vegas(c, g)


def save_flow_params(path, shape, params):
    """shape: dims, n_layers, bins, hidden; params: the flow's f32 parameter vector."""
    p = np.ascontiguousarray(params, dtype=np.float32).ravel()
    if not np.all(np.isfinite(p)):
        raise CheckpointError("non-finite flow parameters")
    head = struct.pack("<IIIIQ", shape["dims"], shape["n_layers"], shape["bins"], shape["hidden"], p.size)
    with open(path, "wb") as f:
        f.write(FLOW_MAGIC + head + p.astype("<f4").tobytes())


def load_flow_params(path):
    """(shape, params) of a file written by save_flow_params."""
    with open(path, "rb") as f:
        data = f.read()
    if data[:8] != FLOW_MAGIC or len(data) < 32:
        raise CheckpointError("not a flow checkpoint")
    dims, layers, bins, hidden, n = struct.unpack("<IIIIQ", data[8:32])
    if len(data) != 32 + 4 * n:
        raise CheckpointError("flow checkpoint size does not match its parameter count")
    params = np.frombuffer(data[32:], dtype="<f4").astype(np.float32)
    return {"dims": dims, "n_layers": layers, "bins": bins, "hidden": hidden}, params


def save_flow(path, flow):
    """Checkpoint a Flow (ps.Flow): its shape and parameters."""
    shape = {"dims": flow.dims, "n_layers": flow.n_layers, "bins": flow.bins, "hidden": flow.hidden}
    save_flow_params(path, shape, flow.get_params())


def load_flow(path, flow):
    """Load a checkpoint into a Flow of the same shape."""
    shape, params = load_flow_params(path)
    mine = {"dims": flow.dims, "n_layers": flow.n_layers, "bins": flow.bins, "hidden": flow.hidden}
    if shape != mine or params.size != flow.n_params:
        raise CheckpointError(f"flow checkpoint of shape {shape} ({params.size} parameters) does not fit a flow "
                              f"of shape {mine} ({flow.n_params} parameters)")
    flow.set_params(params)
