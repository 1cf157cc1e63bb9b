"""Canary-padded outputs: a generation of B events writes the first B columns of every output and
nothing beyond them. The padding keeps a value no output can take, and no written column keeps it.
Ragged tiles, empty channels and both kernels (the interpreter and a compiled program) are
covered."""
import pytest

from paper_2602_06895_gb300 import ps
from paper_2602_06895_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CANARY = -7.0e300  # no momentum component, weight, x or alpha is ever this
PAD = 300


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2602_06895_gb300 import build

    build.build()
    return torch


@pytest.mark.parametrize("case", [("2to5", False), ("ww", True)], ids=["interpreter_2to5", "compiled_2to4"])
def test_outputs_stay_inside_their_columns(torch_cuda, case):
    torch = torch_cuda
    name, jit = case
    if name == "2to5":
        chans, counts, n_mom = W.multichannel_2to5(), [129, 0, 1, 0, 0, 257], 7
    else:
        chans, counts, n_mom = [W.ww_hadronic()], [1000], 6
    prog = ps.program_for(chans, jit=jit)
    B = sum(counts)
    keys = ["weight", "x1", "x2"] + (["alpha"] if chans[0]["integrand"] == "pdf_sde" else [])
    out = {"momenta": torch.full((4 * n_mom, B + PAD), CANARY, dtype=torch.float64, device="cuda")}
    for k in keys:
        out[k] = torch.full((B + PAD,), CANARY, dtype=torch.float64, device="cuda")
    ws = torch.empty(prog.workspace_size(counts) // 8 + 32, dtype=torch.float64, device="cuda")
    prog.generate(counts, 11, out, ws)
    torch.cuda.synchronize()
    for k, v in out.items():
        assert bool(torch.all(v[..., B:] == CANARY)), (k, "written past the last event")
        assert not bool(torch.any(v[..., :B] == CANARY)), (k, "an event's column left unwritten")
