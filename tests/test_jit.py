"""Compiled programs (PS_PROGRAM_JIT): the generated kernel compiles for sm_103a with NVRTC on the
host (no device), and keeps every slot in registers (no local-memory frame beyond the math
library's, no spills)."""
import re

import pytest

from paper_2602_06895_gb300 import ps
from paper_2602_06895_gb300 import workloads as W


def _stats(log):
    stack = [int(m) for m in re.findall(r"(\d+) bytes stack frame", log)]
    spills = [int(m) for m in re.findall(r"(\d+) bytes spill stores", log)]
    return max(stack), max(spills)


def test_compiled_2to4_builds_in_registers(monkeypatch):
    monkeypatch.setenv("PS_JIT_PTXAS_VERBOSE", "1")
    for precision in ("f64", "mixed"):
        log = ps.jit_check([W.ww_hadronic()], 128, precision)
        stack, spills = _stats(log)
        assert spills == 0 and stack <= 64, (precision, log)


def test_compiled_channel_weights_stay_in_registers(monkeypatch):
    """The six 2->5 channels, each with the SDE weights of all six: the weights are generated as
    straight-line code, so the register frame is never indexed at run time."""
    monkeypatch.setenv("PS_JIT_PTXAS_VERBOSE", "1")
    chans = W.multichannel_2to5()
    log = ps.jit_check(chans, 128, "f64")
    stack, spills = _stats(log)
    assert spills == 0 and stack <= 64, log


@pytest.mark.parametrize("precision", ["f64", "mixed"])
def test_split_program_compiles_and_links(monkeypatch, precision):
    """The split form (one NVRTC unit per channel, compiled in parallel as relocatable code, linked
    with nvJitLink into one kernel), forced on the six 2->5 channels."""
    monkeypatch.setenv("PS_JIT_SPLIT", "1")
    monkeypatch.setenv("PS_JIT_PTXAS_VERBOSE", "1")
    log = ps.jit_check(W.multichannel_2to5(), 128, precision)
    assert "ps_jit_map" in log, log


def test_channel_weight_invariants_named_once(monkeypatch, tmp_path):
    """The generated channel weights of the six 2->5 channels declare each distinct invariant once
    (110 propagator factors over 35 momentum sums) and reuse it; a write to a slot an invariant
    reads would end its reuse."""
    dump = tmp_path / "src.cu"
    monkeypatch.setenv("PS_JIT_DUMP", str(dump))
    ps.jit_check(W.multichannel_2to5(), 128, "f64")
    src = dump.read_text()
    decls = re.findall(r"const double (cw\d+) = dev::p4_sq\(", src)
    uses = re.findall(r"dev::sde_factor_s\(den, P, (cw\d+),", src)
    assert len(uses) == 110 and len(decls) == 35  # the names restart in each channel's scope
    assert set(uses) == set(decls)


def test_cta_request_becomes_launch_bounds(monkeypatch, tmp_path):
    """A program asking for k CTAs per SM gets a compiled kernel that fits them: launch bounds
    (block, k) on the kernel and, in the split form, the matching register cap on the channel
    units (65536 / (128 x 4) = 128 registers)."""
    dump = tmp_path / "src.cu"
    monkeypatch.setenv("PS_JIT_DUMP", str(dump))
    monkeypatch.setenv("PS_JIT_SPLIT", "1")
    import ctypes as C

    chans = W.multichannel_2to5()
    graphs = [ps.build_channel(chans, c) for c in range(len(chans))]
    hs = (C.c_void_p * len(graphs))(*[g.h.value for g in graphs])
    opt = ps.Options(128, 4, ps.PRECISION["f64"], ps.PS_PROGRAM_JIT)
    log = C.create_string_buffer(1 << 16)
    assert ps.lib().ps_jit_check(hs, len(graphs), C.byref(opt), log, len(log)) == 0, log.value
    src = dump.read_text()
    assert "__launch_bounds__(128, 4)" in src
    assert src.rstrip().endswith("// maxrregcount 128")


def test_jit_check_rejects_bad_arguments():
    """ps_jit_check returns an error status (never aborts) for a null graph list, a channel count
    out of range, a null graph, or a log buffer that is missing while its size is not zero."""
    import ctypes as C

    L = ps.lib()
    g = ps.build_channel([W.ww_hadronic()], 0)
    one = (C.c_void_p * 1)(g.h.value)
    opt = ps.Options(128, 0, ps.PRECISION["f64"], ps.PS_PROGRAM_JIT)
    buf = C.create_string_buffer(256)
    assert L.ps_jit_check(None, 1, C.byref(opt), buf, len(buf)) != 0
    assert L.ps_jit_check(one, 0, C.byref(opt), buf, len(buf)) != 0
    assert L.ps_jit_check(one, 1000, C.byref(opt), buf, len(buf)) != 0
    assert L.ps_jit_check((C.c_void_p * 1)(None), 1, C.byref(opt), buf, len(buf)) != 0
    assert L.ps_jit_check(one, 1, C.byref(opt), None, 16) != 0
    assert "ps_jit_check" in L.ps_last_error().decode()
