"""Host-side tests of the native library (no GPU needed): it loads, exports every
function declared in include/ps.h, validates graphs, and the topology builder
lays out the random dimensions as the oracle does."""
import os
import re

import pytest

from paper_2602_06895_gb300 import build as B
from paper_2602_06895_gb300 import ps
from paper_2602_06895_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    B.build()
    return ps.lib()


def header_functions():
    txt = open(os.path.join(ROOT, "include", "ps.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ps_[a-z0-9_]+)\s*\(", txt)))


def test_exports_every_declared_function(built):
    declared = header_functions()
    assert len(declared) >= 20
    for name in declared:
        assert hasattr(built, name), name
    assert set(ps.exported_symbols()) == set(declared)


def test_graph_validation_errors(built):
    g = ps.Graph.create(2)
    with pytest.raises(ps.PSError):
        g.add("TWO_BODY_DECAY_COM", [0, 1, 1e6, 0.0], 3)  # too few arguments
    with pytest.raises(ps.PSError):
        g.add("SQRT", [99], 1)  # undefined id
    with pytest.raises(ps.PSError):
        g.add(12345, [0], 1)  # unknown opcode
    p1, p2, j = g.add("TWO_BODY_DECAY_COM", [0, 1, 1e6, 0.0, 0.0], 3)
    with pytest.raises(ps.PSError):
        g.add("SQRT", [p1], 1)  # momentum where a scalar is expected
    with pytest.raises(ps.PSError):
        g.set_outputs([p1], [ps.ROLE_MOMENTUM])  # no weight
    g.set_outputs([p1, p2, j], [ps.ROLE_MOMENTUM, ps.ROLE_MOMENTUM, ps.ROLE_WEIGHT])
    with pytest.raises(ps.PSError):
        g.add("SQRT", [j], 1)  # graph is closed


def test_builder_dimensions_match_oracle(built, oracle_mod):
    chans = [W.two_body_fixed(), W.ww_hadronic()] + W.volume_topologies(3) + W.volume_topologies(4)
    chans += W.multichannel_2to5()
    for ch in chans:
        assert ps.channel_dims(ch) == oracle_mod.dims(ch) == W.n_random_dims(ch)


def test_builder_graph_listing(built):
    g = ps.build_channel([W.ww_hadronic()], 0)
    info = g.info()
    assert info["random"] == 10
    txt = g.dump()
    for op in ("vegas", "stable_invariant_nu", "breit_wigner_invariant", "r_to_x1x2", "com_p_in",
               "two_body_decay", "boost_beam", "reduce_product", "cut_unphysical"):
        assert op in txt, op
    multi = W.multichannel_2to5()
    txt = ps.build_channel(multi, 0).dump()
    for op in ("t_inv_min_max", "two_to_two_particle_scattering_com", "channel_weight", "momentum_sub"):
        assert op in txt, op


def test_builder_rejects_bad_topology(built):
    ch = W.ww_hadronic()
    ch["sorder"] = ch["sorder"][:1]
    with pytest.raises(ps.PSError):
        ps.build_channel([ch], 0)
    ch = W.ww_hadronic()
    ch["nodes"][1]["children"] = [3, 3]
    with pytest.raises(ps.PSError):
        ps.build_channel([ch], 0)


def test_program_without_device_fails_loudly(built):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a device is present")
    g = ps.build_channel([W.two_body_fixed()], 0)
    with pytest.raises(ps.PSError):
        ps.Program([g])


def test_flow_unweight_inverse_argument_checks(built):
    """The flow, unweighting, inverse and global-weight entry points reject bad arguments on the
    host, before touching a device."""
    import ctypes as C

    L = built
    h = C.c_void_p()
    assert L.ps_flow_create(1, 6, 16, 128, 1024, 1, 0, C.byref(h)) == ps.PS_ERR_INVALID_ARGUMENT  # dims < 2
    assert L.ps_flow_create(10, 9, 16, 128, 1024, 1, 0, C.byref(h)) == ps.PS_ERR_INVALID_ARGUMENT  # > 8 layers
    assert L.ps_flow_create(10, 6, 16, 100, 1024, 1, 0, C.byref(h)) == ps.PS_ERR_INVALID_ARGUMENT  # hidden % 16
    assert L.ps_flow_create(10, 6, 33, 128, 1024, 1, 0, C.byref(h)) == ps.PS_ERR_INVALID_ARGUMENT  # > 32 bins
    assert L.ps_flow_sample(None, 10, 1, 0, None, 10, None, None, None) == ps.PS_ERR_INVALID_ARGUMENT
    assert L.ps_flow_generate(None, 10, 1, 0, None, 10, None, None, None) == ps.PS_ERR_INVALID_ARGUMENT
    assert L.ps_flow_train_step(None, None, 1e-3, None) == ps.PS_ERR_INVALID_ARGUMENT
    assert L.ps_flow_free(None) == 0
    n = C.c_size_t()
    assert L.ps_unweight_workspace_size(-1, C.byref(n)) == ps.PS_ERR_INVALID_ARGUMENT
    assert L.ps_unweight_workspace_size(10_000_000, C.byref(n)) == 0 and n.value > 8 * 10_000_000 // 2048
    assert L.ps_unweight_max(None, 10, 1e-3, None, None, 0, None) == ps.PS_ERR_INVALID_ARGUMENT
    assert L.ps_unweight_max(None, 0, -1.0, None, None, 0, None) == ps.PS_ERR_INVALID_ARGUMENT
    assert L.ps_unweight_select(None, 10, None, 1, 0, None, None, None, None, 0, None) == ps.PS_ERR_INVALID_ARGUMENT
    assert L.ps_inverse_map(None, 0, None, 10, None, 10, None, None, None, 10, None, None) == \
        ps.PS_ERR_INVALID_ARGUMENT
    al = (C.c_double * 2)(0.5, -0.5)
    assert L.ps_global_weights(2, 0, None, 0, None, 0, al, None, None, 0.0, 0.0, None, None, None) == \
        ps.PS_ERR_INVALID_ARGUMENT  # negative channel weight
    assert L.ps_global_weights(0, 0, None, 0, None, 0, al, None, None, 0.0, 0.0, None, None, None) == \
        ps.PS_ERR_INVALID_ARGUMENT
    assert L.ps_flow_last_error().decode()  # the last failure left a message


def test_helper_kinds_checked_on_host(built):
    """ps_mixed_helpers (the map kernels' device helpers, exposed for their accuracy tests)
    validates the kind, the count and the pointers on the host: every declared kind accepts an
    empty request without touching a device, anything else is refused."""
    import ctypes as C

    L = built
    kinds = [ps.MIXED_HELPERS[k] for k in ("f2d", "d2f", "sqrt64", "rcp64", "sincos_turn", "tan_quarter")]
    assert kinds == list(range(6))
    for k in kinds:
        assert L.ps_mixed_helpers(k, None, None, 0, None) == 0
    buf = (C.c_double * 4)()
    for k in (-1, 6):
        assert L.ps_mixed_helpers(k, buf, buf, 4, None) == ps.PS_ERR_INVALID_ARGUMENT
    assert L.ps_mixed_helpers(5, buf, buf, -1, None) == ps.PS_ERR_INVALID_ARGUMENT
    assert L.ps_mixed_helpers(5, None, buf, 4, None) == ps.PS_ERR_INVALID_ARGUMENT
    assert L.ps_mixed_helpers(5, buf, None, 4, None) == ps.PS_ERR_INVALID_ARGUMENT
