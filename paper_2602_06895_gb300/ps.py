"""Python binding of the C ABI in include/ps.h (ctypes; argument marshalling only).

Every computation runs in the native library ``libps.so`` (sm_103a kernels and
its host compiler).  There is no Python or CPU fallback: if the library is
missing or no CUDA device is present the calls raise.

The raw C functions are exported under their C names (``ps_graph_create``,
``ps_generate`` ...); :class:`Program` and :func:`build_channel` wrap them for
torch tensors (device memory and streams come from PyTorch).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libps.so")

PS_OK = 0
PS_ERR_INVALID_ARGUMENT, PS_ERR_GRAPH, PS_ERR_CUDA, PS_ERR_DEVICE_STATUS, PS_ERR_CAPACITY, PS_ERR_NO_DEVICE = -1, -2, -3, -4, -5, -6
MAX_NODES, MAX_LEGS = 32, 10

# opcodes (include/ps.h)
OPS = dict(VEGAS=1, INVARIANT_NU=2, INVARIANT_BW=3, R_TO_X1X2=4, COM_P_IN=5, T_INV_MIN_MAX=6, TWO_TO_TWO_COM=7,
           TWO_BODY_DECAY=8, TWO_BODY_DECAY_COM=9, BOOST_BEAM=10, REDUCE_PRODUCT=11, CUT_UNPHYSICAL=12, ADD=13,
           SUB=14, MUL=15, DIV=16, SQRT=17, SQUARE=18, MAX=19, MOM_ADD=20, MOM_SUB=21, PDF_POWER=22,
           PROPAGATOR=23, ONE_PLUS_COS2=24, CHANNEL_WEIGHT=25)
ROLE_MOMENTUM, ROLE_X1, ROLE_X2, ROLE_WEIGHT, ROLE_ALPHA = range(5)
ARG_VALUE, ARG_IMM = 0, 1
INTEGRAND = {"none": 0, "one_plus_cos2": 1, "pdf_props": 2, "pdf_sde": 3}
NODE = {"leaf": 0, "decay": 1, "tchain": 2}


class PSError(RuntimeError):
    pass


class Arg(C.Structure):
    _fields_ = [("kind", C.c_int32), ("id", C.c_int32), ("imm", C.c_double)]


class NodeDesc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_children", C.c_int32), ("children", C.c_int32 * MAX_LEGS),
                ("leaf_index", C.c_int32), ("in_sde", C.c_int32), ("mass", C.c_double),
                ("prop_mass", C.c_double), ("prop_width", C.c_double), ("nu", C.c_double)]


class ChannelDesc(C.Structure):
    _fields_ = [("n_out", C.c_int32), ("hadronic", C.c_int32), ("lab_frame", C.c_int32), ("integrand", C.c_int32),
                ("n_nodes", C.c_int32), ("n_sorder", C.c_int32), ("sorder", C.c_int32 * MAX_NODES),
                ("tside", C.c_int32 * MAX_LEGS), ("vegas_dims", C.c_int32), ("vegas_bins", C.c_int32),
                ("sqrt_s", C.c_double), ("s_beam", C.c_double), ("a_shift", C.c_double),
                ("shat_mass", C.c_double), ("shat_width", C.c_double), ("shat_nu", C.c_double),
                ("t_nu", C.c_double), ("ts_nu", C.c_double), ("t_prop_mass", C.c_double),
                ("pdf_alpha", C.c_double), ("pdf_beta", C.c_double), ("nodes", NodeDesc * MAX_NODES)]


class Options(C.Structure):
    _fields_ = [("block_threads", C.c_int32), ("ctas_per_sm", C.c_int32), ("precision", C.c_int32),
                ("flags", C.c_int32)]


class OutBuffers(C.Structure):
    _fields_ = [("momenta", C.c_void_p), ("x1", C.c_void_p), ("x2", C.c_void_p), ("weight", C.c_void_p),
                ("alpha", C.c_void_p), ("ld", C.c_int64)]


class ChannelStats(C.Structure):
    _fields_ = [("n", C.c_double), ("n_nonzero", C.c_double), ("sum_w", C.c_double), ("sum_w2", C.c_double),
                ("max_w", C.c_double)]


_lock = threading.Lock()
_lib = None

_SIGS = {
    "ps_last_error": (C.c_char_p, []),
    "ps_version": (C.c_int, []),
    "ps_graph_create": (C.c_int, [C.c_int, C.POINTER(C.c_void_p)]),
    "ps_graph_add": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(Arg), C.c_int, C.POINTER(C.c_int), C.c_int]),
    "ps_graph_set_outputs": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int), C.c_int]),
    "ps_graph_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "ps_graph_dump": (C.c_int, [C.c_void_p, C.c_char_p, C.c_size_t, C.POINTER(C.c_size_t)]),
    "ps_graph_free": (C.c_int, [C.c_void_p]),
    "ps_channel_dims": (C.c_int, [C.POINTER(ChannelDesc), C.POINTER(C.c_int)]),
    "ps_graph_build_channel": (C.c_int, [C.POINTER(ChannelDesc), C.c_int, C.c_int, C.POINTER(C.c_void_p)]),
    "ps_program_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.POINTER(Options), C.c_int,
                                    C.POINTER(C.c_void_p)]),
    "ps_program_set_vegas": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double)]),
    "ps_program_get_vegas": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double)]),
    "ps_workspace_size": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_size_t)]),
    "ps_generate": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.c_uint64, C.c_uint64, C.POINTER(OutBuffers),
                              C.c_void_p, C.c_size_t, C.c_void_p]),
    "ps_generate_noalloc": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.c_uint64, C.c_uint64,
                                      C.POINTER(OutBuffers), C.c_void_p]),
    "ps_map": (C.c_int, [C.c_void_p, C.c_int, C.c_int64, C.c_void_p, C.c_int64, C.POINTER(OutBuffers), C.c_void_p,
                         C.c_size_t, C.c_void_p]),
    "ps_exec_create": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(OutBuffers), C.c_void_p, C.c_size_t,
                                 C.POINTER(C.c_void_p)]),
    "ps_exec_launch": (C.c_int, [C.c_void_p, C.c_uint64, C.c_uint64, C.c_void_p]),
    "ps_exec_free": (C.c_int, [C.c_void_p]),
    "ps_stats": (C.c_int, [C.c_void_p, C.POINTER(ChannelStats), C.c_int, C.c_void_p]),
    "ps_stats_accumulate": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "ps_jit_check": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_char_p, C.c_size_t]),
    "ps_vegas_training": (C.c_int, [C.c_void_p, C.c_int]),
    "ps_vegas_histogram": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.c_void_p]),
    "ps_vegas_adapt": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.c_void_p]),
    "ps_status": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.c_int, C.c_void_p]),
    "ps_status_reset": (C.c_int, [C.c_void_p, C.c_void_p]),
    "ps_program_free": (C.c_int, [C.c_void_p]),
    "ps_launch_count": (C.c_int64, []),
    "ps_fp64_probe": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p]),
    "ps_mixed_helpers": (C.c_int, [C.c_int, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    "ps_inverse_map": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(ChannelDesc), C.c_int64, C.c_void_p, C.c_int64,
                                 C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "ps_global_weights": (C.c_int, [C.c_int, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                                    C.POINTER(C.c_double), C.c_void_p, C.c_void_p, C.c_double, C.c_double,
                                    C.c_void_p, C.c_void_p, C.c_void_p]),
    "ps_unweight_last_error": (C.c_char_p, []),
    "ps_unweight_workspace_size": (C.c_int, [C.c_int64, C.POINTER(C.c_size_t)]),
    "ps_unweight_max": (C.c_int, [C.c_void_p, C.c_int64, C.c_double, C.c_void_p, C.c_void_p, C.c_size_t,
                                  C.c_void_p]),
    "ps_unweight_select": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_uint64, C.c_uint64, C.c_void_p,
                                     C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "ps_flow_last_error": (C.c_char_p, []),
    "ps_flow_create": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int64, C.c_uint64, C.c_int,
                                 C.POINTER(C.c_void_p)]),
    "ps_flow_free": (C.c_int, [C.c_void_p]),
    "ps_flow_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                               C.POINTER(C.c_int), C.POINTER(C.c_int64)]),
    "ps_flow_mask": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "ps_flow_get_params": (C.c_int, [C.c_void_p, C.POINTER(C.c_float), C.c_int64]),
    "ps_flow_set_params": (C.c_int, [C.c_void_p, C.POINTER(C.c_float), C.c_int64]),
    "ps_flow_sample": (C.c_int, [C.c_void_p, C.c_int64, C.c_uint64, C.c_uint64, C.c_void_p, C.c_int64, C.c_void_p,
                                 C.c_void_p, C.c_void_p]),
    "ps_flow_generate": (C.c_int, [C.c_void_p, C.c_int64, C.c_uint64, C.c_uint64, C.c_void_p, C.c_int64,
                                   C.c_void_p, C.c_void_p, C.c_void_p]),
    "ps_flow_inverse": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                                  C.c_void_p]),
    "ps_flow_weights": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ps_flow_train_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_void_p]),
    "ps_flow_gradients": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_float), C.c_int64,
                                    C.POINTER(C.c_double), C.c_void_p]),
    "ps_flow_loss": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_void_p]),
    "ps_flow_status": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "ps_flow_set_wait_limit": (C.c_int, [C.c_void_p, C.c_int]),
    "ps_flow_set_debug": (C.c_int, [C.c_void_p, C.c_int]),
}


def lib():
    """Load libps.so (raises if it has not been built: there is no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise PSError(f"native library not built: {LIB_PATH} (run __graft_entry__.build())")
            L = C.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def _check(status, what=""):
    if status != PS_OK:
        msg = lib().ps_last_error().decode(errors="replace")
        raise PSError(f"{what} failed ({status}): {msg}")


def __getattr__(name):
    # raw C entry points under their C names (ps_graph_create, ps_generate, ...)
    if name in _SIGS:
        return getattr(lib(), name)
    raise AttributeError(name)


# ------------------------------------------------------------------ descriptions
def channel_desc(ch):
    """Workload channel dictionary -> ps_channel_desc."""
    d = ChannelDesc()
    d.n_out = ch["n"]
    d.hadronic = 1 if ch["hadronic"] else 0
    d.lab_frame = 0 if ch.get("partonic", False) else 1
    d.integrand = INTEGRAND[ch["integrand"]]
    nodes = ch["nodes"]
    d.n_nodes = len(nodes)
    for j, nd in enumerate(nodes):
        o = d.nodes[j]
        o.kind = NODE[nd["kind"]]
        kids = nd.get("children", [])
        o.n_children = len(kids)
        for k, kid in enumerate(kids):
            o.children[k] = kid
        o.leaf_index = nd.get("leaf", -1)
        o.in_sde = 1 if nd.get("sde", False) else 0
        o.mass = nd.get("mass", 0.0)
        o.prop_mass = nd.get("M", 0.0)
        o.prop_width = nd.get("G", 0.0)
        o.nu = nd.get("nu", 0.8)
    d.n_sorder = len(ch["sorder"])
    for i, j in enumerate(ch["sorder"]):
        d.sorder[i] = j
    for i, sd in enumerate(ch["tside"]):
        d.tside[i + 1] = sd
    d.vegas_dims = ch["vegas_dims"]
    d.vegas_bins = ch["vegas_bins"]
    d.sqrt_s = ch["sqrt_s"]
    d.s_beam = ch["S"]
    d.a_shift = ch["a"]
    d.shat_mass = ch["shat"]["M"]
    d.shat_width = ch["shat"]["G"]
    d.shat_nu = ch["shat"]["nu"]
    d.t_nu = ch["t_nu"]
    d.ts_nu = ch["ts_nu"]
    d.t_prop_mass = ch["Mt"]
    d.pdf_alpha, d.pdf_beta = ch["pdf"]
    return d


def channel_dims(ch):
    n = C.c_int()
    _check(lib().ps_channel_dims(C.byref(channel_desc(ch)), C.byref(n)), "ps_channel_dims")
    return n.value


class Graph:
    """Owning wrapper of a ps_graph handle."""

    def __init__(self, handle):
        self.h = C.c_void_p(handle)

    @classmethod
    def create(cls, n_random):
        h = C.c_void_p()
        _check(lib().ps_graph_create(n_random, C.byref(h)), "ps_graph_create")
        return cls(h.value)

    def add(self, opcode, args, n_out):
        """args: list of ("v", id) / ("i", value) or plain ints (values) / floats (immediates)."""
        arr = (Arg * max(len(args), 1))()
        for k, a in enumerate(args):
            if isinstance(a, tuple):
                kind, val = a
            else:
                kind, val = ("v", a) if isinstance(a, int) else ("i", a)
            if kind == "v":
                arr[k] = Arg(ARG_VALUE, int(val), 0.0)
            else:
                arr[k] = Arg(ARG_IMM, -1, float(val))
        outs = (C.c_int * max(n_out, 1))()
        _check(lib().ps_graph_add(self.h, OPS[opcode] if isinstance(opcode, str) else opcode, arr, len(args), outs,
                                  n_out), "ps_graph_add")
        return list(outs[:n_out])

    def set_outputs(self, ids, roles):
        n = len(ids)
        _check(lib().ps_graph_set_outputs(self.h, (C.c_int * n)(*ids), (C.c_int * n)(*roles), n),
               "ps_graph_set_outputs")

    def info(self):
        a, b, c = C.c_int(), C.c_int(), C.c_int()
        _check(lib().ps_graph_info(self.h, C.byref(a), C.byref(b), C.byref(c)), "ps_graph_info")
        return {"instructions": a.value, "values": b.value, "random": c.value}

    def dump(self):
        need = C.c_size_t()
        _check(lib().ps_graph_dump(self.h, None, 0, C.byref(need)), "ps_graph_dump")
        buf = C.create_string_buffer(need.value)
        _check(lib().ps_graph_dump(self.h, buf, need.value, C.byref(need)), "ps_graph_dump")
        return buf.value.decode()

    def __del__(self):
        if getattr(self, "h", None) and self.h.value and _lib is not None:
            _lib.ps_graph_free(self.h)
            self.h = C.c_void_p()


def build_channel(channels, which=0):
    """Graph of channel `which` of a list of workload channel dictionaries."""
    arr = (ChannelDesc * len(channels))(*[channel_desc(c) for c in channels])
    h = C.c_void_p()
    _check(lib().ps_graph_build_channel(arr, len(channels), which, C.byref(h)), "ps_graph_build_channel")
    return Graph(h.value)


def _stream_ptr(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


PRECISION = {"f64": 0, "mixed": 1}
PS_PROGRAM_JIT = 1


class Program:
    """A compiled multi-channel program on one device (ps_program)."""

    def __init__(self, graphs, block_threads=128, ctas_per_sm=0, device=0, precision="f64", jit=False):
        self.graphs = list(graphs)
        self.n_ch = len(self.graphs)
        self.precision = precision
        self.jit = bool(jit)
        hs = (C.c_void_p * self.n_ch)(*[g.h.value for g in self.graphs])
        opt = Options(block_threads, ctas_per_sm, PRECISION[precision], PS_PROGRAM_JIT if jit else 0)
        h = C.c_void_p()
        _check(lib().ps_program_create(hs, self.n_ch, C.byref(opt), device, C.byref(h)), "ps_program_create")
        self.h = h
        self.device = device
        self.n_random = [g.info()["random"] for g in self.graphs]

    def __del__(self):
        if getattr(self, "h", None) and self.h.value and _lib is not None:
            _lib.ps_program_free(self.h)
            self.h = C.c_void_p()

    # -- VEGAS
    def set_vegas(self, ch, edges):
        import numpy as np

        e = np.ascontiguousarray(edges, dtype=np.float64)
        _check(lib().ps_program_set_vegas(self.h, ch, e.shape[0], e.shape[1] - 1,
                                          e.ctypes.data_as(C.POINTER(C.c_double))), "ps_program_set_vegas")

    def get_vegas(self, ch, dims, bins=64):
        import numpy as np

        e = np.zeros((dims, bins + 1))
        _check(lib().ps_program_get_vegas(self.h, ch, dims, bins, e.ctypes.data_as(C.POINTER(C.c_double))),
               "ps_program_get_vegas")
        return e

    def vegas_training(self, on):
        _check(lib().ps_vegas_training(self.h, 1 if on else 0), "ps_vegas_training")

    def vegas_histogram(self, ch, dims, bins=64, stream=None):
        import numpy as np

        h = np.zeros((dims, bins))
        _check(lib().ps_vegas_histogram(self.h, ch, h.ctypes.data_as(C.POINTER(C.c_double)), _stream_ptr(stream)),
               "ps_vegas_histogram")
        return h

    def vegas_adapt(self, ch, alpha=1.5, stream=None):
        _check(lib().ps_vegas_adapt(self.h, ch, alpha, _stream_ptr(stream)), "ps_vegas_adapt")

    # -- buffers
    def workspace_size(self, events):
        ev = (C.c_int64 * self.n_ch)(*[int(e) for e in events])
        n = C.c_size_t()
        _check(lib().ps_workspace_size(self.h, ev, C.byref(n)), "ps_workspace_size")
        return n.value

    def alloc(self, events, n_momenta, x=True, alpha=False, device=None):
        """Output tensors (float64, CUDA) for `events` (list per channel) and a workspace."""
        import torch

        dev = torch.device("cuda", self.device if device is None else device)
        tot = int(sum(events))
        ft = torch.float32 if self.precision == "mixed" else torch.float64  # momenta, x, alpha
        out = {"momenta": torch.empty((4 * n_momenta, max(tot, 1)), dtype=ft, device=dev),
               "weight": torch.empty(max(tot, 1), dtype=torch.float64, device=dev)}
        if x:
            out["x1"] = torch.empty(max(tot, 1), dtype=ft, device=dev)
            out["x2"] = torch.empty(max(tot, 1), dtype=ft, device=dev)
        if alpha:
            out["alpha"] = torch.empty(max(tot, 1), dtype=ft, device=dev)
        ws = torch.empty(self.workspace_size(events) // 8 + 32, dtype=torch.float64, device=dev)
        return out, ws

    @staticmethod
    def _out_struct(out):
        m = out.get("momenta")
        if m is not None and m.shape[1] > 1 and m.stride(1) != 1:
            raise PSError("momenta must have unit stride along the events")
        ld = (m.stride(0) if m.shape[0] > 1 else m.shape[1]) if m is not None else 0
        return OutBuffers(_ptr(m), _ptr(out.get("x1")), _ptr(out.get("x2")), _ptr(out.get("weight")),
                          _ptr(out.get("alpha")), ld)

    @staticmethod
    def _ws(ws):
        base = ws.data_ptr()
        aligned = (base + 255) // 256 * 256
        return C.c_void_p(aligned), ws.numel() * ws.element_size() - (aligned - base)

    def generate(self, events, seed, out, ws, event_offset=0, stream=None):
        ev = (C.c_int64 * self.n_ch)(*[int(e) for e in events])
        o = self._out_struct(out)
        wp, wn = self._ws(ws)
        _check(lib().ps_generate(self.h, ev, seed, event_offset, C.byref(o), wp, wn, _stream_ptr(stream)),
               "ps_generate")

    def generate_noalloc(self, events, seed, out, event_offset=0, stream=None):
        """ps_generate_noalloc: the same generation without a workspace (fixed library scratch)."""
        ev = (C.c_int64 * self.n_ch)(*[int(e) for e in events])
        o = self._out_struct(out)
        _check(lib().ps_generate_noalloc(self.h, ev, seed, event_offset, C.byref(o), _stream_ptr(stream)),
               "ps_generate_noalloc")

    def map(self, ch, r, out, ws, stream=None):
        """r: float64 CUDA tensor [n_random, batch] (SoA, unit stride along the events)."""
        if r.dim() != 2 or (r.shape[1] > 1 and r.stride(1) != 1):
            raise PSError("r must be a [n_random, batch] tensor with unit stride along the batch")
        ld = r.stride(0) if r.shape[0] > 1 else r.shape[1]  # a size-1 dimension may carry any stride
        o = self._out_struct(out)
        wp, wn = self._ws(ws)
        _check(lib().ps_map(self.h, ch, r.shape[1], _ptr(r), ld, C.byref(o), wp, wn, _stream_ptr(stream)),
               "ps_map")

    def exec_create(self, events, out, ws):
        """Capture one generation for these counts and buffers into a CUDA graph (ps_exec)."""
        return Exec(self, events, out, ws)

    def stats(self, stream=None):
        arr = (ChannelStats * self.n_ch)()
        _check(lib().ps_stats(self.h, arr, self.n_ch, _stream_ptr(stream)), "ps_stats")
        return [{"n": s.n, "n_nonzero": s.n_nonzero, "sum_w": s.sum_w, "sum_w2": s.sum_w2, "max_w": s.max_w}
                for s in arr]

    def stats_accumulate(self, enable, stream=None):
        """Streaming mode (ps_stats_accumulate): zero the statistics and let every later launch add
        its per-channel sums; stats() then returns the running totals."""
        _check(lib().ps_stats_accumulate(self.h, 1 if enable else 0, _stream_ptr(stream)), "ps_stats_accumulate")

    def status(self, stream=None):
        arr = (C.c_int64 * 4)()
        _check(lib().ps_status(self.h, arr, 4, _stream_ptr(stream)), "ps_status")
        return {"nonfinite": arr[0], "cut": arr[1], "clamped": arr[2]}

    def status_reset(self, stream=None):
        _check(lib().ps_status_reset(self.h, _stream_ptr(stream)), "ps_status_reset")


def inverse_map(prog, ch, channel, momenta, x1, x2, r, P=None, stream=None):
    """r = G^-1(p) of program channel `ch` (workload dict `channel`): momenta [4 (n+2), B] and
    r [n_random, B] float64 CUDA tensors with unit stride along the events; x1, x2 [B] for hadronic
    channels; P [B] receives the channel's SDE weight (optional)."""
    B = momenta.shape[1]
    for t in (momenta, r):
        if t.dim() != 2 or (B > 1 and t.stride(1) != 1) or t.shape[1] < B:
            raise PSError("momenta and r must be [rows, batch] tensors with unit stride along the batch")
    d = channel_desc(channel)
    _check(lib().ps_inverse_map(prog.h, ch, C.byref(d), B, _ptr(momenta), momenta.stride(0), _ptr(x1), _ptr(x2),
                                _ptr(r), r.stride(0), _ptr(P), _stream_ptr(stream)), "ps_inverse_map")


def global_weights(J, alphas, w, P=None, x1=None, x2=None, pdf=(0.0, 0.0), f=None, stream=None):
    """Kleiss-Pittau weights w = f / sum_j alpha_j / J_j (ps_global_weights): J [M, B] (and P [M, B])
    float64 CUDA tensors; f defaults to pdf(x1) pdf(x2) sum_j P_j."""
    M, B = J.shape
    al = (C.c_double * M)(*[float(a) for a in alphas])
    ldp = P.stride(0) if P is not None else B
    _check(lib().ps_global_weights(M, B, _ptr(J), J.stride(0), _ptr(P), ldp, al, _ptr(x1), _ptr(x2), float(pdf[0]),
                                   float(pdf[1]), _ptr(f), _ptr(w), _stream_ptr(stream)), "ps_global_weights")


class Exec:
    """CUDA-graph executor of one generation (ps_exec): replay with a new seed and offset."""

    def __init__(self, prog, events, out, ws):
        self.prog = prog
        self.out, self.ws = out, ws  # the captured graph refers to these buffers
        ev = (C.c_int64 * prog.n_ch)(*[int(e) for e in events])
        o = Program._out_struct(out)
        wp, wn = Program._ws(ws)
        h = C.c_void_p()
        _check(lib().ps_exec_create(prog.h, ev, C.byref(o), wp, wn, C.byref(h)), "ps_exec_create")
        self.h = h

    def launch(self, seed, event_offset=0, stream=None):
        _check(lib().ps_exec_launch(self.h, seed, event_offset, _stream_ptr(stream)), "ps_exec_launch")

    def __del__(self):
        if getattr(self, "h", None) and self.h.value and _lib is not None:
            _lib.ps_exec_free(self.h)
            self.h = C.c_void_p()


def autotune(channels, events, precision="f64", blocks=(64, 128, 256), ctas=(1, 2, 3, 4), seed=1, reps=3,
             device=0, jit=False, pairs=None):
    """Pick block_threads and CTAs per SM for a workload by timing ps_generate on it.

    The candidates are blocks x ctas, or the (block_threads, ctas_per_sm) `pairs` when given.
    Every candidate compiles the program, generates the full event counts `reps` times after
    one warm-up and keeps the median CUDA-event time; returns (best options, table)."""
    import torch

    table = []
    for b, k in (pairs if pairs is not None else [(b, k) for b in blocks for k in ctas]):
        try:
            prog = program_for(channels, block_threads=b, ctas_per_sm=k, device=device, precision=precision,
                               jit=jit)
        except PSError:
            continue
        n_mom = channels[0]["n"] + 2
        out, ws = prog.alloc(events, n_mom, x=channels[0]["hadronic"],
                             alpha=channels[0]["integrand"] == "pdf_sde", device=device)
        prog.generate(events, seed, out, ws)
        times = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            prog.generate(events, seed, out, ws)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        times.sort()
        table.append({"block_threads": b, "ctas_per_sm": k, "ms": times[len(times) // 2]})
        del prog, out, ws
    best = min(table, key=lambda t: t["ms"])
    return {"block_threads": best["block_threads"], "ctas_per_sm": best["ctas_per_sm"]}, table


def launch_count():
    return lib().ps_launch_count()


PROBES = {"dfma": 0, "dadd": 1, "dmul": 2, "empty": 9, "div": 10, "sqrt": 11, "rsqrt": 12, "exp": 13,
          "expm1": 14, "log": 15, "log1p": 16, "pow": 17, "atan": 18, "atan2": 19, "tan": 20, "sin": 21,
          "cos": 22, "sincospi": 23}


def fp64_probe(kind, blocks, iters, sink, stream=None):
    """Launch one FP64-pipe probe (ps_fp64_probe) writing blocks x 256 doubles to `sink`."""
    _check(lib().ps_fp64_probe(PROBES[kind], blocks, iters, _ptr(sink), _stream_ptr(stream)), "ps_fp64_probe")


MIXED_HELPERS = {"f2d": 0, "d2f": 1, "sqrt64": 2, "rcp64": 3, "sincos_turn": 4, "tan_quarter": 5}


def mixed_helper(kind, x, out, stream=None):
    """Apply one device helper of the map kernels (ps_mixed_helpers) to the device tensor x into
    out (f2d: float32 -> float64; d2f: float64 -> float32; sqrt64, rcp64: float64 -> float64;
    sincos_turn: float64 r -> (cos 2 pi r, sin 2 pi r) pairs, out twice as long; tan_quarter:
    float64 x -> tan x for |x| <= pi/4)."""
    _check(lib().ps_mixed_helpers(MIXED_HELPERS[kind], _ptr(x), _ptr(out), x.numel(), _stream_ptr(stream)),
           "ps_mixed_helpers")


def program_for(channels, block_threads=128, ctas_per_sm=0, device=0, precision="f64", jit=False):
    """Build every channel of a workload list and compile them into one program (jit: the
    instruction lists compiled into one kernel at creation, PS_PROGRAM_JIT)."""
    graphs = [build_channel(channels, c) for c in range(len(channels))]
    return Program(graphs, block_threads=block_threads, ctas_per_sm=ctas_per_sm, device=device,
                   precision=precision, jit=jit)


def jit_check(channels, block_threads=128, precision="f64"):
    """Generate and compile (NVRTC, no device) the kernel of a compiled program; returns the log."""
    graphs = [build_channel(channels, c) for c in range(len(channels))]
    hs = (C.c_void_p * len(graphs))(*[g.h.value for g in graphs])
    opt = Options(block_threads, 0, PRECISION[precision], PS_PROGRAM_JIT)
    log = C.create_string_buffer(1 << 16)
    _check(lib().ps_jit_check(hs, len(graphs), C.byref(opt), log, len(log)), "ps_jit_check")
    return log.value.decode(errors="replace")


# ------------------------------------------------------------------ coupling flow (ps_flow_*)
def _fcheck(status, what=""):
    if status != PS_OK:
        msg = lib().ps_flow_last_error().decode(errors="replace")
        raise PSError(f"{what} failed ({status}): {msg}")


class Flow:
    """Rational-quadratic-spline coupling flow on one device (ps_flow): the learned proposal
    that feeds r into :meth:`Program.map`."""

    def __init__(self, dims, n_layers=6, bins=16, hidden=128, max_batch=1 << 16, init_seed=1, device=0):
        h = C.c_void_p()
        _fcheck(lib().ps_flow_create(dims, n_layers, bins, hidden, max_batch, init_seed, device, C.byref(h)),
                "ps_flow_create")
        self.h, self.device, self.max_batch = h, device, max_batch
        d, L, K, H, n = C.c_int(), C.c_int(), C.c_int(), C.c_int(), C.c_int64()
        _fcheck(lib().ps_flow_info(h, C.byref(d), C.byref(L), C.byref(K), C.byref(H), C.byref(n)), "ps_flow_info")
        self.dims, self.n_layers, self.bins, self.hidden, self.n_params = d.value, L.value, K.value, H.value, n.value

    def __del__(self):
        if getattr(self, "h", None) and self.h.value and _lib is not None:
            _lib.ps_flow_free(self.h)
            self.h = C.c_void_p()

    def mask(self, layer):
        arr, n = (C.c_int * self.dims)(), C.c_int()
        _fcheck(lib().ps_flow_mask(self.h, layer, arr, C.byref(n)), "ps_flow_mask")
        return list(arr[: n.value])

    def get_params(self):
        import numpy as np

        p = np.zeros(self.n_params, dtype=np.float32)
        _fcheck(lib().ps_flow_get_params(self.h, p.ctypes.data_as(C.POINTER(C.c_float)), self.n_params),
                "ps_flow_get_params")
        return p

    def set_params(self, p):
        import numpy as np

        p = np.ascontiguousarray(p, dtype=np.float32)
        _fcheck(lib().ps_flow_set_params(self.h, p.ctypes.data_as(C.POINTER(C.c_float)), p.size),
                "ps_flow_set_params")

    def sample(self, batch, seed, r, logdet=None, z=None, event_offset=0, stream=None):
        """r (and z): float64 CUDA tensors [dims, >= batch] with unit stride along the events."""
        if r.dim() != 2 or r.shape[0] != self.dims or r.shape[1] < batch or (r.shape[1] > 1 and r.stride(1) != 1):
            raise PSError("r must be a [dims, batch] tensor with unit stride along the batch")
        if z is not None and z.stride() != r.stride():
            raise PSError("z must have the layout of r")
        ld = r.stride(0)
        _fcheck(lib().ps_flow_sample(self.h, batch, seed, event_offset, _ptr(r), ld, _ptr(logdet), _ptr(z),
                                     _stream_ptr(stream)), "ps_flow_sample")

    def generate(self, batch, seed, r, logdet=None, z=None, event_offset=0, stream=None):
        """Inference sampling (ps_flow_generate): same outputs as sample(), any batch size."""
        if r.dim() != 2 or r.shape[0] != self.dims or r.shape[1] < batch or (r.shape[1] > 1 and r.stride(1) != 1):
            raise PSError("r must be a [dims, batch] tensor with unit stride along the batch")
        if z is not None and z.stride() != r.stride():
            raise PSError("z must have the layout of r")
        _fcheck(lib().ps_flow_generate(self.h, batch, seed, event_offset, _ptr(r), r.stride(0), _ptr(logdet),
                                       _ptr(z), _stream_ptr(stream)), "ps_flow_generate")

    def inverse(self, r, z, logq=None, stream=None):
        """z = flow^-1(r), logq = log g(r): float64 CUDA tensors [dims, batch] and [batch]."""
        if r.dim() != 2 or r.shape[0] != self.dims or (r.shape[1] > 1 and r.stride(1) != 1) or z.stride() != r.stride():
            raise PSError("r and z must be [dims, batch] tensors of one layout with unit stride along the batch")
        _fcheck(lib().ps_flow_inverse(self.h, r.shape[1], _ptr(r), r.stride(0), _ptr(z), _ptr(logq),
                                      _stream_ptr(stream)), "ps_flow_inverse")

    def weights(self, w_map, logdet, w, stream=None):
        _fcheck(lib().ps_flow_weights(self.h, w_map.numel(), _ptr(w_map), _ptr(logdet), _ptr(w),
                                      _stream_ptr(stream)), "ps_flow_weights")

    def train_step(self, w_map, lr, stream=None):
        _fcheck(lib().ps_flow_train_step(self.h, _ptr(w_map), lr, _stream_ptr(stream)), "ps_flow_train_step")

    def gradients(self, w_map, stream=None):
        import numpy as np

        g = np.zeros(self.n_params, dtype=np.float32)
        loss = C.c_double()
        _fcheck(lib().ps_flow_gradients(self.h, _ptr(w_map), g.ctypes.data_as(C.POINTER(C.c_float)), self.n_params,
                                        C.byref(loss), _stream_ptr(stream)), "ps_flow_gradients")
        return loss.value, g

    def status(self):
        """Tensor-core waits of the fused sampling kernels that ran out since the last call
        (0 in a healthy run); clears the count."""
        v = C.c_int64()
        _fcheck(lib().ps_flow_status(self.h, C.byref(v)), "ps_flow_status")
        return v.value

    def set_wait_limit(self, polls):
        """Bound of the fused kernels' completion waits in polls (<= 0: the default)."""
        _fcheck(lib().ps_flow_set_wait_limit(self.h, int(polls)), "ps_flow_set_wait_limit")

    def set_debug(self, flags):
        """Test flags of the fused kernels (bit 0: withhold the first completion signal; bit 1: the
        training forward layer by layer instead of the tcgen05 layer kernel)."""
        _fcheck(lib().ps_flow_set_debug(self.h, int(flags)), "ps_flow_set_debug")

    def loss(self, stream=None):
        loss, sw = C.c_double(), C.c_double()
        _fcheck(lib().ps_flow_loss(self.h, C.byref(loss), C.byref(sw), _stream_ptr(stream)), "ps_flow_loss")
        return loss.value, sw.value


def flow_param_layout(dims, n_layers, bins, hidden, masks):
    """Logical parameter layout of a flow: list over layers of {name: (offset, shape)}."""
    out, o = [], 0
    for l in range(n_layers):
        nb = len(masks[l])
        na = dims - nb
        P = nb * (3 * bins + 1)
        lay = {}
        for name, shape in (("W1", (hidden, na)), ("b1", (hidden,)), ("W2", (hidden, hidden)), ("b2", (hidden,)),
                            ("W3", (P, hidden)), ("b3", (P,))):
            n = 1
            for x in shape:
                n *= x
            lay[name] = (o, shape)
            o += n
        out.append(lay)
    return out, o


# ------------------------------------------------------------------ unweighting (ps_unweight_*)
def _ucheck(status, what=""):
    if status != PS_OK:
        msg = lib().ps_unweight_last_error().decode(errors="replace")
        raise PSError(f"{what} failed ({status}): {msg}")


class Unweighter:
    """Maximum weight with a bounded over-weight share and accept/reject (ps_unweight_*) for
    batches of up to `capacity` weights on one device."""

    def __init__(self, capacity, device=0):
        import torch

        n = C.c_size_t()
        _ucheck(lib().ps_unweight_workspace_size(capacity, C.byref(n)), "ps_unweight_workspace_size")
        self.capacity = capacity
        self._ws = torch.empty(n.value // 8 + 64, dtype=torch.float64, device=torch.device("cuda", device))
        self.result = torch.zeros(5, dtype=torch.float64, device=self._ws.device)
        self.n_accepted = torch.zeros(1, dtype=torch.int64, device=self._ws.device)

    def _wsp(self):
        base = self._ws.data_ptr()
        aligned = (base + 255) // 256 * 256
        return C.c_void_p(aligned), self._ws.numel() * 8 - (aligned - base)

    def max_weight(self, w, eps=1e-3, stream=None):
        """Fills self.result = [w_max, sum w, max w, n over w_max, n invalid] (asynchronous)."""
        if w.numel() > self.capacity:
            raise PSError("more weights than the unweighter's capacity")
        wp, wn = self._wsp()
        _ucheck(lib().ps_unweight_max(_ptr(w), w.numel(), eps, _ptr(self.result), wp, wn, _stream_ptr(stream)),
                "ps_unweight_max")
        return self.result

    def select(self, w, seed, idx, w_out, event_offset=0, w_max=None, stream=None):
        """Accept against w_max (device scalar; default self.result[0]); fills idx, w_out and
        self.n_accepted (asynchronous)."""
        if w.numel() > self.capacity:
            raise PSError("more weights than the unweighter's capacity")
        wm = self.result[0:1] if w_max is None else w_max
        wp, wn = self._wsp()
        _ucheck(lib().ps_unweight_select(_ptr(w), w.numel(), _ptr(wm), seed, event_offset, _ptr(idx), _ptr(w_out),
                                         _ptr(self.n_accepted), wp, wn, _stream_ptr(stream)), "ps_unweight_select")
