"""Python binding of the NDGSBP C ABI (include/ndgsbp.h).

Argument marshalling only: every step of decoding runs in the CUDA library.  Device buffers
are torch tensors (their data_ptr() is passed through), streams are torch CUDA streams.
Importing this module loads paper_1202_1060_gb300/_lib/libndgsbp.so and raises if it is
missing -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libndgsbp.so")
if not os.path.exists(_LIB_PATH):
    raise ImportError(f"NDGSBP CUDA library not built ({_LIB_PATH} missing): run "
                      "`python -c 'import __graft_entry__ as g; g.build()'` first")
_lib = ctypes.CDLL(_LIB_PATH)

OK = 0
ERR_INVALID, ERR_INFEASIBLE, ERR_CUDA, ERR_WORKSPACE = -1, -2, -3, -4
ERR_BUDGET, ERR_TIMEOUT, ERR_DEVICE, ERR_UNSUPPORTED, ERR_NOMEM = -5, -6, -7, -8, -9
F32, F16, BF16, F64 = 0, 1, 2, 3
UNIT_CN, UNIT_LAYER = 0, 1
GROUPS_CYCLIC, GROUPS_NATURAL, GROUPS_STRUCTURED = 1, 2, 4
SCHEDULE_GROUPS, SCHEDULE_FLOOD = 0, 1
VARIANT_AUTO, VARIANT_SMEM, VARIANT_GLOBAL, VARIANT_QC, VARIANT_QC_GLOBAL = 0, 1, 2, 3, 4
VARIANT_TILE = 7
VARIANT_STREAM, VARIANT_STREAM_SMEM, VARIANT_STREAM_GLOBAL, VARIANT_STREAM_BULK = 12, 13, 14, 15
VARIANT_RAGGED_PER_CODE = 11   # ragged launches: each code on its own plan, forked streams
TUNE_TILE_ONLY = 1
GA_PHI_EXACT, GA_PHI_CLOSED = 0, 1
STAT_FRAMES, STAT_FRAME_ERRORS, STAT_BIT_ERRORS, STAT_UNDETECTED = 0, 1, 2, 3
STAT_ITERATIONS, STAT_UNSATISFIED, STAT_INVALID, STATS_LEN = 4, 5, 6, 8


class NdgsbpError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"[{status}] {message}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("schedule", ctypes.c_int32), ("max_iter", ctypes.c_int32),
                ("msg_dtype", ctypes.c_int32), ("llr_max", ctypes.c_float),
                ("early_stop", ctypes.c_int32), ("variant", ctypes.c_int32),
                ("block_threads", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("frames_per_cta", ctypes.c_int32), ("lanes_per_cn", ctypes.c_int32)]


class Plan(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int32), ("block_threads", ctypes.c_int32),
                ("grid", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("max_row_degree", ctypes.c_int32), ("delta_in_smem", ctypes.c_int32),
                ("smem_bytes", ctypes.c_int64), ("workspace_bytes", ctypes.c_int64),
                ("stored_edges", ctypes.c_int64), ("edge_updates_per_iter", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Extras(ctypes.Structure):
    _fields_ = [("d_ref_bits", ctypes.c_void_p), ("ref_per_frame", ctypes.c_int32),
                ("d_stats", ctypes.c_void_p), ("d_iter_hist", ctypes.c_void_p),
                ("d_start_ns", ctypes.c_void_p), ("d_retire_ns", ctypes.c_void_p),
                ("d_messages", ctypes.c_void_p)]


class Batch(ctypes.Structure):
    _fields_ = [("groups", ctypes.c_void_p), ("d_llr", ctypes.c_void_p), ("llr_dtype", ctypes.c_int32),
                ("n_frames", ctypes.c_int64), ("d_hard_bits", ctypes.c_void_p), ("d_iters", ctypes.c_void_p),
                ("d_syndrome_ok", ctypes.c_void_p), ("d_posterior", ctypes.c_void_p), ("d_stats", ctypes.c_void_p),
                ("d_start_ns", ctypes.c_void_p), ("d_retire_ns", ctypes.c_void_p),
                ("frames_per_cta", ctypes.c_int32), ("lanes_per_cn", ctypes.c_int32)]


class TuneResult(ctypes.Structure):
    _fields_ = [("best", Params), ("best_ms", ctypes.c_double), ("default_ms", ctypes.c_double),
                ("candidates", ctypes.c_int32), ("from_cache", ctypes.c_int32)]


class ServerStats(ctypes.Structure):
    _fields_ = [("requests_submitted", ctypes.c_int64), ("requests_completed", ctypes.c_int64),
                ("frames_completed", ctypes.c_int64), ("frame_errors_unsatisfied", ctypes.c_int64),
                ("epochs", ctypes.c_int64), ("iterations", ctypes.c_int64), ("busy_seconds", ctypes.c_double),
                ("slots_total", ctypes.c_int64), ("slots_in_use", ctypes.c_int64),
                ("admit_seconds", ctypes.c_double), ("device_seconds", ctypes.c_double),
                ("harvest_seconds", ctypes.c_double), ("launches", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_P, _I32, _I64, _U64, _D, _U32 = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                                  ctypes.c_double, ctypes.c_uint32)
_SIGS = {
    "ndgsbp_params_default": (None, [ctypes.POINTER(Params)]),
    "ndgsbp_last_error": (ctypes.c_char_p, []),
    "ndgsbp_version": (ctypes.c_char_p, []),
    "ndgsbp_code_create": (_I32, [_P, _P, _I32, _I32, _I32, ctypes.POINTER(_P)]),
    "ndgsbp_code_destroy": (_I32, [_P]),
    "ndgsbp_code_info": (_I32, [_P, _P, _P, _P, _P, _P, _P]),
    "ndgsbp_group_sizes": (_I32, [_I32, _I32, _D, _I32, _P, _P]),
    "ndgsbp_groups_build": (_I32, [_P, _I32, _D, _U64, _I32, _I32, ctypes.POINTER(_P)]),
    "ndgsbp_groups_from_lists": (_I32, [_P, _P, _P, _I32, ctypes.POINTER(_P)]),
    "ndgsbp_groups_build_cycled": (_I32, [_P, _I32, _D, _U64, _I32, _I32, _I32, ctypes.POINTER(_P)]),
    "ndgsbp_groups_query_grouping": (_I32, [_P, _I32, _P, _P, _P, _P]),
    "ndgsbp_groups_query": (_I32, [_P, _P, _P, _P, _P, _P, _P, _P]),
    "ndgsbp_groups_destroy": (_I32, [_P]),
    "ndgsbp_vgroups_build": (_I32, [_P, _I32, _U64, _I32, ctypes.POINTER(_P)]),
    "ndgsbp_vgroups_from_lists": (_I32, [_P, _P, _P, _I32, ctypes.POINTER(_P)]),
    "ndgsbp_vgroups_query": (_I32, [_P, _P, _P, _P, _P]),
    "ndgsbp_vgroups_destroy": (_I32, [_P]),
    "ndgsbp_vertical_workspace_size": (_I32, [_P, ctypes.POINTER(Params), _I64, ctypes.POINTER(ctypes.c_size_t)]),
    "ndgsbp_decode_vertical": (_I32, [_P, ctypes.POINTER(Params), _P, _I32, _I64, _P, ctypes.c_size_t,
                                      _P, _P, _P, _P, ctypes.POINTER(Extras), _P]),
    "ndgsbp_awgn_llr": (_I32, [_P, _I64, _D, _D, _U64, _P, _I32, _P, _I32, _P]),
    "ndgsbp_philox4x32_10": (_I32, [_P, _U32, _U32, _I64, _P, _P]),
    "ndgsbp_decode_plan": (_I32, [_P, ctypes.POINTER(Params), _I64, ctypes.POINTER(Plan)]),
    "ndgsbp_workspace_size": (_I32, [_P, ctypes.POINTER(Params), _I64, ctypes.POINTER(ctypes.c_size_t)]),
    "ndgsbp_decode": (_I32, [_P, ctypes.POINTER(Params), _P, _I32, _I64, _P, ctypes.c_size_t,
                             _P, _P, _P, _P, _P]),
    "ndgsbp_decode_ex": (_I32, [_P, ctypes.POINTER(Params), _P, _I32, _I64, _P, ctypes.c_size_t,
                                _P, _P, _P, _P, ctypes.POINTER(Extras), _P]),
    "ndgsbp_decode_static": (_I32, [_P, ctypes.POINTER(Params), _P, _I32, _I64, _P, _P, _P, _P, _P]),
    "ndgsbp_workspace_status": (_I32, [_P, ctypes.POINTER(_U32), _P]),
    "ndgsbp_test_hooks": (_I32, [_I32, _U32]),
    "ndgsbp_mufu_probe": (_I32, [_I32, _I64, _I32, _I32, _P, _P]),
    "ndgsbp_ragged_create": (_I32, [_P, _I32, ctypes.POINTER(Params), ctypes.POINTER(_P)]),
    "ndgsbp_ragged_info": (_I32, [_P, ctypes.POINTER(Plan), _P]),
    "ndgsbp_ragged_launch": (_I32, [_P, _P]),
    "ndgsbp_ragged_graph_launch": (_I32, [_P, _P]),
    "ndgsbp_ragged_destroy": (_I32, [_P]),
    "ndgsbp_autotune": (_I32, [_P, ctypes.POINTER(Params), _P, _I32, _I64, _I32, ctypes.c_char_p,
                               ctypes.POINTER(TuneResult)]),
    "ndgsbp_ragged_autotune": (_I32, [_P, _I32, ctypes.POINTER(Params), _I64, ctypes.c_char_p,
                                      ctypes.POINTER(Params), ctypes.POINTER(_D)]),
    "ndgsbp_ga_flood": (_I32, [_P, _I32, _P, _I32, _D, _P, _I32, _I32, _I32, _D, _P, _P, _P]),
    "ndgsbp_ga_groups": (_I32, [_P, _I32, _P, _I32, _D, _I32, _D, _P, _I32, _I32, _I32, _D, _P, _P, _P]),
    "ndgsbp_ga_groups_threshold": (_I32, [_P, _I32, _P, _I32, _D, _I32, _D, _I32, _I32, _D, _D, _D, _D,
                                          ctypes.POINTER(_D)]),
    "ndgsbp_ga_flood_threshold": (_I32, [_P, _I32, _P, _I32, _D, _I32, _I32, _D, _D, _D, _D,
                                         ctypes.POINTER(_D)]),
    "ndgsbp_server_create": (_I32, [_P, _I32, _P, ctypes.POINTER(Params), ctypes.c_size_t, _I32,
                                    ctypes.POINTER(_P)]),
    "ndgsbp_server_submit": (_I32, [_P, _I32, _P, _I64, _P, _P, _P, ctypes.POINTER(_I64)]),
    "ndgsbp_server_poll": (_I32, [_P, _I64, ctypes.POINTER(_I32), ctypes.POINTER(_D)]),
    "ndgsbp_server_wait": (_I32, [_P, _I64, _I32, ctypes.POINTER(_D)]),
    "ndgsbp_server_stats_get": (_I32, [_P, ctypes.POINTER(ServerStats)]),
    "ndgsbp_server_destroy": (_I32, [_P]),
}
STATIC_SCRATCH_BYTES = 16 * 1024 * 1024


def _bind(lib, sigs):
    for name, (res, args) in sigs.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args


_bind(_lib, _SIGS)
DECLARED_SYMBOLS = tuple(_SIGS)


def library_path() -> str:
    return _LIB_PATH


def last_error() -> str:
    return _lib.ndgsbp_last_error().decode()


def version() -> str:
    return _lib.ndgsbp_version().decode()


def _check(status: int):
    if status != OK:
        raise NdgsbpError(status, last_error())


def _dptr(t):
    """Device pointer of a torch tensor (or None)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _addr(t):
    """Device address of a CUDA tensor as an int (None for None)."""
    return None if t is None else _dptr(t).value


def _hptr(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _stream(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(getattr(stream, "cuda_stream", stream) or 0)


def params_default(**overrides) -> Params:
    p = Params()
    _lib.ndgsbp_params_default(ctypes.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


def group_sizes(M_units: int, G: int, r: float, flags: int = 0):
    ng, o = ctypes.c_int32(), ctypes.c_int32()
    _check(_lib.ndgsbp_group_sizes(M_units, G, float(r), flags, ctypes.byref(ng), ctypes.byref(o)))
    return ng.value, o.value


class Code:
    """Owned ndgsbp_code handle (ndgsbp_code_create / ndgsbp_code_destroy)."""

    def __init__(self, row_ptr, col_idx, M: int, N: int, lift_Z: int = 0):
        rp = np.ascontiguousarray(row_ptr, np.int32)
        ci = np.ascontiguousarray(col_idx, np.int32)
        h = ctypes.c_void_p()
        _check(_lib.ndgsbp_code_create(_hptr(rp), _hptr(ci), M, N, lift_Z, ctypes.byref(h)))
        self._h = h
        self.M, self.N, self.E, self.Z = M, N, int(rp[-1]), lift_Z

    @classmethod
    def from_inputs(cls, code):
        """From a paper_1202_1060_gb300.inputs.Code."""
        return cls(code.row_ptr, code.col_idx, code.M, code.N, code.Z)

    @property
    def handle(self):
        return self._h

    def info(self):
        M, N, mr, mc, Z = (ctypes.c_int32() for _ in range(5))
        E = ctypes.c_int64()
        _check(_lib.ndgsbp_code_info(self._h, ctypes.byref(M), ctypes.byref(N), ctypes.byref(E),
                                     ctypes.byref(mr), ctypes.byref(mc), ctypes.byref(Z)))
        return dict(M=M.value, N=N.value, E=E.value, max_row_degree=mr.value,
                    max_col_degree=mc.value, lift_Z=Z.value)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _lib.ndgsbp_code_destroy(h)
            self._h = None


class Groups:
    """Owned ndgsbp_groups handle (Step 1 grouping plus its device layout)."""

    def __init__(self, handle, code: Code):
        self._h = handle
        self.code = code

    @classmethod
    def build(cls, code: Code, G: int, r: float, seed: int, unit: int = UNIT_CN, flags: int = 0,
              n_groupings: int = 1):
        """ndgsbp_groups_build, or with n_groupings > 1 ndgsbp_groups_build_cycled (groupings cycled
        by iteration)."""
        h = ctypes.c_void_p()
        if n_groupings == 1:
            _check(_lib.ndgsbp_groups_build(code.handle, G, float(r), seed & (2**64 - 1), unit, flags,
                                            ctypes.byref(h)))
        else:
            _check(_lib.ndgsbp_groups_build_cycled(code.handle, G, float(r), seed & (2**64 - 1), unit, flags,
                                                   int(n_groupings), ctypes.byref(h)))
        return cls(h, code)

    def groupings(self):
        """All groupings cycled by iteration: list of (grp_ptr, cn_idx)."""
        K = ctypes.c_int32()
        _check(_lib.ndgsbp_groups_query_grouping(self._h, 0, ctypes.byref(K), None, None, None))
        out = []
        for k in range(K.value):
            n = ctypes.c_int64()
            _check(_lib.ndgsbp_groups_query_grouping(self._h, k, None, ctypes.byref(n), None, None))
            gp = np.zeros(self.query()["G"] + 1, np.int32)
            gc = np.zeros(n.value, np.int32)
            _check(_lib.ndgsbp_groups_query_grouping(self._h, k, None, None, _hptr(gp), _hptr(gc)))
            out.append((gp, gc))
        return out

    @classmethod
    def from_lists(cls, code: Code, grp_ptr, cn_idx):
        gp = np.ascontiguousarray(grp_ptr, np.int32)
        gc = np.ascontiguousarray(cn_idx, np.int32)
        h = ctypes.c_void_p()
        _check(_lib.ndgsbp_groups_from_lists(code.handle, _hptr(gp), _hptr(gc), len(gp) - 1,
                                             ctypes.byref(h)))
        return cls(h, code)

    @property
    def handle(self):
        return self._h

    def query(self):
        G, n = ctypes.c_int32(), ctypes.c_int64()
        _check(_lib.ndgsbp_groups_query(self._h, ctypes.byref(G), ctypes.byref(n), None, None,
                                        None, None, None))
        gp = np.zeros(G.value + 1, np.int32)
        gc = np.zeros(n.value, np.int32)
        cocsg = ctypes.c_double()
        cnu, edu = ctypes.c_int64(), ctypes.c_int64()
        _check(_lib.ndgsbp_groups_query(self._h, None, None, _hptr(gp), _hptr(gc), ctypes.byref(cocsg),
                                        ctypes.byref(cnu), ctypes.byref(edu)))
        return dict(G=G.value, grp_ptr=gp, cn_idx=gc, cocsg=cocsg.value,
                    cn_updates_per_iter=cnu.value, edge_updates_per_iter=edu.value)

    def plan(self, params: Params, n_frames: int) -> Plan:
        pl = Plan()
        _check(_lib.ndgsbp_decode_plan(self._h, ctypes.byref(params), n_frames, ctypes.byref(pl)))
        return pl

    def workspace_size(self, params: Params, n_frames: int) -> int:
        b = ctypes.c_size_t()
        _check(_lib.ndgsbp_workspace_size(self._h, ctypes.byref(params), n_frames, ctypes.byref(b)))
        return b.value

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _lib.ndgsbp_groups_destroy(h)
            self._h = None


class VGroups:
    """Owned ndgsbp_vgroups handle: VN groups of the vertical shuffled schedule."""

    def __init__(self, handle, code: Code):
        self._h = handle
        self.code = code

    @classmethod
    def build(cls, code: Code, G: int, seed: int, flags: int = 0):
        h = ctypes.c_void_p()
        _check(_lib.ndgsbp_vgroups_build(code.handle, G, seed & (2**64 - 1), flags, ctypes.byref(h)))
        return cls(h, code)

    @classmethod
    def from_lists(cls, code: Code, grp_ptr, grp_vn):
        gp = np.ascontiguousarray(grp_ptr, np.int32)
        gv = np.ascontiguousarray(grp_vn, np.int32)
        h = ctypes.c_void_p()
        _check(_lib.ndgsbp_vgroups_from_lists(code.handle, _hptr(gp), _hptr(gv), len(gp) - 1, ctypes.byref(h)))
        return cls(h, code)

    @property
    def handle(self):
        return self._h

    def query(self):
        G, me = ctypes.c_int32(), ctypes.c_int32()
        _check(_lib.ndgsbp_vgroups_query(self._h, ctypes.byref(G), None, None, None))
        gp = np.zeros(G.value + 1, np.int32)
        gv = np.zeros(self.code.N, np.int32)
        _check(_lib.ndgsbp_vgroups_query(self._h, None, _hptr(gp), _hptr(gv), ctypes.byref(me)))
        return dict(G=G.value, grp_ptr=gp, grp_vn=gv, max_group_edges=me.value)

    def workspace_size(self, params: Params, n_frames: int) -> int:
        b = ctypes.c_size_t()
        _check(_lib.ndgsbp_vertical_workspace_size(self._h, ctypes.byref(params), n_frames, ctypes.byref(b)))
        return b.value

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _lib.ndgsbp_vgroups_destroy(h)
            self._h = None


_DT = {}


def dtype_code(t) -> int:
    import torch
    if not _DT:
        _DT.update({torch.float32: F32, torch.float16: F16, torch.bfloat16: BF16, torch.float64: F64})
    return _DT[t.dtype]


def awgn_llr(code: Code, n_frames: int, ebn0_db: float, rate: float, seed: int, out,
             codeword_bits=None, codeword_per_frame: bool = False, stream=None):
    """ndgsbp_awgn_llr into the CUDA tensor ``out`` [n_frames, N] (float32/16/bf16)."""
    _check(_lib.ndgsbp_awgn_llr(code.handle, n_frames, float(ebn0_db), float(rate), seed & (2**64 - 1),
                                _dptr(codeword_bits), int(codeword_per_frame), _dptr(out),
                                dtype_code(out), _stream(stream)))
    return out


def philox4x32_10(ctr, key0: int, key1: int, out, stream=None):
    """Raw Philox4x32-10 blocks: ctr, out are CUDA int32/uint32 tensors [n, 4]."""
    _check(_lib.ndgsbp_philox4x32_10(_dptr(ctr), key0 & 0xFFFFFFFF, key1 & 0xFFFFFFFF, ctr.shape[0],
                                     _dptr(out), _stream(stream)))
    return out


def decode(groups: Groups, params: Params, llr, workspace, hard_bits, iters=None, syndrome_ok=None,
           posterior=None, ref_bits=None, ref_per_frame: bool = False, stats=None, iter_hist=None,
           start_ns=None, retire_ns=None, messages=None, stream=None):
    """ndgsbp_decode_ex on CUDA tensors; llr is [n_frames, N]."""
    n_frames = llr.shape[0]
    ex = Extras(d_ref_bits=_addr(ref_bits), ref_per_frame=int(ref_per_frame), d_stats=_addr(stats),
                d_iter_hist=_addr(iter_hist), d_start_ns=_addr(start_ns), d_retire_ns=_addr(retire_ns),
                d_messages=_addr(messages))
    _check(_lib.ndgsbp_decode_ex(groups.handle, ctypes.byref(params), _dptr(llr), dtype_code(llr), n_frames,
                                 _dptr(workspace), workspace.numel() * workspace.element_size(),
                                 _dptr(hard_bits), _dptr(iters), _dptr(syndrome_ok), _dptr(posterior),
                                 ctypes.byref(ex), _stream(stream)))


def decode_vertical(vgroups: VGroups, params: Params, llr, workspace, hard_bits, iters=None, syndrome_ok=None,
                    posterior=None, ref_bits=None, ref_per_frame: bool = False, stats=None, iter_hist=None,
                    start_ns=None, retire_ns=None, messages=None, stream=None):
    """ndgsbp_decode_vertical on CUDA tensors; llr is [n_frames, N]."""
    ex = Extras(d_ref_bits=_addr(ref_bits), ref_per_frame=int(ref_per_frame), d_stats=_addr(stats),
                d_iter_hist=_addr(iter_hist), d_start_ns=_addr(start_ns), d_retire_ns=_addr(retire_ns),
                d_messages=_addr(messages))
    _check(_lib.ndgsbp_decode_vertical(vgroups.handle, ctypes.byref(params), _dptr(llr), dtype_code(llr),
                                       llr.shape[0], _dptr(workspace), workspace.numel() * workspace.element_size(),
                                       _dptr(hard_bits), _dptr(iters), _dptr(syndrome_ok), _dptr(posterior),
                                       ctypes.byref(ex), _stream(stream)))


def decode_plain(groups: Groups, params: Params, llr, workspace, hard_bits, iters=None, syndrome_ok=None,
                 posterior=None, stream=None):
    """ndgsbp_decode (no extras)."""
    _check(_lib.ndgsbp_decode(groups.handle, ctypes.byref(params), _dptr(llr), dtype_code(llr), llr.shape[0],
                              _dptr(workspace), workspace.numel() * workspace.element_size(),
                              _dptr(hard_bits), _dptr(iters), _dptr(syndrome_ok), _dptr(posterior),
                              _stream(stream)))


def decode_static(groups: Groups, params: Params, llr, hard_bits, iters=None, syndrome_ok=None,
                  posterior=None, stream=None):
    """ndgsbp_decode_static: decode without a workspace (the library's static scratch array).
    The grouping must have been planned on this device first (Groups.plan)."""
    _check(_lib.ndgsbp_decode_static(groups.handle, ctypes.byref(params), _dptr(llr), dtype_code(llr),
                                     llr.shape[0], _dptr(hard_bits), _dptr(iters), _dptr(syndrome_ok),
                                     _dptr(posterior), _stream(stream)))


def workspace_status(workspace, stream=None) -> int:
    """ndgsbp_workspace_status: the status word of the last decode that used ``workspace``."""
    v = ctypes.c_uint32(0)
    _check(_lib.ndgsbp_workspace_status(_dptr(workspace), ctypes.byref(v), _stream(stream)))
    return int(v.value)


def test_hooks(skip_first_bulk_load: int = 0, wait_polls: int = 0):
    """ndgsbp_test_hooks: drive the bulk-staged stream kernel's bounded waits to give up (tests)."""
    _check(_lib.ndgsbp_test_hooks(int(skip_first_bulk_load), int(wait_polls)))


def mufu_probe(op: int, iters: int, blocks: int, threads: int, sink, stream=None):
    """ndgsbp_mufu_probe: blocks x threads x iters x 8 MUFU operations of kind op (0 ex2, 1 rcp, 2 lg2)."""
    _check(_lib.ndgsbp_mufu_probe(int(op), int(iters), int(blocks), int(threads), _dptr(sink), _stream(stream)))


def _batch_array(batches):
    arr = (Batch * len(batches))()
    for i, b in enumerate(batches):
        llr = b["llr"]
        arr[i] = Batch(groups=b["groups"].handle.value, d_llr=_addr(llr), llr_dtype=dtype_code(llr),
                       n_frames=llr.shape[0], d_hard_bits=_addr(b["hard_bits"]), d_iters=_addr(b.get("iters")),
                       d_syndrome_ok=_addr(b.get("syndrome_ok")), d_posterior=_addr(b.get("posterior")),
                       d_stats=_addr(b.get("stats")), d_start_ns=_addr(b.get("start_ns")),
                       d_retire_ns=_addr(b.get("retire_ns")), frames_per_cta=int(b.get("frames_per_cta", 0)),
                       lanes_per_cn=int(b.get("lanes_per_cn", 0)))
    return arr


def autotune(groups: Groups, params: Params, llr, flags: int = 0, cache_path: str | None = None):
    """ndgsbp_autotune on the frames of llr (CUDA tensor [F, N]): returns (best Params, info dict)."""
    r = TuneResult()
    _check(_lib.ndgsbp_autotune(groups.handle, ctypes.byref(params), _dptr(llr), dtype_code(llr), llr.shape[0],
                                int(flags), None if cache_path is None else cache_path.encode(), ctypes.byref(r)))
    best = Params.from_buffer_copy(r.best)
    return best, {"best_ms": r.best_ms, "default_ms": r.default_ms, "candidates": r.candidates,
                  "from_cache": bool(r.from_cache)}


def ragged_autotune(batches, params: Params, sample_frames: int = 0, cache_path: str | None = None):
    """ndgsbp_ragged_autotune: sets frames_per_cta / lanes_per_cn in each batch dict and returns
    (Params for the launch, launch ms)."""
    arr = _batch_array(batches)
    out = Params()
    ms = ctypes.c_double()
    _check(_lib.ndgsbp_ragged_autotune(arr, len(batches), ctypes.byref(params), int(sample_frames),
                                       None if cache_path is None else cache_path.encode(), ctypes.byref(out),
                                       ctypes.byref(ms)))
    for i, b in enumerate(batches):
        b["frames_per_cta"] = arr[i].frames_per_cta
        b["lanes_per_cn"] = arr[i].lanes_per_cn
    return out, ms.value


class Ragged:
    """ndgsbp_ragged handle: one persistent launch over batches of several codes.  Each batch is
    a dict with groups, llr (CUDA tensor [F, N]) and output tensors hard_bits, iters,
    syndrome_ok, posterior, stats, start_ns, retire_ns (optional), frames_per_cta, lanes_per_cn."""

    def __init__(self, batches, params: Params):
        arr = _batch_array(batches)
        self._keep = batches
        h = ctypes.c_void_p()
        _check(_lib.ndgsbp_ragged_create(arr, len(batches), ctypes.byref(params), ctypes.byref(h)))
        self._h = h

    def info(self):
        pl = Plan()
        n = ctypes.c_int32()
        _check(_lib.ndgsbp_ragged_info(self._h, ctypes.byref(pl), ctypes.byref(n)))
        return pl.as_dict(), n.value

    def launch(self, stream=None):
        _check(_lib.ndgsbp_ragged_launch(self._h, _stream(stream)))

    def graph_launch(self, stream=None):
        _check(_lib.ndgsbp_ragged_graph_launch(self._h, _stream(stream)))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _lib.ndgsbp_ragged_destroy(h)
            self._h = None


class Server:
    """ndgsbp_server handle: continuous batching of decode requests over device-resident frame
    slots.  codes is a list of Groups (QC codes grouped in whole layers); weights split
    hbm_budget_bytes between their pools.  submit() takes host FP32 LLRs [F, N] and returns a
    Request whose host outputs are filled when it completes."""

    class Request:
        def __init__(self, server, ticket, llr, hard, iters, ok, N):
            self.server, self.ticket, self.N = server, ticket, N
            self._llr, self.hard_words, self.iters, self.syndrome_ok = llr, hard, iters, ok
            self.latency_ms = None

        def done(self) -> bool:
            if self.latency_ms is None:
                d, lat = ctypes.c_int32(), ctypes.c_double()
                _check(_lib.ndgsbp_server_poll(self.server._h, self.ticket, ctypes.byref(d), ctypes.byref(lat)))
                if d.value:
                    self._finish(lat.value)
            return self.latency_ms is not None

        def wait(self, timeout_ms: int = 60000) -> float:
            """Block until done; returns the request latency in ms (host clock)."""
            if self.latency_ms is None:
                lat = ctypes.c_double()
                _check(_lib.ndgsbp_server_wait(self.server._h, self.ticket, int(timeout_ms), ctypes.byref(lat)))
                self._finish(lat.value)
            return self.latency_ms

        def _finish(self, lat):
            self.latency_ms = lat
            self.server._live.pop(self.ticket, None)

        def hard_bits(self):
            return unpack_bits(self.hard_words, self.N)

    def __init__(self, codes, params: Params, hbm_budget_bytes: int, epoch_iters: int = 1, weights=None):
        arr = (ctypes.c_void_p * len(codes))(*[g.handle.value for g in codes])
        w = None if weights is None else np.ascontiguousarray(weights, np.float64)
        h = ctypes.c_void_p()
        self._codes = list(codes)
        self._live = {}   # requests in flight: their host buffers stay alive until completion
        _check(_lib.ndgsbp_server_create(arr, len(codes), _hptr(w), ctypes.byref(params), int(hbm_budget_bytes),
                                         int(epoch_iters), ctypes.byref(h)))
        self._h = h

    def submit(self, code: int, llr) -> "Server.Request":
        llr = np.ascontiguousarray(llr, np.float32)
        F, N = llr.shape
        hard = np.zeros((F, (N + 31) // 32), np.uint32)
        iters = np.zeros(F, np.int32)
        ok = np.zeros(F, np.uint8)
        t = ctypes.c_int64()
        _check(_lib.ndgsbp_server_submit(self._h, int(code), _hptr(llr), F, _hptr(hard), _hptr(iters), _hptr(ok),
                                         ctypes.byref(t)))
        req = Server.Request(self, t.value, llr, hard, iters, ok, N)
        self._live[t.value] = req
        return req

    def stats(self) -> dict:
        st = ServerStats()
        _check(_lib.ndgsbp_server_stats_get(self._h, ctypes.byref(st)))
        return st.as_dict()

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _lib.ndgsbp_server_destroy(h)
            self._h = None
            self._live.clear()

    def __del__(self):
        self.close()


def _degree_array(frac: dict):
    d = max(frac)
    a = np.zeros(d + 1, np.float64)
    for k, v in frac.items():
        a[k] = v
    return a, d


def ga_flood(lam: dict, rho: dict, rate: float, ebn0_db, phi_kind: int = GA_PHI_EXACT, max_iter: int = 20000,
             mu_cap: float = 60.0):
    """ndgsbp_ga_flood: (converged bool [n], iterations int [n], mu_c [n]) for each Eb/N0."""
    la, dv = _degree_array(lam)
    ra, dc = _degree_array(rho)
    e = np.ascontiguousarray(np.atleast_1d(ebn0_db), np.float64)
    n = e.size
    cv = np.zeros(n, np.uint8)
    it = np.zeros(n, np.int32)
    mu = np.zeros(n, np.float64)
    _check(_lib.ndgsbp_ga_flood(_hptr(la), dv, _hptr(ra), dc, float(rate), _hptr(e), n, int(phi_kind),
                                int(max_iter), float(mu_cap), _hptr(cv), _hptr(it), _hptr(mu)))
    return cv.astype(bool), it, mu


def ga_flood_threshold(lam: dict, rho: dict, rate: float, phi_kind: int = GA_PHI_EXACT, lo_db: float = 0.0,
                       hi_db: float = 3.0, tol_db: float = 1e-4, max_iter: int = 20000, mu_cap: float = 60.0) -> float:
    la, dv = _degree_array(lam)
    ra, dc = _degree_array(rho)
    out = ctypes.c_double()
    _check(_lib.ndgsbp_ga_flood_threshold(_hptr(la), dv, _hptr(ra), dc, float(rate), int(phi_kind), int(max_iter),
                                          float(mu_cap), float(lo_db), float(hi_db), float(tol_db),
                                          ctypes.byref(out)))
    return out.value


def ga_groups(lam: dict, rho: dict, rate: float, G: int, r: float, ebn0_db, phi_kind: int = GA_PHI_EXACT,
              max_iter: int = 20000, mu_cap: float = 60.0):
    """ndgsbp_ga_groups: (converged bool [n], iterations int [n], mu_c [n]) for each Eb/N0."""
    la, dv = _degree_array(lam)
    ra, dc = _degree_array(rho)
    e = np.ascontiguousarray(np.atleast_1d(ebn0_db), np.float64)
    n = e.size
    cv = np.zeros(n, np.uint8)
    it = np.zeros(n, np.int32)
    mu = np.zeros(n, np.float64)
    _check(_lib.ndgsbp_ga_groups(_hptr(la), dv, _hptr(ra), dc, float(rate), int(G), float(r), _hptr(e), n,
                                 int(phi_kind), int(max_iter), float(mu_cap), _hptr(cv), _hptr(it), _hptr(mu)))
    return cv.astype(bool), it, mu


def ga_groups_threshold(lam: dict, rho: dict, rate: float, G: int, r: float, phi_kind: int = GA_PHI_EXACT,
                        lo_db: float = 0.0, hi_db: float = 3.0, tol_db: float = 1e-4, max_iter: int = 20000,
                        mu_cap: float = 60.0) -> float:
    la, dv = _degree_array(lam)
    ra, dc = _degree_array(rho)
    out = ctypes.c_double()
    _check(_lib.ndgsbp_ga_groups_threshold(_hptr(la), dv, _hptr(ra), dc, float(rate), int(G), float(r), int(phi_kind),
                                           int(max_iter), float(mu_cap), float(lo_db), float(hi_db), float(tol_db),
                                           ctypes.byref(out)))
    return out.value


def unpack_bits(words, N: int):
    """Packed decisions [F, W] (int32/uint32, numpy or torch) -> uint8 [F, N] (host)."""
    a = words.cpu().numpy() if hasattr(words, "cpu") else np.asarray(words)
    a = np.ascontiguousarray(a).view(np.uint32)
    bits = ((a[:, :, None] >> np.arange(32, dtype=np.uint32)) & 1).astype(np.uint8)
    return bits.reshape(a.shape[0], -1)[:, :N]


def pack_bits(bits):
    """uint8 [F, N] or [N] (host) -> packed uint32 words as int32 numpy [F, W] / [W]."""
    b = np.atleast_2d(np.asarray(bits, np.uint8))
    F, N = b.shape
    W = (N + 31) // 32
    pad = np.zeros((F, W * 32), np.uint64)
    pad[:, :N] = b
    words = (pad.reshape(F, W, 32) << np.arange(32, dtype=np.uint64)).sum(axis=2).astype(np.uint32)
    out = words.view(np.int32)
    return out if np.ndim(bits) == 2 else out[0]
