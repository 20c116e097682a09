"""Python binding of libare, the GB300 aggregate-risk-analysis engine.

Argument marshalling only: every function here forwards to the C ABI entry
point of the same name in ``libare.so`` (declared in ``include/are.h``); all
computation happens in the library's CUDA kernels.  Arrays may be numpy
arrays (host memory), torch tensors (host or device) or raw integer
addresses.  A failed call raises :class:`AreError` with the library's status
and message.  If ``libare.so`` has not been built the import of any function
fails loudly: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import math
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libare.so")

ARE_OK, ARE_EINVAL, ARE_ENOMEM, ARE_ECUDA, ARE_ETIMEOUT, ARE_EBUSY, ARE_ENOTFOUND = range(7)
ARE_FP64, ARE_FP32_KAHAN, ARE_FP32_FP64AGG = 0, 1, 2
ARE_MAX_ELTS_PER_LAYER = 32
ARE_LAYOUT_DIRECT, ARE_LAYOUT_COMPACT = 0, 1
STATUS_NAMES = {0: "ARE_OK", 1: "ARE_EINVAL", 2: "ARE_ENOMEM", 3: "ARE_ECUDA",
                4: "ARE_ETIMEOUT", 5: "ARE_EBUSY", 6: "ARE_ENOTFOUND"}
PRECISIONS = {"fp64": ARE_FP64, "fp32_kahan": ARE_FP32_KAHAN, "fp32_fp64agg": ARE_FP32_FP64AGG}


class AreError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status
        self.message = message


class FinTerms(C.Structure):
    _fields_ = [("fx", C.c_double), ("deductible", C.c_double), ("limit", C.c_double),
                ("share", C.c_double)]


class TuneResult(C.Structure):
    _fields_ = [("kernel", C.c_int32), ("rows_in_flight", C.c_int32),
                ("trials_per_item", C.c_int32), ("blocks_per_sm", C.c_int32), ("ms", C.c_double)]


class CeilingShape(C.Structure):
    _fields_ = [("kind", C.c_int32), ("rows_in_flight", C.c_int32), ("blocks_per_sm", C.c_int32),
                ("rows_per_s", C.c_double)]


class LayerTerms(C.Structure):
    _fields_ = [("occ_ret", C.c_double), ("occ_lim", C.c_double), ("agg_ret", C.c_double),
                ("agg_lim", C.c_double)]


class ServerCfg(C.Structure):
    _fields_ = [("max_inflight", C.c_int32), ("max_pending", C.c_int32),
                ("arena_bytes", C.c_size_t), ("events_per_launch", C.c_int64),
                ("trials_per_item", C.c_int32), ("one_at_a_time", C.c_int32),
                ("precision", C.c_int), ("stall_us", C.c_int64), ("folded", C.c_int32),
                ("least_work_first", C.c_int32)]


class Request(C.Structure):
    _fields_ = [("elt_handles", C.c_void_p), ("n_elts", C.c_int32), ("terms", LayerTerms),
                ("n_trials", C.c_int64), ("return_periods", C.c_void_p), ("n_rp", C.c_int32),
                ("tvar_levels", C.c_void_p), ("n_tv", C.c_int32)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int32), ("n_rp", C.c_int32), ("n_tv", C.c_int32),
                ("pml", C.c_double * 8), ("tvar", C.c_double * 8), ("n_trials", C.c_int64),
                ("queue_us", C.c_double), ("run_us", C.c_double), ("total_us", C.c_double)]


_lib = None
_P = C.c_void_p
_SIGS = {
    "are_create": (C.c_int32, [C.POINTER(C.c_void_p), C.c_int, C.c_size_t]),
    "are_destroy": (C.c_int32, [_P]),
    "are_last_error": (C.c_char_p, [_P]),
    "are_memory_used": (C.c_int32, [_P, C.POINTER(C.c_size_t)]),
    "are_launch_count": (C.c_int32, [_P, C.POINTER(C.c_uint64)]),
    "are_load_yet": (C.c_int32, [_P, C.c_int32, C.c_int64, _P, C.c_int32, _P, _P,
                                 C.POINTER(C.c_int32)]),
    "are_load_elt": (C.c_int32, [_P, C.c_int32, _P, _P, C.POINTER(FinTerms),
                                 C.POINTER(C.c_int32)]),
    "are_define_layer": (C.c_int32, [_P, _P, C.c_int32, C.POINTER(LayerTerms),
                                     C.POINTER(C.c_int32)]),
    "are_free_yet": (C.c_int32, [_P, C.c_int32]),
    "are_free_elt": (C.c_int32, [_P, C.c_int32]),
    "are_free_layer": (C.c_int32, [_P, C.c_int32]),
    "are_prepare": (C.c_int32, [_P, C.c_int32, C.c_int32, C.c_int, _P]),
    "are_simulate": (C.c_int32, [_P, C.c_int32, C.c_int32, C.c_int64, C.c_int64, C.c_int, _P,
                                 _P]),
    "are_risk_measures": (C.c_int32, [_P, _P, C.c_int64, _P, C.c_int32, _P, _P, C.c_int32, _P,
                                      _P]),
    "are_risk_measures_static": (C.c_int32, [_P, C.c_int64, _P, C.c_int32, _P, _P, C.c_int32,
                                             _P, _P]),
    "are_simulate_portfolio": (C.c_int32, [_P, _P, C.c_int32, C.c_int32, C.c_int64, C.c_int64,
                                           C.c_int, _P, _P]),
    "are_risk_measures_batch": (C.c_int32, [_P, _P, C.c_int32, C.c_int64, _P, C.c_int32, _P, _P,
                                            C.c_int32, _P, _P]),
    "are_autotune": (C.c_int32, [_P, _P, C.c_int32, C.c_int32, C.c_int, _P,
                                 C.POINTER(TuneResult)]),
    "are_tune_save": (C.c_int32, [_P, C.c_char_p]),
    "are_tune_load": (C.c_int32, [_P, C.c_char_p]),
    "are_simulate_occurrences": (C.c_int32, [_P, C.c_int32, C.c_int32, C.c_int64, C.c_int64,
                                             C.c_int, _P, _P, _P, _P]),
    "are_set_table_layout": (C.c_int32, [_P, C.c_int32, C.c_int32]),
    "are_layer_rows": (C.c_int32, [_P, C.c_int32, C.c_int32, C.c_int, C.c_int32,
                                   C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "are_prepare_folded": (C.c_int32, [_P, C.c_int32, C.c_int32, _P]),
    "are_simulate_folded": (C.c_int32, [_P, C.c_int32, C.c_int32, C.c_int64, C.c_int64, _P, _P]),
    "are_simulate_streamed": (C.c_int32, [_P, C.c_int32, C.c_int32, C.c_int64, _P, C.c_int32, _P,
                                          C.c_int64, C.c_int, _P, _P]),
    "are_simulate_streamed_packed": (C.c_int32, [_P, C.c_int32, C.c_int32, C.c_int64, _P, C.c_int32, _P,
                                                 C.c_int32, C.c_int64, C.c_int, _P, _P]),
    "are_pack_ids": (C.c_int32, [_P, _P, C.c_int64, C.c_int32, _P]),
    "are_gather_ceiling": (C.c_int32, [_P, C.c_int32, C.c_int32, C.c_int64, C.c_int64,
                                       C.c_int32, C.POINTER(C.c_double),
                                       C.POINTER(CeilingShape), C.c_int32,
                                       C.POINTER(C.c_int32)]),
    "are_server_start": (C.c_int32, [_P, C.c_int32, C.POINTER(ServerCfg)]),
    "are_submit": (C.c_int32, [_P, C.POINTER(Request), C.POINTER(C.c_int64)]),
    "are_wait": (C.c_int32, [_P, C.c_int64, C.c_int64, C.POINTER(Result)]),
    "are_cancel": (C.c_int32, [_P, C.c_int64]),
    "are_server_stop": (C.c_int32, [_P]),
}


def lib():
    """The loaded libare.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(ctx, status: int):
    if status != ARE_OK:
        msg = lib().are_last_error(ctx)
        raise AreError(status, (msg or b"").decode(errors="replace"))


def _addr(x, dtype=None):
    """Address of an array argument: None, int, numpy array or torch tensor."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be contiguous")
        if dtype is not None and x.dtype != np.dtype(dtype):
            raise TypeError(f"expected {np.dtype(dtype)}, got {x.dtype}")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if dtype is not None and str(x.dtype).replace("torch.", "") != np.dtype(dtype).name:
            raise TypeError(f"expected {np.dtype(dtype)}, got {x.dtype}")
        return x.data_ptr()
    raise TypeError(f"unsupported array argument {type(x)}")


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return int(s.cuda_stream)


def _len(x) -> int:
    return int(x.shape[0]) if x is not None else 0


# ---------------------------------------------------------------------------
# context
# ---------------------------------------------------------------------------

def are_create(device: int = 0, mem_budget_bytes: int = 0):
    out = C.c_void_p()
    _check(None, lib().are_create(C.byref(out), int(device), int(mem_budget_bytes)))
    return out


def are_destroy(ctx) -> None:
    _check(None, lib().are_destroy(ctx))


def are_last_error(ctx) -> str:
    return (lib().are_last_error(ctx) or b"").decode(errors="replace")


def are_memory_used(ctx) -> int:
    n = C.c_size_t()
    _check(ctx, lib().are_memory_used(ctx, C.byref(n)))
    return int(n.value)


def are_launch_count(ctx) -> int:
    n = C.c_uint64()
    _check(ctx, lib().are_launch_count(ctx, C.byref(n)))
    return int(n.value)


# ---------------------------------------------------------------------------
# inputs
# ---------------------------------------------------------------------------

def are_load_yet(ctx, catalog_size: int, n_trials: int, offsets, events_per_trial: int,
                 event_ids, timestamps=None) -> int:
    h = C.c_int32()
    _check(ctx, lib().are_load_yet(ctx, int(catalog_size), int(n_trials),
                                   _addr(offsets, np.int64), int(events_per_trial or 0),
                                   _addr(event_ids, np.int32), _addr(timestamps, np.float32),
                                   C.byref(h)))
    return h.value


def are_load_elt(ctx, event_ids, losses, fx: float = 1.0, deductible: float = 0.0,
                 limit: float = math.inf, share: float = 1.0) -> int:
    n = _len(event_ids)
    if _len(losses) != n:
        raise ValueError("event_ids and losses differ in length")
    t = FinTerms(fx, deductible, limit, share)
    h = C.c_int32()
    _check(ctx, lib().are_load_elt(ctx, n, _addr(event_ids, np.int32), _addr(losses, np.float64),
                                   C.byref(t), C.byref(h)))
    return h.value


def are_define_layer(ctx, elt_handles: Sequence[int], occ_ret: float = 0.0,
                     occ_lim: float = math.inf, agg_ret: float = 0.0,
                     agg_lim: float = math.inf) -> int:
    hs = np.ascontiguousarray(elt_handles, dtype=np.int32)
    t = LayerTerms(occ_ret, occ_lim, agg_ret, agg_lim)
    h = C.c_int32()
    _check(ctx, lib().are_define_layer(ctx, hs.ctypes.data, hs.shape[0], C.byref(t), C.byref(h)))
    return h.value


def are_free_yet(ctx, h: int) -> None:
    _check(ctx, lib().are_free_yet(ctx, int(h)))


def are_free_elt(ctx, h: int) -> None:
    _check(ctx, lib().are_free_elt(ctx, int(h)))


def are_free_layer(ctx, h: int) -> None:
    _check(ctx, lib().are_free_layer(ctx, int(h)))


# ---------------------------------------------------------------------------
# analysis stage and filters
# ---------------------------------------------------------------------------

def are_prepare(ctx, layer: int, yet: int, precision: int = ARE_FP64, stream=None) -> None:
    _check(ctx, lib().are_prepare(ctx, int(layer), int(yet), int(precision), _stream(stream)))


def are_simulate(ctx, layer: int, yet: int, trial_begin: int, n_trials: int,
                 precision: int, ylt, stream=None) -> None:
    _check(ctx, lib().are_simulate(ctx, int(layer), int(yet), int(trial_begin), int(n_trials),
                                   int(precision), _addr(ylt, np.float64), _stream(stream)))


def are_simulate_occurrences(ctx, layer: int, yet: int, trial_begin: int, n_trials: int,
                             precision: int, marginals, occ_max=None, ylt=None,
                             stream=None) -> None:
    """Per-occurrence marginals, per-trial occurrence maxima and the YLT."""
    _check(ctx, lib().are_simulate_occurrences(ctx, int(layer), int(yet), int(trial_begin),
                                               int(n_trials), int(precision),
                                               _addr(marginals, np.float64),
                                               _addr(occ_max, np.float64),
                                               _addr(ylt, np.float64), _stream(stream)))


def are_set_table_layout(ctx, layer: int, layout: int) -> None:
    """ARE_LAYOUT_DIRECT (one row per catalog event) or ARE_LAYOUT_COMPACT."""
    _check(ctx, lib().are_set_table_layout(ctx, int(layer), int(layout)))


def are_layer_rows(ctx, layer: int, yet: int, precision: int, kernel: int = -1):
    """(row_bytes, packed): the table row an analysis of the layer over the
    YET reads per occurrence, under a kernel choice (-1: the current one)."""
    rb, pk = C.c_int32(0), C.c_int32(0)
    _check(ctx, lib().are_layer_rows(ctx, int(layer), int(yet), int(precision), int(kernel),
                                     C.byref(rb), C.byref(pk)))
    return rb.value, bool(pk.value)


def are_prepare_folded(ctx, layer: int, yet: int, stream=None) -> None:
    """Build the layer's folded table (FP64 occurrence loss per catalog event)."""
    _check(ctx, lib().are_prepare_folded(ctx, int(layer), int(yet), _stream(stream)))


def are_simulate_folded(ctx, layer: int, yet: int, trial_begin: int, n_trials: int, ylt,
                        stream=None) -> None:
    """YLT from the folded table: one lookup per occurrence, exact trial sums."""
    _check(ctx, lib().are_simulate_folded(ctx, int(layer), int(yet), int(trial_begin),
                                          int(n_trials), _addr(ylt, np.float64),
                                          _stream(stream)))


def are_simulate_streamed(ctx, layer: int, catalog_size: int, n_trials: int, offsets,
                          events_per_trial: int, event_ids, precision: int, ylt,
                          chunk_events: int = 0, stream=None) -> None:
    """Analysis over a host-resident YET, its copy to the device overlapped
    with the analysis chunk by chunk."""
    _check(ctx, lib().are_simulate_streamed(ctx, int(layer), int(catalog_size), int(n_trials),
                                            _addr(offsets, np.int64), int(events_per_trial),
                                            _addr(event_ids, np.int32), int(chunk_events),
                                            int(precision), _addr(ylt, np.float64),
                                            _stream(stream)))


def are_simulate_streamed_packed(ctx, layer: int, catalog_size: int, n_trials: int, offsets,
                                 events_per_trial: int, packed_ids, id_bits: int, precision: int, ylt,
                                 chunk_events: int = 0, stream=None) -> None:
    """are_simulate_streamed over ids packed id_bits bits each (see
    are_pack_ids)."""
    _check(ctx, lib().are_simulate_streamed_packed(ctx, int(layer), int(catalog_size), int(n_trials),
                                                   _addr(offsets, np.int64), int(events_per_trial),
                                                   _addr(packed_ids, np.uint32), int(id_bits),
                                                   int(chunk_events), int(precision),
                                                   _addr(ylt, np.float64), _stream(stream)))


def packed_words(n: int, id_bits: int) -> int:
    """32-bit words that n ids of id_bits bits take."""
    return (int(n) * int(id_bits) + 31) // 32


def are_pack_ids(ctx, ids, id_bits: int, out=None):
    """Packs host int32 ids id_bits bits each into uint32 words (a new numpy
    array, or `out`: a host numpy array or pinned tensor of packed_words
    words); returns the words."""
    n = _len(ids)
    if out is None:
        out = np.empty(packed_words(n, id_bits), np.uint32)
    _check(ctx, lib().are_pack_ids(ctx, _addr(ids, np.int32), n, int(id_bits), _addr(out, np.uint32)))
    return out


def are_gather_ceiling(ctx, yet: int, row_bytes: int, trial_begin: int = 0,
                       n_trials: Optional[int] = None, reps: int = 3, shapes: bool = False):
    """Rows per second of a pure id-stream + table-row gather over the YET,
    best over every launch shape; with shapes=True also the list of
    (kind, rows_in_flight, blocks_per_sm, rows_per_s) of each shape timed."""
    if n_trials is None:
        raise ValueError("n_trials is required")
    out = C.c_double()
    buf = (CeilingShape * 64)()
    n = C.c_int32(0)
    _check(ctx, lib().are_gather_ceiling(ctx, int(yet), int(row_bytes), int(trial_begin),
                                         int(n_trials), int(reps), C.byref(out), buf, 64,
                                         C.byref(n)))
    if not shapes:
        return out.value
    got = [(b.kind, b.rows_in_flight, b.blocks_per_sm, b.rows_per_s) for b in buf[: min(n.value, 64)]]
    return out.value, got


def are_risk_measures(ctx, ylt, n: Optional[int] = None,
                      return_periods: Sequence[float] = (100.0, 250.0),
                      tvar_levels: Sequence[float] = (0.99,), stream=None, out=None):
    """Returns (pml, tvar) as numpy float64 arrays; with out=(pml, tvar)
    (device float64 arrays, a device YLT) the call only enqueues the
    selection into them and returns None."""
    n = _len(ylt) if n is None else int(n)
    rp = np.ascontiguousarray(return_periods, dtype=np.float64)
    lv = np.ascontiguousarray(tvar_levels, dtype=np.float64)
    if out is not None:
        pml, tv = out
        _check(ctx, lib().are_risk_measures(ctx, _addr(ylt, np.float64), n, rp.ctypes.data,
                                            rp.shape[0], _addr(pml, np.float64), lv.ctypes.data,
                                            lv.shape[0], _addr(tv, np.float64), _stream(stream)))
        return None
    pml = np.empty(rp.shape[0], np.float64)
    tv = np.empty(lv.shape[0], np.float64)
    _check(ctx, lib().are_risk_measures(ctx, _addr(ylt, np.float64), n, rp.ctypes.data,
                                        rp.shape[0], pml.ctypes.data, lv.ctypes.data, lv.shape[0],
                                        tv.ctypes.data, _stream(stream)))
    return pml, tv


def are_risk_measures_static(ylt, n: Optional[int] = None,
                             return_periods: Sequence[float] = (100.0, 250.0),
                             tvar_levels: Sequence[float] = (0.99,), stream=None):
    """Context-free, allocation-free PML/TVaR of a device YLT (see are.h)."""
    n = _len(ylt) if n is None else int(n)
    rp = np.ascontiguousarray(return_periods, dtype=np.float64)
    lv = np.ascontiguousarray(tvar_levels, dtype=np.float64)
    pml = np.empty(rp.shape[0], np.float64)
    tv = np.empty(lv.shape[0], np.float64)
    _check(None, lib().are_risk_measures_static(_addr(ylt, np.float64), n, rp.ctypes.data,
                                                rp.shape[0], pml.ctypes.data, lv.ctypes.data,
                                                lv.shape[0], tv.ctypes.data, _stream(stream)))
    return pml, tv


def are_simulate_portfolio(ctx, layers: Sequence[int], yet: int, trial_begin: int, n_trials: int,
                           precision: int, ylts: Sequence, stream=None) -> None:
    """Analysis stage for several layers in one persistent, graph-replayed launch."""
    hs = np.ascontiguousarray(layers, dtype=np.int32)
    ptrs = (C.c_void_p * len(ylts))(*[_addr(y, np.float64) for y in ylts])
    if len(ylts) != hs.shape[0]:
        raise ValueError("one YLT per layer")
    _check(ctx, lib().are_simulate_portfolio(ctx, hs.ctypes.data, hs.shape[0], int(yet),
                                             int(trial_begin), int(n_trials), int(precision),
                                             C.cast(ptrs, C.c_void_p), _stream(stream)))


def are_risk_measures_batch(ctx, ylts: Sequence, n: int,
                            return_periods: Sequence[float] = (100.0, 250.0),
                            tvar_levels: Sequence[float] = (0.99,), stream=None):
    """(pml[n_ylt, n_rp], tvar[n_ylt, n_tv]) for several device YLTs."""
    ptrs = (C.c_void_p * len(ylts))(*[_addr(y, np.float64) for y in ylts])
    rp = np.ascontiguousarray(return_periods, dtype=np.float64)
    lv = np.ascontiguousarray(tvar_levels, dtype=np.float64)
    pml = np.empty((len(ylts), rp.shape[0]), np.float64)
    tv = np.empty((len(ylts), lv.shape[0]), np.float64)
    _check(ctx, lib().are_risk_measures_batch(ctx, C.cast(ptrs, C.c_void_p), len(ylts), int(n),
                                              rp.ctypes.data, rp.shape[0], pml.ctypes.data,
                                              lv.ctypes.data, lv.shape[0], tv.ctypes.data,
                                              _stream(stream)))
    return pml, tv


def are_autotune(ctx, layers: Sequence[int], yet: int, precision: int, stream=None) -> dict:
    """Time the candidate launch configurations and keep the fastest."""
    hs = np.ascontiguousarray(layers, dtype=np.int32)
    r = TuneResult()
    _check(ctx, lib().are_autotune(ctx, hs.ctypes.data, hs.shape[0], int(yet), int(precision),
                                   _stream(stream), C.byref(r)))
    return {f: getattr(r, f) for f, _ in TuneResult._fields_}


def are_tune_save(ctx, path: str) -> None:
    _check(ctx, lib().are_tune_save(ctx, os.fsencode(path)))


def are_tune_load(ctx, path: str) -> None:
    _check(ctx, lib().are_tune_load(ctx, os.fsencode(path)))


# ---------------------------------------------------------------------------
# pricing server
# ---------------------------------------------------------------------------

def are_server_start(ctx, yet: int, max_inflight: int = 32, max_pending: int = 4096,
                     arena_bytes: int = 4 << 30, events_per_launch: int = 0,
                     trials_per_item: int = 0, one_at_a_time: bool = False,
                     precision: int = ARE_FP32_KAHAN, stall_us: int = 0,
                     folded: bool = False, least_work_first: bool = False) -> None:
    cfg = ServerCfg(max_inflight, max_pending, arena_bytes, events_per_launch, trials_per_item,
                    int(bool(one_at_a_time)), precision, stall_us, int(bool(folded)),
                    int(bool(least_work_first)))
    _check(ctx, lib().are_server_start(ctx, int(yet), C.byref(cfg)))


def are_submit(ctx, elt_handles: Sequence[int], occ_ret: float, occ_lim: float, agg_ret: float,
               agg_lim: float, n_trials: int, return_periods: Sequence[float] = (100.0, 250.0),
               tvar_levels: Sequence[float] = (0.99,)) -> int:
    hs = np.ascontiguousarray(elt_handles, dtype=np.int32)
    rp = np.ascontiguousarray(return_periods, dtype=np.float64)
    lv = np.ascontiguousarray(tvar_levels, dtype=np.float64)
    req = Request(hs.ctypes.data, hs.shape[0], LayerTerms(occ_ret, occ_lim, agg_ret, agg_lim),
                  int(n_trials), rp.ctypes.data, rp.shape[0], lv.ctypes.data, lv.shape[0])
    t = C.c_int64()
    _check(ctx, lib().are_submit(ctx, C.byref(req), C.byref(t)))
    return t.value


def are_wait(ctx, ticket: int, timeout_us: int = -1) -> dict:
    """The request's result: status, pml, tvar, n_trials and its timings (us)."""
    r = Result()
    _check(ctx, lib().are_wait(ctx, int(ticket), int(timeout_us), C.byref(r)))
    return {"status": r.status, "pml": list(r.pml[: r.n_rp]), "tvar": list(r.tvar[: r.n_tv]),
            "n_trials": r.n_trials, "queue_us": r.queue_us, "run_us": r.run_us,
            "total_us": r.total_us}


def are_cancel(ctx, ticket: int) -> None:
    _check(ctx, lib().are_cancel(ctx, int(ticket)))


def are_server_stop(ctx) -> None:
    _check(ctx, lib().are_server_stop(ctx))
