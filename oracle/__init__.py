"""Python handle on the FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE: only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package.  It shares no code with
the GPU library and never loads it.

``build()`` compiles ``oracle.c`` with gcc into ``liboracle.so`` beside it.
``ARE_ORACLE_LIB`` names another build of the same source to load instead
(the mutation tests point it at copies with planted mistakes).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, -O2, no FP contraction, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp",
                               "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        path = os.environ.get("ARE_ORACLE_LIB")
        if not path:
            path = build()
        lib = C.CDLL(path)
        P = C.c_void_p
        lib.or_simulate.restype = C.c_int
        lib.or_simulate.argtypes = [
            C.c_int64, P, C.c_int32, P, C.c_int32, P, P, P, P, P, P, P,
            C.c_double, C.c_double, C.c_double, C.c_double,
            C.c_int64, P, P, P, P, P, P, P, P, P, C.c_int32]
        lib.or_risk_measures.restype = C.c_int
        lib.or_risk_measures.argtypes = [P, C.c_int64, P, C.c_int32, P, P, C.c_int32, P]
        lib.or_rank_for_return_period.restype = C.c_int64
        lib.or_rank_for_return_period.argtypes = [C.c_int64, C.c_double]
        lib.or_rank_for_level.restype = C.c_int64
        lib.or_rank_for_level.argtypes = [C.c_int64, C.c_double]
        lib.or_max_threads.restype = C.c_int
        _lib = lib
    return _lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


@dataclass
class TrialResult:
    ylt: np.ndarray        # A_k per trial (the YLT)
    s_total: np.ndarray    # S_k, cumulative occurrence loss
    gross: np.ndarray      # sum of fx * x over the trial's events and ELTs
    lr_literal: np.ndarray # literal sum of the marginals
    occ_max: np.ndarray    # largest occurrence loss after occurrence terms
    n_events: np.ndarray   # events per trial
    marginals: Optional[np.ndarray] = None


def simulate(yet_ids: np.ndarray, n_trials: int, offsets: Optional[np.ndarray], k: Optional[int],
             elt_off: np.ndarray, elt_ids: np.ndarray, elt_loss: np.ndarray,
             fx: np.ndarray, ded: np.ndarray, lim: np.ndarray, share: np.ndarray,
             occ_r: float, occ_l: float, agg_r: float, agg_l: float,
             trials: Optional[np.ndarray] = None, marginals: bool = False,
             threads: int = 0) -> TrialResult:
    """Run the oracle for one layer over the selected trials (all if None)."""
    lib = _load()
    ids = np.ascontiguousarray(yet_ids, dtype=np.int32)
    off = None if offsets is None else np.ascontiguousarray(offsets, dtype=np.int64)
    sel = None if trials is None else np.ascontiguousarray(trials, dtype=np.int64)
    n_sel = n_trials if sel is None else sel.shape[0]
    eo = np.ascontiguousarray(elt_off, dtype=np.int32)
    ei = np.ascontiguousarray(elt_ids, dtype=np.int32)
    el = np.ascontiguousarray(elt_loss, dtype=np.float64)
    t = [np.ascontiguousarray(a, dtype=np.float64) for a in (fx, ded, lim, share)]
    out = [np.empty(n_sel, np.float64) for _ in range(5)]
    nev = np.empty(n_sel, np.int64)
    marg = moff = None
    if marginals:
        if off is None:
            counts = np.full(n_sel, k, dtype=np.int64)
        else:
            tt = np.arange(n_trials) if sel is None else sel
            counts = off[tt + 1] - off[tt]
        moff = np.zeros(n_sel + 1, dtype=np.int64)
        np.cumsum(counts, out=moff[1:])
        marg = np.empty(int(moff[-1]), np.float64)
    rc = lib.or_simulate(n_trials, _ptr(off), 0 if k is None else int(k), _ptr(ids),
                         len(eo) - 1, _ptr(eo), _ptr(ei), _ptr(el), *(_ptr(a) for a in t),
                         float(occ_r), float(occ_l), float(agg_r), float(agg_l),
                         n_sel, _ptr(sel), *(_ptr(a) for a in out), _ptr(nev),
                         _ptr(marg), _ptr(moff), int(threads))
    if rc != 0:
        raise ValueError(f"oracle or_simulate failed with code {rc}")
    return TrialResult(*out, nev, marg)


def simulate_layer(workload, layer_index: int = 0, trials=None, marginals=False, threads=0):
    """Convenience wrapper over a ``workloads.Workload``."""
    from workloads import layer_arrays
    y = workload.yet
    L = workload.layers[layer_index]
    eo, ei, el, fx, ded, lim, share = layer_arrays(workload.elts, L)
    return simulate(y.ids, y.n_trials, y.offsets, y.k, eo, ei, el, fx, ded, lim, share,
                    L.occ_r, L.occ_l, L.agg_r, L.agg_l, trials=trials,
                    marginals=marginals, threads=threads)


def risk_measures(ylt: np.ndarray, return_periods: Sequence[float] = (100.0, 250.0),
                  levels: Sequence[float] = (0.99,)):
    """(PML per return period, TVaR per level) from a full sort of the YLT."""
    lib = _load()
    y = np.ascontiguousarray(ylt, dtype=np.float64)
    rp = np.ascontiguousarray(return_periods, dtype=np.float64)
    lv = np.ascontiguousarray(levels, dtype=np.float64)
    pml = np.empty(rp.shape[0], np.float64)
    tv = np.empty(lv.shape[0], np.float64)
    rc = lib.or_risk_measures(_ptr(y), y.shape[0], _ptr(rp), rp.shape[0], _ptr(pml),
                              _ptr(lv), lv.shape[0], _ptr(tv))
    if rc != 0:
        raise ValueError(f"oracle or_risk_measures failed with code {rc}")
    return pml, tv


def rank_for_return_period(n: int, rp: float) -> int:
    return int(_load().or_rank_for_return_period(int(n), float(rp)))


def rank_for_level(n: int, a: float) -> int:
    return int(_load().or_rank_for_level(int(n), float(a)))


def max_threads() -> int:
    return int(_load().or_max_threads())
