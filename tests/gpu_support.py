"""Shared helpers for the GPU parity tests: load a workload through the C ABI
and compare GPU results with the oracle's."""
from __future__ import annotations

import math

import numpy as np

import workloads as W

# by precision: FP64, FP32+Kahan, FP32+FP64 sum; "folded": the FP64 folded table
RTOL = {0: 1e-12, 1: 1e-5, 2: 1e-5, "folded": 1e-12}


class Loaded:
    """A workload's YET, ELTs and layers loaded into one context."""

    def __init__(self, are, ctx, wl: W.Workload, device_inputs: bool = True,
                 timestamps: bool = True):
        import torch
        self.are, self.ctx, self.wl = are, ctx, wl
        y = wl.yet
        if device_inputs:
            ids = torch.from_numpy(y.ids).cuda()
            off = None if y.offsets is None else torch.from_numpy(y.offsets).cuda()
            ts = (torch.from_numpy(y.timestamps).cuda()
                  if (timestamps and y.timestamps is not None) else None)
        else:
            ids, off = y.ids, y.offsets
            ts = y.timestamps if timestamps else None
        self.yet = are.are_load_yet(ctx, y.catalog, y.n_trials, off, y.k or 0, ids, ts)
        del ids, off, ts
        self.elts = [are.are_load_elt(ctx, e.ids, e.losses, e.fx, e.ded, e.lim, e.share)
                     for e in wl.elts]
        self.layers = [self.define(L) for L in wl.layers]

    def define(self, L: W.Layer) -> int:
        return self.are.are_define_layer(self.ctx, [self.elts[m] for m in L.elts],
                                         L.occ_r, L.occ_l, L.agg_r, L.agg_l)

    def simulate(self, layer: int, precision: int, begin: int = 0, n: int | None = None,
                 device: bool = True, handle: int | None = None) -> np.ndarray:
        import torch
        y = self.wl.yet
        n = y.n_trials - begin if n is None else n
        h = self.layers[layer] if handle is None else handle
        if device:
            out = torch.full((n,), -1.0, dtype=torch.float64, device="cuda")
            self.are.are_simulate(self.ctx, h, self.yet, begin, n, precision, out)
            return out.cpu().numpy()
        out = np.full(n, -1.0)
        self.are.are_simulate(self.ctx, h, self.yet, begin, n, precision, out)
        return out

    def folded(self, layer: int, begin: int = 0, n: int | None = None,
               device: bool = True) -> np.ndarray:
        import torch
        y = self.wl.yet
        n = y.n_trials - begin if n is None else n
        if device:
            out = torch.full((n,), -1.0, dtype=torch.float64, device="cuda")
            self.are.are_simulate_folded(self.ctx, self.layers[layer], self.yet, begin, n, out)
            return out.cpu().numpy()
        out = np.full(n, -1.0)
        self.are.are_simulate_folded(self.ctx, self.layers[layer], self.yet, begin, n, out)
        return out

    def run(self, layer: int, precision, begin: int = 0, n: int | None = None) -> np.ndarray:
        """are_simulate in a precision, or the folded table for "folded"."""
        if precision == "folded":
            return self.folded(layer, begin, n)
        return self.simulate(layer, precision, begin, n)

    def release(self):
        for h in self.layers:
            self.are.are_free_layer(self.ctx, h)
        for h in self.elts:
            self.are.are_free_elt(self.ctx, h)
        self.are.are_free_yet(self.ctx, self.yet)


def mixed_check(got: np.ndarray, ref: np.ndarray, gross: np.ndarray, rtol: float):
    """Tolerance of the method's arithmetic: a YLT entry passes if its error is
    within rtol of the reference value or within rtol of the trial's gross
    loss (which bounds every intermediate of the trial, so a cancellation
    near a retention cannot fail it).  Returns (all ok, stats)."""
    d = np.abs(got - ref)
    plain = d <= rtol * np.abs(ref)
    ok = plain | (d <= rtol * gross)
    rel = np.where(ref != 0, d / np.where(ref != 0, np.abs(ref), 1), np.where(d == 0, 0, np.inf))
    stats = {"n": int(ref.size), "exact": int((d == 0).sum()), "plain_rel_ok": int(plain.sum()),
             "mixed_ok": int(ok.sum()), "max_abs": float(d.max(initial=0)),
             "max_rel_of_gross": float((d / np.maximum(gross, 1e-300)).max(initial=0)),
             "max_rel_finite": float(rel[np.isfinite(rel)].max(initial=0))}
    return bool(ok.all()), stats


def rel_close(a, b, rtol):
    return all(abs(x - y) <= rtol * max(abs(y), 1e-300) for x, y in zip(a, b))


def tail_candidates(gpu_ylt: np.ndarray, m_max: int, margin: int):
    """Indices of the m_max + margin largest GPU trial losses, descending."""
    k = min(gpu_ylt.size, m_max + margin)
    idx = np.argpartition(-gpu_ylt, k - 1)[:k]
    return idx[np.argsort(-gpu_ylt[idx], kind="stable")]


def ranks(n, rps, levels, orc):
    return ([orc.rank_for_return_period(n, r) for r in rps],
            [orc.rank_for_level(n, a) for a in levels])


def gross_bound(wl, layer, trials):
    """Sum over the trials' events of every ELT's converted loss (host numpy)."""
    members = [wl.elts[m] for m in wl.layers[layer].elts]
    dense = np.zeros(wl.yet.catalog)
    for e in members:
        dense[e.ids] += e.fx * e.losses
    return np.array([dense[wl.yet.trial(int(t))].sum() for t in trials])


def finite_or_none(x):
    return None if (x is None or not math.isfinite(x)) else x
