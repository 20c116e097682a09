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


def mixed_check(got: np.ndarray, ref: np.ndarray, bound: np.ndarray, rtol: float,
                min_plain: float | None = None):
    """Tolerance of the method's arithmetic.  An entry passes if its error is
    within rtol of the reference value (the plain test) or within rtol of
    `bound`, the largest quantity that a cancellation in that entry's
    arithmetic can scale an error by (trial_bound, running_bound): a trial
    loss min(max(S - R, 0), L) near its retention, or an occurrence loss
    whose event loss sits near the occurrence retention, has no plain
    relative error bound for any summation order but the oracle's.

    With `min_plain`, at least that fraction of the entries must also pass
    the plain test (at most floor((1 - min_plain) n) may need the bound), so
    a regression cannot hide behind it.  Returns (ok, stats); the stats
    count the entries that pass only through the bound."""
    d = np.abs(got - ref)
    plain = d <= rtol * np.abs(ref)
    ok = plain | (d <= rtol * bound)
    rel = np.where(ref != 0, d / np.where(ref != 0, np.abs(ref), 1), np.where(d == 0, 0, np.inf))
    n_not_plain = int(ref.size - plain.sum())
    stats = {"n": int(ref.size), "exact": int((d == 0).sum()), "plain_rel_ok": int(plain.sum()),
             "only_through_bound": int((ok & ~plain).sum()), "mixed_ok": int(ok.sum()),
             "max_abs": float(d.max(initial=0)),
             "max_rel_of_bound": float((d / np.maximum(bound, 1e-300)).max(initial=0)),
             "max_rel_finite": float(rel[np.isfinite(rel)].max(initial=0))}
    good = bool(ok.all())
    if min_plain is not None:
        allowed = int(math.floor((1.0 - min_plain) * ref.size + 1e-9))
        stats["plain_required"] = min_plain
        good = good and n_not_plain <= allowed
    print("mixed_check", stats)
    return good, stats


def _bound_terms(wl, layer: int) -> np.ndarray:
    """Per catalog event: its event loss g (after the per-ELT terms, before
    the occurrence terms, host FP64) when g reaches the occurrence retention
    R to within 1e-5, else 0.  Only such an event has a non-zero occurrence
    loss o <= g on any path, and an FP32 rounding of its g carries into o at
    the scale of g, because g - R may cancel."""
    L = wl.layers[layer]
    g = np.zeros(wl.yet.catalog)
    for m in L.elts:
        e = wl.elts[m]
        g[e.ids] += e.share * np.minimum(np.maximum(e.fx * e.losses - e.ded, 0.0), e.lim)
    return np.where(g >= L.occ_r * (1.0 - 1e-5), g, 0.0)


def trial_bound(wl, layer: int, trials=None) -> np.ndarray:
    """Per trial (all, or the selected ones in order): the sum of the event
    losses that reach the occurrence retention (see _bound_terms).  It is at
    least S_k, the running total before the aggregate terms, and at most the
    trial's gross loss; every intermediate whose rounding can reach the trial
    loss is at most this."""
    w = _bound_terms(wl, layer)
    y = wl.yet
    if trials is None:
        tix = np.repeat(np.arange(y.n_trials), y.counts())
        return np.bincount(tix, weights=w[y.ids], minlength=y.n_trials)
    return np.array([w[y.trial(int(t))].sum() for t in trials])


def running_bound(wl, layer: int, trials=None) -> np.ndarray:
    """Per occurrence (the selected trials' events in order): the bound of
    trial_bound taken over the trial's events up to and including this one,
    so a marginal m_d = A_d - A_(d-1) is judged against 2x the running total
    S_d at that occurrence, not the whole trial's."""
    w = _bound_terms(wl, layer)
    y = wl.yet
    trials = range(y.n_trials) if trials is None else trials
    parts = [np.cumsum(w[y.trial(int(t))]) for t in trials]
    return 2.0 * (np.concatenate(parts) if parts else np.zeros(0))


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


def finite_or_none(x):
    return None if (x is None or not math.isfinite(x)) else x
