"""Seeded synthetic inputs shaped like the paper's workloads.

The paper's Year Event Tables and Event Loss Tables are proprietary and not
published (Section III-C says the parameter ranges come from discussions with
practitioners).  This module builds stand-ins with the shapes the paper gives:
trials of 800-1500 events (Section II-A, item 1), ELTs of 10,000-30,000 nonzero
losses (item 2), layers of 3-30 ELTs (item 3), and the 1M-trial x 1000-event,
one-layer workload of the experiments (Section III-C).

It holds no arithmetic of the method: it draws event ids, loss values and term
values, and nothing else.  Both the GPU library's tests and the CPU oracle take
their inputs from here; neither side imports the other.

Every draw comes from a numpy PCG64 stream seeded from (20130809 + workload
index, sub-stream), so a recipe gives the same integers and uniforms on every
machine.  Lognormal draws go through the host libm, so their last bit may
differ between x86 and Arm hosts; a test always computes its expected values on
the machine that drew its inputs.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

SEED_BASE = 20130809


def rng(workload: int, stream: int = 0) -> np.random.Generator:
    """PCG64 generator for one (workload, sub-stream) pair."""
    return np.random.Generator(np.random.PCG64([SEED_BASE + int(workload), int(stream)]))


# ---------------------------------------------------------------------------
# data model (Section II-A)
# ---------------------------------------------------------------------------

@dataclass
class YET:
    """Year Event Table: trials as ordered event-id sequences.

    Either every trial holds exactly ``k`` events (``offsets`` is None) or the
    trials are ragged and ``offsets[i]:offsets[i+1]`` delimits trial i in
    ``ids`` (CSR, int64 offsets).  ``timestamps`` (float32, sorted within each
    trial) may be None; the method only uses the stored order.
    """
    catalog: int
    n_trials: int
    ids: np.ndarray
    k: Optional[int] = None
    offsets: Optional[np.ndarray] = None
    timestamps: Optional[np.ndarray] = None

    @property
    def n_events(self) -> int:
        return int(self.ids.shape[0])

    def bounds(self, i: int) -> tuple[int, int]:
        if self.offsets is None:
            return i * self.k, (i + 1) * self.k
        return int(self.offsets[i]), int(self.offsets[i + 1])

    def trial(self, i: int) -> np.ndarray:
        b, e = self.bounds(i)
        return self.ids[b:e]

    def counts(self) -> np.ndarray:
        if self.offsets is None:
            return np.full(self.n_trials, self.k, dtype=np.int64)
        return np.diff(self.offsets)


@dataclass
class ELT:
    """Event Loss Table: (event id, loss) pairs plus its financial terms.

    ``fx`` (currency rate) and ``share`` default to 1; ``ded``/``lim`` are the
    per-ELT deductible and limit.  Ids are unique and in random order.
    """
    ids: np.ndarray
    losses: np.ndarray
    ded: float = 0.0
    lim: float = float("inf")
    fx: float = 1.0
    share: float = 1.0


@dataclass
class Layer:
    """A layer: indices into an ELT list plus the four layer terms (Table I)."""
    elts: List[int]
    occ_r: float = 0.0
    occ_l: float = float("inf")
    agg_r: float = 0.0
    agg_l: float = float("inf")


@dataclass
class Workload:
    name: str
    yet: YET
    elts: List[ELT]
    layers: List[Layer] = field(default_factory=list)


# ---------------------------------------------------------------------------
# primitive draws
# ---------------------------------------------------------------------------

def _sorted_uniform_timestamps(g: np.random.Generator, counts: np.ndarray) -> np.ndarray:
    n = int(counts.sum())
    ts = g.random(n, dtype=np.float32)
    if n == 0:
        return ts
    kmax = int(counts.max())
    if np.all(counts == kmax):
        return np.sort(ts.reshape(-1, kmax), axis=1).reshape(-1)
    off = np.concatenate([[0], np.cumsum(counts)])
    for i in range(len(counts)):
        ts[off[i]:off[i + 1]].sort()
    return ts


def yet_fixed(g: np.random.Generator, n_trials: int, k: int, catalog: int,
              timestamps: bool = True) -> YET:
    """n_trials trials of exactly k events, ids uniform over [0, catalog)."""
    ids = g.integers(0, catalog, size=n_trials * k, dtype=np.int32)
    ts = None
    if timestamps:
        ts = _sorted_uniform_timestamps(g, np.full(n_trials, k, dtype=np.int64))
    return YET(catalog=catalog, n_trials=n_trials, ids=ids, k=k, timestamps=ts)


def yet_poisson(g: np.random.Generator, n_trials: int, mean: float, catalog: int,
                max_events: Optional[int] = None, timestamps: bool = True) -> YET:
    """Ragged trials with Poisson(mean) events each (optionally truncated)."""
    counts = g.poisson(mean, size=n_trials).astype(np.int64)
    if max_events is not None:
        np.minimum(counts, max_events, out=counts)
    offsets = np.zeros(n_trials + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    ids = g.integers(0, catalog, size=int(offsets[-1]), dtype=np.int32)
    ts = _sorted_uniform_timestamps(g, counts) if timestamps else None
    return YET(catalog=catalog, n_trials=n_trials, ids=ids, offsets=offsets, timestamps=ts)


def elt_ids(g: np.random.Generator, catalog: int, nnz: int) -> np.ndarray:
    """nnz distinct event ids drawn uniformly without replacement."""
    return g.choice(catalog, size=nnz, replace=False).astype(np.int32)


def elt_lognormal(g: np.random.Generator, catalog: int, nnz: int,
                  mu: float = 11.0, sigma: float = 1.5) -> ELT:
    ids = elt_ids(g, catalog, nnz)
    losses = g.lognormal(mu, sigma, size=nnz).astype(np.float64)
    return ELT(ids=ids, losses=losses)


def elt_pareto(g: np.random.Generator, catalog: int, nnz: int, alpha: float = 1.3,
               xmin: float = 1e2, cap: float = 1e9) -> ELT:
    """Pareto(alpha, xmin) by inverse CDF, x = xmin * u**(-1/alpha), capped."""
    ids = elt_ids(g, catalog, nnz)
    u = 1.0 - g.random(nnz)            # (0, 1]
    losses = np.minimum(xmin * u ** (-1.0 / alpha), cap)
    return ELT(ids=ids, losses=losses)


def nearest_rank(values: np.ndarray, permille: int) -> float:
    """Nearest-rank quantile: the ceil(p*n)-th smallest value, p = permille/1000.

    The rank is computed in integers so 10th and 99th percentiles land on the
    same element on every machine.
    """
    v = np.sort(np.asarray(values, dtype=np.float64))
    n = v.shape[0]
    rank = max(1, (permille * n + 999) // 1000)
    return float(v[rank - 1])


def percentile_terms(elt: ELT, ded_permille: int = 100, lim_permille: int = 990) -> ELT:
    """Set an ELT's deductible and limit at percentiles of its own losses."""
    elt.ded = nearest_rank(elt.losses, ded_permille)
    elt.lim = nearest_rank(elt.losses, lim_permille)
    return elt


# ---------------------------------------------------------------------------
# the five workload recipes
# ---------------------------------------------------------------------------

def plain_tiny(n_trials: int = 10_000, k: int = 100, catalog: int = 10_000,
               timestamps: bool = True) -> Workload:
    """10,000 trials x 100 events over a 10,000-event catalog; one layer of 4
    lognormal(11, 1.5) ELTs of 2,000 entries, deductible at p10 and limit at
    p99 of each ELT; occurrence retention 5e4 and limit 2e6; aggregate
    retention 1e5 and limit 1e7."""
    g = rng(0)
    yet = yet_fixed(g, n_trials, k, catalog, timestamps=timestamps)
    elts = [percentile_terms(elt_lognormal(g, catalog, 2000)) for _ in range(4)]
    layer = Layer(elts=[0, 1, 2, 3], occ_r=5e4, occ_l=2e6, agg_r=1e5, agg_l=1e7)
    return Workload("plain_tiny_10k_x_100_j4", yet, elts, [layer])


def paper_scale(n_trials: int = 1_000_000, k: int = 1000, catalog: int = 1_000_000,
                n_elts: int = 16, nnz: int = 20_000, timestamps: bool = False,
                shard: int = 0) -> Workload:
    """1,000,000 trials x 1000 events over a 1,000,000-event catalog; one layer
    of 16 lognormal ELTs of 20,000 entries; per-ELT terms at p10/p99; layer
    terms ten times those of the tiny workload.  Timestamps are off by default
    at this size: the method reads only the stored order.  ``shard`` > 0 draws
    another block of trials of the same recipe (the ELTs stay the same)."""
    g = rng(1) if shard == 0 else rng(1, 1000 + shard)
    yet = yet_fixed(g, n_trials, k, catalog, timestamps=timestamps)
    elts = [percentile_terms(elt_lognormal(rng(1, 1 + j), catalog, nnz)) for j in range(n_elts)]
    layer = Layer(elts=list(range(n_elts)), occ_r=5e5, occ_l=2e7, agg_r=1e6, agg_l=1e8)
    return Workload(f"paper_scale_{n_trials}_x_{k}_j{n_elts}", yet, elts, [layer])


def portfolio(n_trials: int = 200_000, mean_events: float = 1000.0, catalog: int = 1_000_000,
              n_layers: int = 64, pool: int = 256, max_j: int = 32,
              nnz_range: tuple = (5000, 50000), timestamps: bool = False) -> Workload:
    """Shared ragged YET (Poisson(1000) events per trial); 64 layers whose ELT
    counts are uniform on 1..32, drawn from a pool of 256 lognormal ELTs with
    5,000-50,000 entries.  Per-ELT deductible at a U(0,20) percentile and limit
    at a U(95,100) percentile of its losses; layer terms at random percentiles
    of the layer's pooled ELT losses (occurrence retention U(0,50), limit
    U(90,100); aggregate terms the occurrence ones times U(1,10))."""
    g = rng(2)
    yet = yet_poisson(g, n_trials, mean_events, catalog, timestamps=timestamps)
    ge = rng(2, 1)
    elts = []
    for _ in range(pool):
        nnz = int(ge.integers(nnz_range[0], nnz_range[1] + 1))
        e = elt_lognormal(ge, catalog, nnz)
        percentile_terms(e, int(ge.integers(0, 201)), int(ge.integers(950, 1001)))
        elts.append(e)
    gl = rng(2, 2)
    layers = []
    for _ in range(n_layers):
        j = int(gl.integers(1, max_j + 1))
        members = [int(x) for x in gl.choice(pool, size=j, replace=False)]
        pooled = np.concatenate([elts[m].losses for m in members])
        occ_r = nearest_rank(pooled, int(gl.integers(0, 501)))
        occ_l = nearest_rank(pooled, int(gl.integers(900, 1001)))
        layers.append(Layer(elts=members, occ_r=occ_r, occ_l=occ_l,
                            agg_r=occ_r * float(gl.uniform(1, 10)),
                            agg_l=occ_l * float(gl.uniform(1, 10))))
    return Workload(f"portfolio_{n_trials}_poisson{int(mean_events)}_{n_layers}layers",
                    yet, elts, layers)


def precision_stress(n_trials: int = 1_000_000, mean_events: float = 1000.0,
                     max_events: int = 3000, catalog: int = 2_000_000, n_elts: int = 32,
                     nnz: int = 20_000, agg_l: float = float("inf"),
                     timestamps: bool = False) -> Workload:
    """1,000,000 ragged trials (Poisson(1000), at most 3000 events) over a
    2,000,000-event catalog; one layer of 32 Pareto(1.3, 1e2) ELTs capped at
    1e9 with 20,000 entries each; neutral financial and occurrence terms and
    an unbounded aggregate limit, so whole-trial sums reach the YLT."""
    g = rng(3)
    yet = yet_poisson(g, n_trials, mean_events, catalog, max_events=max_events,
                      timestamps=timestamps)
    elts = [elt_pareto(rng(3, 1 + j), catalog, nnz) for j in range(n_elts)]
    layer = Layer(elts=list(range(n_elts)), agg_l=agg_l)
    return Workload(f"precision_stress_{n_trials}_poisson{int(mean_events)}_j{n_elts}",
                    yet, elts, [layer])


def serving_pool(n_trials: int = 1_000_000, k: int = 1000, catalog: int = 1_000_000,
                 pool: int = 256, nnz: int = 20_000, timestamps: bool = False) -> Workload:
    """Resident YET of 1,000,000 x 1000 events and a pool of 256 lognormal
    ELTs of 20,000 entries (terms at p10/p99); requests are drawn separately
    by :func:`pricing_requests`."""
    g = rng(4)
    yet = yet_fixed(g, n_trials, k, catalog, timestamps=timestamps)
    elts = [percentile_terms(elt_lognormal(rng(4, 1 + j), catalog, nnz)) for j in range(pool)]
    return Workload(f"serving_pool_{n_trials}_x_{k}_pool{pool}", yet, elts, [])


@dataclass
class PricingRequest:
    arrival_s: float
    layer: Layer
    n_trials: int
    return_periods: Sequence[float] = (100.0, 250.0)
    tvar_levels: Sequence[float] = (0.99,)


def pricing_requests(n: int, rate_per_s: float, pool: int, max_trials: int,
                     min_trials: int = 10_000, max_j: int = 16, stream: int = 10,
                     pooled_losses: Optional[np.ndarray] = None) -> List[PricingRequest]:
    """Poisson arrivals at ``rate_per_s``; each request a layer of 1..max_j
    distinct pool ELTs with fresh layer terms and a log-uniform trial count in
    [min_trials, max_trials] (it prices the YET's first n_trials trials)."""
    g = rng(4, stream)
    t = 0.0
    out = []
    for _ in range(n):
        t += float(g.exponential(1.0 / rate_per_s))
        j = int(g.integers(1, max_j + 1))
        members = [int(x) for x in g.choice(pool, size=j, replace=False)]
        base = 1e5 if pooled_losses is None else nearest_rank(pooled_losses, 500)
        occ_r = base * float(g.uniform(0.5, 5.0))
        occ_l = occ_r * float(g.uniform(5.0, 50.0))
        agg_r = occ_r * float(g.uniform(1.0, 4.0))
        agg_l = occ_l * float(g.uniform(2.0, 10.0))
        nt = int(round(np.exp(g.uniform(np.log(min_trials), np.log(max_trials)))))
        out.append(PricingRequest(t, Layer(members, occ_r, occ_l, agg_r, agg_l), nt))
    return out


def layer_arrays(elts: Sequence[ELT], layer: Layer):
    """Concatenate a layer's ELTs into flat arrays in layer order:
    (offsets int32[J+1], ids int32[], losses float64[], fx, ded, lim, share)."""
    members = [elts[m] for m in layer.elts]
    off = np.zeros(len(members) + 1, dtype=np.int32)
    off[1:] = np.cumsum([len(e.ids) for e in members])
    ids = (np.concatenate([e.ids for e in members]) if members
           else np.zeros(0, np.int32)).astype(np.int32)
    losses = (np.concatenate([e.losses for e in members]) if members
              else np.zeros(0, np.float64)).astype(np.float64)
    fx = np.array([e.fx for e in members], dtype=np.float64)
    ded = np.array([e.ded for e in members], dtype=np.float64)
    lim = np.array([e.lim for e in members], dtype=np.float64)
    share = np.array([e.share for e in members], dtype=np.float64)
    return off, ids, losses, fx, ded, lim, share
