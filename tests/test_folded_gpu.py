"""The folded layer table (are_prepare_folded / are_simulate_folded) against
the oracle.

The folded table holds one FP64 occurrence loss h[e] per catalog event and
the trial pass sums them exactly.  So, beside the usual tolerance against
the oracle's sequential sums, its results are pinned exactly:

* h[e] is the oracle's occurrence loss of event e bit for bit (a one-event
  trial per catalog event gives it as that trial's loss);
* a trial's loss is min(max(S - AggR, 0), AggL) with S the correctly rounded
  exact sum of the trial's h[e_d], each first rounded to a multiple of
  2^-s with s = 125 - floor(log2(max h)) (a no-op for every h of 2^-52 of
  the largest or more), computed here with Python fractions;
* it does not depend on the order of a trial's events or on how the trials
  are split into calls."""
import json
import math
from fractions import Fraction

import numpy as np
import pytest

import workloads as W
from gpu_support import Loaded, RTOL, mixed_check, trial_bound

pytestmark = pytest.mark.gpu
INF = math.inf


@pytest.fixture(scope="module")
def are():
    import torch
    assert torch.cuda.is_available()
    import paper_1308_2066_gb300 as are
    are.lib()
    return are


@pytest.fixture(scope="module")
def ctx(are):
    c = are.are_create(0)
    yield c
    are.are_destroy(c)


def net(v, r, l):
    a = v - r
    if not a > 0.0:
        a = 0.0
    return l if a > l else a


def oracle_h(orc, wl, layer):
    """The oracle's occurrence loss of every catalog event: one trial per
    event, aggregate terms neutral, so the trial loss is the event's h."""
    C = wl.yet.catalog
    probe = W.Workload("h", W.YET(catalog=C, n_trials=C, ids=np.arange(C, dtype=np.int32), k=1),
                       wl.elts, [W.Layer(wl.layers[layer].elts, wl.layers[layer].occ_r,
                                         wl.layers[layer].occ_l, 0.0, INF)])
    return orc.simulate_layer(probe, 0).ylt


def exact_ylt(wl, layer, h, trials):
    """The folded table's defined result, from exact rational arithmetic."""
    hmax = float(h.max())
    s = 125 - (math.frexp(hmax)[1] - 1) if hmax > 0 else 0
    scale = Fraction(2) ** s
    q = {}
    L = wl.layers[layer]
    out = np.empty(len(trials))
    for n, i in enumerate(trials):
        tot = 0
        for e in wl.yet.trial(int(i)):
            e = int(e)
            if e not in q:
                x = Fraction(float(h[e])) * scale
                q[e] = math.floor(x + Fraction(1, 2))
            tot += q[e]
        out[n] = net(float(Fraction(tot) / scale), L.agg_r, L.agg_l)
    return out


def small_workload(seed, J, catalog, n_trials, mean, ragged, pareto=False):
    g = np.random.Generator(np.random.PCG64(seed))
    yet = (W.yet_poisson(g, n_trials, mean, catalog, timestamps=False) if ragged
           else W.yet_fixed(g, n_trials, int(mean), catalog, timestamps=False))
    elts = []
    for j in range(J):
        nnz = int(g.integers(catalog // 50, catalog // 10))
        e = W.elt_pareto(g, catalog, nnz) if pareto else W.elt_lognormal(g, catalog, nnz)
        e = W.percentile_terms(e, int(g.integers(0, 200)), int(g.integers(950, 1000)))
        e.share = float(g.choice([1.0, 0.5, 0.25]))
        e.fx = float(g.choice([1.0, 1.1]))
        elts.append(e)
    pooled = np.concatenate([e.losses for e in elts])
    q = lambda p: W.nearest_rank(pooled, p)
    layers = [W.Layer(list(range(J)), q(300), q(995) * 3, q(500), q(999) * 30),
              W.Layer(list(range(J))[::-1], q(100), INF, 0.0, INF)]
    return W.Workload("fold", yet, elts, layers)


@pytest.mark.parametrize("J,ragged", [(1, False), (4, True), (16, False), (27, True), (32, False)])
def test_folded_is_the_exact_sum_of_oracle_occurrence_losses(are, ctx, orc, J, ragged):
    wl = small_workload(100 + J, J, 20_000, 3000, 60, ragged)
    L = Loaded(are, ctx, wl, timestamps=False)
    try:
        for layer in (0, 1):
            got = L.folded(layer)
            ref = orc.simulate_layer(wl, layer)
            ok, st = mixed_check(got, ref.ylt, trial_bound(wl, layer), RTOL["folded"])
            assert ok, (layer, st)
            h = oracle_h(orc, wl, layer)
            pick = np.random.default_rng(J).choice(wl.yet.n_trials, 400, replace=False)
            np.testing.assert_array_equal(got[pick], exact_ylt(wl, layer, h, pick))
    finally:
        L.release()


@pytest.mark.parametrize("J,ragged", [(4, True), (9, False), (16, True), (32, False)])
def test_fp64_per_elt_analysis_equals_the_exact_sum(are, ctx, orc, tmp_path, J, ragged):
    """The FP64 analysis over the per-ELT rows forms every occurrence loss as
    the oracle does and sums a trial's exactly, in whatever order it takes
    them, so on trials of many events it gives the folded pass's result bit
    for bit (every occurrence loss here converts to both fixed-point scales
    without rounding), with one or two groups of 32 events per batch and
    32- or 64-byte rows (4 and 9 ELTs hold few entries per catalog event,
    16 and 32 many)."""
    wl = small_workload(300 + J, J, 20_000, 3000, 90, ragged)
    L = Loaded(are, ctx, wl, timestamps=False)
    try:
        are.are_autotune(ctx, L.layers[:1], L.yet, 0)
        path = tmp_path / "t.jsonl"
        are.are_tune_save(ctx, str(path))
        entries = [json.loads(l) for l in open(path) if l.strip()]
        key = [e for e in entries if e["key"].startswith("p0_") and e["key"].endswith("_single")]
        assert key
        for layer in (0, 1):
            want = L.folded(layer)
            assert (want > 0).mean() > 0.2
            for u in (1, 2):
                path.write_text("".join(json.dumps(dict(e, kernel=2, rows_in_flight=u)) + "\n"
                                        for e in key))
                are.are_tune_load(ctx, str(path))
                np.testing.assert_array_equal(L.simulate(layer, 0), want, err_msg=f"layer {layer}, U {u}")
    finally:
        L.release()


def test_one_event_trials_give_the_oracle_occurrence_loss(are, ctx, orc):
    """With one event per trial the trial loss is net(h[e]) exactly, so it
    equals the oracle's bit for bit, for every catalog event."""
    base = small_workload(7, 12, 30_000, 10, 10, False)
    C = base.yet.catalog
    yet = W.YET(catalog=C, n_trials=C, ids=np.random.default_rng(1).permutation(C).astype(np.int32), k=1)
    wl = W.Workload("one", yet, base.elts, base.layers)
    L = Loaded(are, ctx, wl, timestamps=False)
    try:
        for layer in (0, 1):
            np.testing.assert_array_equal(L.folded(layer), orc.simulate_layer(wl, layer).ylt)
            # the FP64 per-ELT path forms the same event losses
            np.testing.assert_array_equal(L.simulate(layer, 0), L.folded(layer))
    finally:
        L.release()


def test_order_and_split_invariance(are, ctx, orc):
    wl = small_workload(11, 9, 20_000, 4000, 80, True)
    L = Loaded(are, ctx, wl, timestamps=False)
    try:
        whole = L.folded(0)
        parts = np.concatenate([L.folded(0, b, n) for b, n in ((0, 1), (1, 1234), (1235, 2765))])
        np.testing.assert_array_equal(parts, whole)
        host = L.folded(0, 100, 900, device=False)
        np.testing.assert_array_equal(host, whole[100:1000])
    finally:
        L.release()
    # the same events in reversed order within every trial
    y = wl.yet
    rev = np.concatenate([y.trial(i)[::-1] for i in range(y.n_trials)]).astype(np.int32)
    wl2 = W.Workload("rev", W.YET(catalog=y.catalog, n_trials=y.n_trials, ids=rev,
                                  offsets=y.offsets), wl.elts, wl.layers)
    L2 = Loaded(are, ctx, wl2, timestamps=False)
    try:
        np.testing.assert_array_equal(L2.folded(0), whole)
    finally:
        L2.release()


def test_large_catalog_bitmap_outside_shared_memory(are, ctx, orc):
    """A 2,000,000-event catalog: the bitmap (250 KB) is read from global
    memory instead of shared memory."""
    wl = small_workload(21, 32, 2_000_000, 3000, 200, True, pareto=True)
    L = Loaded(are, ctx, wl, timestamps=False)
    try:
        got = L.folded(0)
        ref = orc.simulate_layer(wl, 0)
        ok, st = mixed_check(got, ref.ylt, trial_bound(wl, 0), RTOL["folded"])
        assert ok, st
        assert (got > 0).mean() > 0.2
    finally:
        L.release()


def test_empty_and_long_trials(are, ctx, orc):
    """Trials of 0 events, and trials longer than one pass (1024 ids)."""
    g = np.random.Generator(np.random.PCG64(5))
    counts = g.choice([0, 1, 3, 1023, 1024, 1025, 2500], size=600)
    off = np.zeros(601, np.int64)
    np.cumsum(counts, out=off[1:])
    C = 5000
    ids = g.integers(0, C, size=int(off[-1]), dtype=np.int32)
    elts = [W.percentile_terms(W.elt_lognormal(g, C, 800)) for _ in range(6)]
    wl = W.Workload("e", W.YET(catalog=C, n_trials=600, ids=ids, offsets=off), elts,
                    [W.Layer(list(range(6)), 1e4, 1e6, 5e4, INF)])
    L = Loaded(are, ctx, wl, timestamps=False)
    try:
        got = L.folded(0)
        assert np.all(got[counts == 0] == 0)
        ref = orc.simulate_layer(wl, 0)
        ok, st = mixed_check(got, ref.ylt, trial_bound(wl, 0), RTOL["folded"])
        assert ok, st
        h = oracle_h(orc, wl, 0)
        np.testing.assert_array_equal(got, exact_ylt(wl, 0, h, np.arange(600)))
    finally:
        L.release()


def test_all_zero_layer_and_arguments(are, ctx):
    import torch
    g = np.random.Generator(np.random.PCG64(8))
    yet = W.yet_fixed(g, 200, 50, 1000, timestamps=False)
    e = W.elt_lognormal(g, 1000, 100)
    e.ded = 1e300                        # nothing exceeds the deductible: h = 0 everywhere
    wl = W.Workload("z", yet, [e], [W.Layer([0], 0.0, INF, 0.0, INF)])
    L = Loaded(are, ctx, wl, timestamps=False)
    try:
        assert np.all(L.folded(0) == 0)
        with pytest.raises(are.AreError):
            are.are_simulate_folded(ctx, L.layers[0], L.yet, 150, 51,
                                    torch.zeros(51, dtype=torch.float64, device="cuda"))
        with pytest.raises(are.AreError):
            are.are_simulate_folded(ctx, 987654, L.yet, 0, 1,
                                    torch.zeros(1, dtype=torch.float64, device="cuda"))
        are.are_prepare_folded(ctx, L.layers[0], L.yet)
    finally:
        L.release()
