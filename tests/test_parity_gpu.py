"""GPU path (libare through its C ABI) against the FP64 CPU oracle.

Every comparison is element by element on the same seeded inputs.  FP64
results must agree within 1e-12 and the FP32 paths within 1e-5, relative to
the oracle's value or, for trial losses, to the trial's cancellation bound
(gpu_support.trial_bound: the running total before the aggregate terms plus
the event losses that reach the occurrence retention; see
gpu_support.mixed_check).  Ids, counts and selected order statistics are
exact."""
import math

import numpy as np
import pytest

import workloads as W
from gpu_support import Loaded, RTOL, mixed_check, rel_close, tail_candidates, trial_bound

pytestmark = pytest.mark.gpu
INF = math.inf
PRECISIONS = [0, 1, 2]


@pytest.fixture(scope="module")
def are():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1308_2066_gb300 as are
    are.lib()
    return are


@pytest.fixture(scope="module")
def ctx(are):
    c = are.are_create(0)
    yield c
    are.are_destroy(c)


@pytest.fixture(scope="module")
def tiny(are, ctx):
    wl = W.plain_tiny()
    wl.layers.append(W.Layer(elts=[0, 1, 2, 3], occ_r=5e4, occ_l=2e6, agg_r=1e5, agg_l=INF))
    L = Loaded(are, ctx, wl)
    yield L
    L.release()


@pytest.fixture(scope="module")
def tiny_oracle(orc, tiny):
    return [orc.simulate_layer(tiny.wl, i) for i in range(len(tiny.wl.layers))]


# ---------------------------------------------------------------------------
# the 10,000 x 100 workload, every trial
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("layer", [0, 1])
def test_tiny_workload_every_trial(tiny, tiny_oracle, precision, layer):
    ref = tiny_oracle[layer]
    got = tiny.simulate(layer, precision)
    ok, st = mixed_check(got, ref.ylt, trial_bound(tiny.wl, layer), RTOL[precision],
                         min_plain=0.999)
    assert ok, st
    assert np.all(got >= 0) and np.all(got <= tiny.wl.layers[layer].agg_l)
    at_cap = ref.ylt == tiny.wl.layers[layer].agg_l
    np.testing.assert_array_equal(got[at_cap], ref.ylt[at_cap])
    capped = float(np.mean(at_cap))
    if layer == 0:
        assert capped > 0.3      # the recipe's aggregate limit binds often
    else:
        assert capped == 0.0


@pytest.mark.parametrize("precision", PRECISIONS)
def test_tiny_workload_risk_measures(are, ctx, orc, tiny, tiny_oracle, precision):
    rps, lv = [100.0, 250.0, 10.0, 2.0], [0.99, 0.9, 0.5]
    for layer in (0, 1):
        got_ylt = tiny.simulate(layer, precision)
        pml, tv = are.are_risk_measures(ctx, got_ylt, None, rps, lv)
        rpml, rtv = orc.risk_measures(tiny_oracle[layer].ylt, rps, lv)
        assert rel_close(pml, rpml, RTOL[precision]), (pml, rpml)
        assert rel_close(tv, rtv, RTOL[precision]), (tv, rtv)
        if layer == 1:
            assert len(set(pml)) == len(pml)   # the uncapped variant is not degenerate


# ---------------------------------------------------------------------------
# PML / TVaR selection on given YLTs
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 100, 4097, 100_000, 1_000_003])
def test_risk_measures_on_oracle_ylt(are, ctx, orc, n):
    import torch
    g = np.random.default_rng(n)
    y = np.round(g.lognormal(13, 2.5, n), 2)
    y[g.random(n) < 0.2] = 0.0
    y[g.random(n) < 0.05] = 1e7
    rps = [1.0, 1.5, 2.0, 10.0, 100.0, 250.0, 500.0, 1000.0, 10000.0]
    lv = [0.5, 0.9, 0.99, 0.995, 0.999]
    rpml, rtv = orc.risk_measures(y, rps, lv)
    for src in (y, torch.from_numpy(y).cuda()):
        pml, tv = are.are_risk_measures(ctx, src, n, rps, lv)
        np.testing.assert_array_equal(pml, rpml)
        assert rel_close(tv, rtv, 1e-13), (tv, rtv)


def test_risk_measures_long_ties_and_successive_calls(are, ctx, orc):
    """The single-YLT selection keeps up to 16384 keys of a target's bucket
    (1/16 of an octave) for its last step; a longer run of equal values
    there is selected from the whole YLT instead.  Successive calls on
    YLTs of falling magnitude and of other lengths leave no state behind."""
    import torch
    g = np.random.default_rng(9)
    n = 200_000
    y = np.concatenate([10.0 + g.lognormal(3, 1, 80_000), np.full(120_000, 5.0)])
    y = y[g.permutation(n)]
    rps, lv = [1.0, 2.0, 3.0, 100.0], [0.3, 0.5, 0.99]
    for arr in (y, -y, y * 1e-200, y[:4097], np.full(50_000, 7.25), y * 1e200, y):
        rpml, rtv = orc.risk_measures(arr, rps, lv)
        pml, tv = are.are_risk_measures(ctx, torch.from_numpy(arr).cuda(), None, rps, lv)
        np.testing.assert_array_equal(pml, rpml)
        # the tail sum is exact and rounded once, then divided: math.fsum's
        # correctly rounded sum over m gives the same double; the oracle's
        # sequential sum is within its own rounding of it
        top = np.sort(arr)[::-1]
        want = [math.fsum(top[: orc.rank_for_level(arr.size, a)]) / orc.rank_for_level(arr.size, a)
                for a in lv]
        np.testing.assert_array_equal(tv, want)
        assert rel_close(tv, rtv, 1e-11), (tv, rtv)


def test_risk_measures_into_device_arrays(are, ctx, orc):
    """With device output arrays the selection is only enqueued: the same
    values as the host-output call, for more targets than one selection
    batch takes (the PML and TVaR runs split across batches)."""
    import torch
    g = np.random.default_rng(5)
    y = np.round(g.lognormal(12, 2.0, 300_001), 2)
    rps = [1.0, 2.0, 5.0, 10.0, 50.0, 100.0, 250.0]
    lv = [0.5, 0.9, 0.99, 0.995, 0.999]
    yd = torch.from_numpy(y).cuda()
    want_pml, want_tv = are.are_risk_measures(ctx, yd, None, rps, lv)
    s = torch.cuda.Stream()
    pml = torch.full((len(rps),), -1.0, dtype=torch.float64, device="cuda")
    tv = torch.full((len(lv),), -1.0, dtype=torch.float64, device="cuda")
    assert are.are_risk_measures(ctx, yd, None, rps, lv, stream=s, out=(pml, tv)) is None
    s.synchronize()
    np.testing.assert_array_equal(pml.cpu().numpy(), want_pml)
    np.testing.assert_array_equal(tv.cpu().numpy(), want_tv)
    rpml, rtv = orc.risk_measures(y, rps, lv)
    np.testing.assert_array_equal(want_pml, rpml)
    # host and device outputs mixed, or a host YLT with device outputs
    for ylt, out in ((yd, (pml, np.empty(len(lv)))), (y, (pml, tv))):
        with pytest.raises(are.AreError) as e:
            are.are_risk_measures(ctx, ylt, None, rps, lv, out=out)
        assert e.value.status == are.ARE_EINVAL


def test_risk_measures_negative_and_tied_values(are, ctx, orc):
    y = np.array([-5.0, 3.0, 3.0, 3.0, -0.0, 0.0, 2.5, -1e300, 1e300, 7.0])
    rps, lv = [1.0, 2.0, 3.0, 10.0], [0.5, 0.7, 0.95]
    rpml, rtv = orc.risk_measures(y, rps, lv)
    pml, tv = are.are_risk_measures(ctx, y, None, rps, lv)
    np.testing.assert_array_equal(pml, rpml)
    assert rel_close(tv, rtv, 1e-13)


def test_layer_rows_arguments(are, ctx, tiny):
    """are_layer_rows reports, launches nothing and rejects bad arguments."""
    h, y = tiny.layers[0], tiny.yet
    l0 = are.are_launch_count(ctx)
    for p in PRECISIONS:
        for k in (-1, 0, 1, 2, 3):
            rb, packed = are.are_layer_rows(ctx, h, y, p, k)
            assert rb in (32, 64, 128) and (not packed or k in (-1, 2))
    assert are.are_launch_count(ctx) == l0
    with pytest.raises(are.AreError) as e:
        are.are_layer_rows(ctx, h, y, 1, 4)
    assert e.value.status == are.ARE_EINVAL
    with pytest.raises(are.AreError) as e:
        are.are_layer_rows(ctx, 987654, y, 1)
    assert e.value.status == are.ARE_ENOTFOUND


def test_risk_measure_arguments_rejected(are, ctx):
    y = np.ones(10)
    for rps, lv in (([0.5], []), ([], [1.0]), ([], [0.0]), ([float("nan")], [])):
        with pytest.raises(are.AreError) as e:
            are.are_risk_measures(ctx, y, None, rps, lv)
        assert e.value.status == are.ARE_EINVAL
    with pytest.raises(are.AreError):
        are.are_risk_measures(ctx, y, 0, [2.0], [])


# ---------------------------------------------------------------------------
# ragged YETs, every table width, financial-term variety
# ---------------------------------------------------------------------------

def ragged_workload(seed, J, n_trials=3000, mean=60, catalog=5000, nnz=300):
    g = np.random.Generator(np.random.PCG64(1000 + seed))
    yet = W.yet_poisson(g, n_trials, mean, catalog)
    elts = []
    for j in range(J):
        e = W.percentile_terms(W.elt_lognormal(g, catalog, nnz), int(g.integers(0, 300)),
                               int(g.integers(900, 1001)))
        e.fx = float(g.choice([1.0, 1.0, 0.83, 1.27]))
        e.share = float(g.choice([1.0, 1.0, 0.5, 0.35]))
        if j % 5 == 4:
            e.lim = INF
        elts.append(e)
    pooled = np.concatenate([e.losses for e in elts])
    occ_r = W.nearest_rank(pooled, 300)
    layer = W.Layer(list(range(J)), occ_r, W.nearest_rank(pooled, 995) * 3,
                    occ_r * 4, [INF, occ_r * 40][seed % 2])
    return W.Workload(f"ragged_j{J}", yet, elts, [layer])


@pytest.mark.parametrize("J", [1, 3, 4, 5, 8, 9, 12, 16, 17, 20, 24, 25, 31, 32])
def test_ragged_every_table_width(are, ctx, orc, J):
    wl = ragged_workload(J, J)
    L = Loaded(are, ctx, wl, device_inputs=bool(J % 2))
    try:
        ref = orc.simulate_layer(wl)
        for p in PRECISIONS:
            got = L.simulate(0, p)
            ok, st = mixed_check(got, ref.ylt, trial_bound(wl, 0), RTOL[p])
            assert ok, (p, st)
            assert np.all(got[ref.n_events == 0] == 0)
    finally:
        L.release()


@pytest.mark.parametrize("k", [1, 31, 32, 33, 63, 64, 65, 128, 129])
def test_fixed_trial_lengths_at_batch_edges(are, ctx, orc, k):
    """Trials whose length is a whole number of staging batches (32 or 64
    events), one more or one less: every batch full, or a last batch of a
    single event, in each precision."""
    g = np.random.Generator(np.random.PCG64(500 + k))
    yet = W.yet_fixed(g, 600, k, 5000)
    elts = [W.percentile_terms(W.elt_lognormal(g, 5000, 1500)) for _ in range(16)]
    pooled = np.concatenate([e.losses for e in elts])
    occ_r = W.nearest_rank(pooled, 200)
    wl = W.Workload(f"edges_k{k}", yet, elts,
                    [W.Layer(list(range(16)), occ_r, W.nearest_rank(pooled, 990) * 4, occ_r, INF)])
    L = Loaded(are, ctx, wl)
    try:
        ref = orc.simulate_layer(wl)
        for p in PRECISIONS:
            ok, st = mixed_check(L.simulate(0, p), ref.ylt, trial_bound(wl, 0), RTOL[p])
            assert ok, (p, st)
    finally:
        L.release()


# (J, catalog, events every ELT holds, other entries per ELT,
#  FP32 rows, FP64 rows) -- rows as (bytes, packed) from are_layer_rows
PACKED_CASES = [
    (8, 40_000, 200, 300, (32, False), (32, True)),
    (9, 40_000, 200, 300, (32, True), (32, True)),
    (12, 40_000, 200, 300, (32, True), (32, True)),
    (20, 40_000, 200, 300, (32, True), (32, True)),
    (32, 40_000, 200, 300, (32, True), (32, True)),
    (32, 20_000, 100, 1500, (64, True), (64, True)),
    (12, 3000, 600, 400, (64, False), (64, True)),
    (17, 3000, 600, 400, (64, True), (64, True)),
]


@pytest.mark.parametrize("case", PACKED_CASES, ids=lambda c: f"j{c[0]}_c{c[1]}")
def test_packed_rows_past_the_inline_terms(are, orc, case):
    """The register-rows kernels read packed rows -- the mask of an event's
    non-zero terms, then up to 7 or 15 FP32 terms (3 or 7 FP64) inline, the
    rest of a longer row in an overflow array -- of 32 bytes where the
    layer's entries per catalog event are few, else 64 bytes (or, for up to
    16 ELTs in FP32, the dense row).  The events that every ELT holds have J
    non-zero terms, past the inline ones; the others have a few.  Every
    precision matches the oracle, with the row size the layer calls for, on
    a fresh context (the untuned default)."""
    J, C, n_shared, n_other, rows32, rows64 = case
    g = np.random.Generator(np.random.PCG64(900 + J + C))
    yet = W.yet_poisson(g, 2000, 40, C)
    shared = g.permutation(C)[:n_shared]
    elts = []
    for _ in range(J):
        ids = np.unique(np.concatenate([shared, g.permutation(C)[:n_other]])).astype(np.int32)
        elts.append(W.ELT(ids, np.exp(g.normal(9.0, 1.5, ids.size))))
    wl = W.Workload("packed", yet, elts, [W.Layer(list(range(J)), 1e3, INF, 1e4, INF)])
    c = are.are_create(0)
    try:
        L = Loaded(are, c, wl)
        assert are.are_layer_rows(c, L.layers[0], L.yet, 1) == rows32
        assert are.are_layer_rows(c, L.layers[0], L.yet, 0) == rows64
        ref = orc.simulate_layer(wl)
        assert np.isin(yet.ids, shared).sum() > 50     # rows past the inline terms are read
        for p in (0, 1, 2):
            ok, st = mixed_check(L.simulate(0, p), ref.ylt, trial_bound(wl, 0), RTOL[p])
            assert ok, (p, st)
        L.release()
    finally:
        are.are_destroy(c)


def test_empty_trials_and_short_tails(are, ctx, orc):
    g = np.random.Generator(np.random.PCG64(77))
    yet = W.yet_poisson(g, 4000, 3, 300)         # many empty and 1-2 event trials
    elts = [W.percentile_terms(W.elt_lognormal(g, 300, 100)) for _ in range(6)]
    wl = W.Workload("short", yet, elts, [W.Layer(list(range(6)), 1e4, 5e5, 2e4, 1e6)])
    L = Loaded(are, ctx, wl)
    try:
        ref = orc.simulate_layer(wl)
        assert np.sum(ref.n_events == 0) > 100
        for p in PRECISIONS:
            ok, st = mixed_check(L.simulate(0, p), ref.ylt, trial_bound(wl, 0), RTOL[p])
            assert ok, (p, st)
    finally:
        L.release()


def test_trial_ranges_and_host_buffers(are, ctx, tiny):
    for p in PRECISIONS:
        whole = tiny.simulate(0, p)
        parts = [tiny.simulate(0, p, a, b - a) for a, b in ((0, 1), (1, 4093), (4093, 10_000))]
        np.testing.assert_array_equal(np.concatenate(parts), whole)
        np.testing.assert_array_equal(tiny.simulate(0, p, 17, 5000, device=False), whole[17:5017])


def test_negative_zero_terms_read_as_zero(are, ctx, orc, tiny):
    """Retentions and limits of -0.0 pass validation (they are >= 0) and act
    as +0.0: with both retentions 0 and then the occurrence limit 0, every
    precision gives the same trial losses as the layer defined with +0.0,
    and the oracle's."""
    for occ_r, occ_l, agg_r in ((0.0, 2e6, 0.0), (5e4, 0.0, 1e5)):
        pos = tiny.define(W.Layer([0, 1, 2, 3], occ_r, occ_l, agg_r, INF))
        neg = tiny.define(W.Layer([0, 1, 2, 3], -occ_r if occ_r == 0 else occ_r,
                                  -occ_l if occ_l == 0 else occ_l, -agg_r if agg_r == 0 else agg_r, INF))
        try:
            wl = W.Workload("z", tiny.wl.yet, tiny.wl.elts, [W.Layer([0, 1, 2, 3], occ_r, occ_l, agg_r, INF)])
            ref = orc.simulate_layer(wl, 0)
            for p in PRECISIONS:
                want = tiny.simulate(0, p, handle=pos)
                np.testing.assert_array_equal(tiny.simulate(0, p, handle=neg), want)
                ok, st = mixed_check(want, ref.ylt, trial_bound(wl, 0), RTOL[p])
                assert ok, (occ_r, occ_l, p, st)
            if occ_l == 0:
                assert np.all(want == 0)
        finally:
            are.are_free_layer(ctx, neg)
            are.are_free_layer(ctx, pos)


def test_single_trial_single_event(are, ctx, orc, golden):
    """The hand-worked cases of tests/golden through the GPU, every precision."""
    spec = golden["layers"]["two_elts"]
    cases = [c for c in golden["trials"] if c["layer"] == "two_elts"]
    counts = [len(c["events"]) for c in cases]
    off = np.zeros(len(cases) + 1, np.int64)
    off[1:] = np.cumsum(counts)
    ids = np.array([e for c in cases for e in c["events"]], np.int32)
    yet = W.YET(12, len(cases), ids, offsets=off)
    elts = [W.ELT(np.array(e["ids"], np.int32), np.array(e["losses"]), e["ded"],
                  INF if e["lim"] == "inf" else e["lim"], e["fx"], e["share"]) for e in spec["elts"]]
    wl = W.Workload("hand", yet, elts, [W.Layer([0, 1], spec["occ_r"], spec["occ_l"],
                                                 spec["agg_r"], spec["agg_l"])])
    L = Loaded(are, ctx, wl, timestamps=False)
    try:
        for p in PRECISIONS:
            np.testing.assert_array_equal(L.simulate(0, p), [c["ylt"] for c in cases])
    finally:
        L.release()


@pytest.mark.parametrize("share", [1.0, 0.35])
def test_term_arithmetic_bit_exact(are, ctx, share):
    """One event per trial, one ELT, neutral layer terms: each trial loss is
    one financial term, which the header fixes exactly.  The term
    share * min(max(fx * x - D, 0), Lim) is formed in FP64 as the terms
    define it and rounded once to the mode's type.  The expected values below
    restate that arithmetic in numpy."""
    g = np.random.Generator(np.random.PCG64(2024))
    catalog, n = 4096, 3000
    ids = g.permutation(catalog)[:n].astype(np.int32)        # 1096 events absent
    loss = np.exp(g.normal(11.0, 1.5, n))
    fx, ded, lim = 1.27, float(np.quantile(loss, 0.2)), float(np.quantile(loss, 0.9))
    elt = W.ELT(ids, loss, ded, lim, fx, share)
    yet = W.YET(catalog=catalog, n_trials=catalog, ids=np.arange(catalog, dtype=np.int32), k=1)
    wl = W.Workload("terms", yet, [elt], [W.Layer([0], 0.0, INF, 0.0, INF)])
    x = np.zeros(catalog)
    x[ids] = loss
    present = np.zeros(catalog, bool)
    present[ids] = True
    e64 = np.float64(fx) * x - ded                           # two FP64 roundings, as defined
    want64 = np.where(present, np.minimum(np.maximum(e64, 0.0), lim) * share, 0.0)
    want32 = want64.astype(np.float32).astype(np.float64)    # one rounding to FP32
    L = Loaded(are, ctx, wl, timestamps=False)
    try:
        np.testing.assert_array_equal(L.simulate(0, 0), want64)
        for p in (1, 2):
            np.testing.assert_array_equal(L.simulate(0, p), want32)
    finally:
        L.release()


# ---------------------------------------------------------------------------
# input validation through the boundary
# ---------------------------------------------------------------------------

def test_invalid_inputs_rejected(are, ctx):
    E = are.AreError
    ids = np.array([0, 1, 2, 3], np.int32)
    with pytest.raises(E) as e:
        are.are_load_yet(ctx, 3, 2, None, 2, ids)          # id 3 outside catalog of 3
    assert e.value.status == are.ARE_EINVAL
    with pytest.raises(E):
        are.are_load_yet(ctx, 4, 2, np.array([0, 3, 2], np.int64), 0, ids[:2])
    with pytest.raises(E):
        are.are_load_yet(ctx, 4, 2, np.array([0, 2, 4], np.int64), 0, ids,
                         np.array([0.1, 0.2, 0.9, 0.3], np.float32))
    with pytest.raises(E):
        are.are_load_yet(ctx, 4, 1, None, 0, ids)
    with pytest.raises(E):
        are.are_load_elt(ctx, np.array([1, 1], np.int32), np.array([1.0, 2.0]))
    with pytest.raises(E):
        are.are_load_elt(ctx, np.array([1], np.int32), np.array([-1.0]))
    with pytest.raises(E):
        are.are_load_elt(ctx, np.array([1], np.int32), np.array([1.0]), share=1.5)
    with pytest.raises(E):
        are.are_load_elt(ctx, np.array([1], np.int32), np.array([1.0]), deductible=INF)
    h = are.are_load_elt(ctx, np.array([1, 7], np.int32), np.array([1.0, 2.0]))
    with pytest.raises(E):
        are.are_define_layer(ctx, [h, h])
    with pytest.raises(E):
        are.are_define_layer(ctx, [h], occ_ret=-1.0)
    with pytest.raises(E):
        are.are_define_layer(ctx, [h] * 0)
    with pytest.raises(E) as e:
        are.are_define_layer(ctx, [h, 99999])
    assert e.value.status == are.ARE_ENOTFOUND
    lay = are.are_define_layer(ctx, [h])
    y = are.are_load_yet(ctx, 5, 2, None, 2, ids)
    with pytest.raises(E):          # ELT id 7 outside the YET's 5-event catalog
        are.are_simulate(ctx, lay, y, 0, 2, 0, np.zeros(2))
    with pytest.raises(E):
        are.are_simulate(ctx, lay, y, 1, 2, 0, np.zeros(2))
    with pytest.raises(E):
        are.are_simulate(ctx, lay, y, 0, 2, 7, np.zeros(2))
    with pytest.raises(E):
        are.are_free_elt(ctx, h)    # still used by the layer
    are.are_free_layer(ctx, lay)
    are.are_free_elt(ctx, h)
    are.are_free_yet(ctx, y)
    with pytest.raises(E) as e:
        are.are_free_yet(ctx, y)
    assert e.value.status == are.ARE_ENOTFOUND


def test_memory_budget(are):
    c = are.are_create(0, 1 << 20)
    try:
        before = are.are_memory_used(c)
        with pytest.raises(are.AreError) as e:
            are.are_load_yet(c, 10, 1000, None, 1000, np.zeros(10**6, np.int32))
        assert e.value.status == are.ARE_ENOMEM
        assert are.are_memory_used(c) == before
        y = are.are_load_yet(c, 10, 10, None, 10, np.zeros(100, np.int32))
        assert are.are_memory_used(c) > before
        are.are_free_yet(c, y)
        assert are.are_memory_used(c) == before
    finally:
        are.are_destroy(c)


def test_contexts_on_two_devices(are, orc):
    """A context on the second GPU, made after one on the first has run every
    precision, launches the same kernels (their shared-memory limits and
    grid sizes are kept per device) and gives the oracle's results."""
    import torch
    if torch.cuda.device_count() < 2:
        pytest.skip("needs two visible GPUs")
    wl = W.plain_tiny(n_trials=600)
    ref = orc.simulate_layer(wl)
    for dev in (0, 1):
        c = are.are_create(dev)
        try:
            torch.cuda.set_device(dev)
            L = Loaded(are, c, wl)
            for p in PRECISIONS:
                ok, st = mixed_check(L.simulate(0, p), ref.ylt, trial_bound(wl, 0), RTOL[p])
                assert ok, (dev, p, st)
            L.release()
        finally:
            are.are_destroy(c)
            torch.cuda.set_device(0)


# ---------------------------------------------------------------------------
# full-size workloads, in the launch configuration the benchmark times:
# sampled trials one by one, and PML/TVaR through their tail trials
# ---------------------------------------------------------------------------

def check_full_size(are, ctx, orc, wl, precisions, n_sample=1500, seed=0):
    rps, lv = [100.0, 250.0], [0.99]
    n = wl.yet.n_trials
    m_max = max(orc.rank_for_return_period(n, r) for r in rps)
    m_max = max(m_max, max(orc.rank_for_level(n, a) for a in lv))
    sample = np.sort(np.random.default_rng(seed).choice(n, n_sample, replace=False))
    L = Loaded(are, ctx, wl, timestamps=False)
    report = {}
    try:
        for p in precisions:
            got = L.run(0, p)
            assert np.all(np.isfinite(got)) and np.all(got >= 0)
            ref = orc.simulate_layer(wl, trials=sample)
            # at least 99.9% of the sampled trials pass the plain relative
            # test; the rest pass against the trial's cancellation bound
            ok, st = mixed_check(got[sample], ref.ylt, trial_bound(wl, 0, sample), RTOL[p],
                                 min_plain=0.999)
            assert ok, (p, st)
            np.testing.assert_array_equal(ref.n_events, wl.yet.counts()[sample])
            # tail: the m_max + margin largest GPU losses hold every trial the
            # oracle can rank in its top m_max, unless an error exceeds the gap
            cand = tail_candidates(got, m_max, margin=m_max // 5 + 100)
            rc = orc.simulate_layer(wl, trials=cand)
            err = np.abs(got[cand] - rc.ylt)
            gap = np.sort(rc.ylt)[::-1][m_max - 1] - got[cand[-1]]
            assert err.max() < gap, (p, err.max(), gap)
            full = np.zeros(n)
            full[cand] = rc.ylt
            rpml, rtv = orc.risk_measures(full, rps, lv)
            pml, tv = are.are_risk_measures(ctx, got, None, rps, lv)
            assert rel_close(pml, rpml, RTOL[p]), (p, pml, rpml)
            assert rel_close(tv, rtv, RTOL[p]), (p, tv, rtv)
            report[p] = {"ylt": st, "pml": list(pml), "pml_ref": list(rpml), "tvar": list(tv),
                         "tvar_ref": list(rtv)}
    finally:
        L.release()
    return report


def test_paper_scale_full_size(are, ctx, orc):
    """1,000,000 trials x 1000 events, 16 ELTs: every precision and the
    folded table."""
    wl = W.paper_scale()
    rep = check_full_size(are, ctx, orc, wl, PRECISIONS + ["folded"])
    print("paper_scale", rep)


def test_precision_stress_full_size(are, ctx, orc):
    """1,000,000 ragged trials (Poisson 1000, <= 3000), 2,000,000-event
    catalog, 32 Pareto ELTs, neutral terms: whole-trial sums reach the YLT."""
    wl = W.precision_stress()
    assert wl.yet.counts().max() <= 3000
    rep = check_full_size(are, ctx, orc, wl, PRECISIONS + ["folded"], n_sample=1000, seed=3)
    print("precision_stress", rep)
