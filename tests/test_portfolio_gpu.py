"""Portfolio batching through the C ABI: several layers in one persistent,
graph-replayed launch (are_simulate_portfolio), batched PML/TVaR
(are_risk_measures_batch) and the autotuner, against the oracle and against
one-layer-at-a-time runs."""
import math
import os

import numpy as np
import pytest

import workloads as W
from gpu_support import Loaded, RTOL, mixed_check, rel_close, tail_candidates, trial_bound

pytestmark = pytest.mark.gpu
PRECISIONS = [0, 1, 2]


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


def small_portfolio(ragged: bool, n_trials=4000, n_layers=12):
    wl = W.portfolio(n_trials=n_trials, mean_events=150.0, catalog=20_000, n_layers=n_layers,
                     pool=40, max_j=32, nnz_range=(200, 2000))
    if not ragged:
        g = np.random.Generator(np.random.PCG64(5))
        wl.yet = W.yet_fixed(g, n_trials, 150, 20_000, timestamps=False)
    return wl


def device_ylts(n_layers, n):
    import torch
    return [torch.full((n,), -1.0, dtype=torch.float64, device="cuda") for _ in range(n_layers)]


@pytest.fixture(scope="module", params=[False, True], ids=["fixed", "ragged"])
def loaded(request, are, ctx, orc):
    wl = small_portfolio(request.param)
    L = Loaded(are, ctx, wl, timestamps=False)
    refs = [orc.simulate_layer(wl, i) for i in range(len(wl.layers))]
    yield L, refs
    L.release()


@pytest.mark.parametrize("precision", PRECISIONS)
def test_portfolio_matches_oracle_every_layer(are, ctx, loaded, precision):
    L, refs = loaded
    n = L.wl.yet.n_trials
    outs = device_ylts(len(L.layers), n)
    are.are_simulate_portfolio(ctx, L.layers, L.yet, 0, n, precision, outs)
    widths = set()
    for i, (o, ref) in enumerate(zip(outs, refs)):
        ok, st = mixed_check(o.cpu().numpy(), ref.ylt, trial_bound(L.wl, i), RTOL[precision])
        assert ok, (i, st)
        widths.add(len(L.wl.layers[i].elts))
    assert min(widths) <= 8 and max(widths) > 16      # every table width is exercised


@pytest.mark.parametrize("precision", PRECISIONS)
def test_graph_replay_and_trial_ranges(are, ctx, loaded, precision):
    L, _ = loaded
    n = L.wl.yet.n_trials
    a, b = device_ylts(len(L.layers), n), device_ylts(len(L.layers), n)
    are.are_simulate_portfolio(ctx, L.layers, L.yet, 0, n, precision, a)
    are.are_simulate_portfolio(ctx, L.layers, L.yet, 0, n, precision, a)   # replay
    are.are_simulate_portfolio(ctx, L.layers, L.yet, 0, n, precision, b)   # new plan
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x.cpu().numpy(), y.cpu().numpy())
    part = device_ylts(len(L.layers), n - 1001)
    are.are_simulate_portfolio(ctx, L.layers, L.yet, 1001, n - 1001, precision, part)
    for x, y in zip(a, part):
        np.testing.assert_array_equal(x.cpu().numpy()[1001:], y.cpu().numpy())


def test_fp64_portfolio_identical_to_single_layer_runs(are, ctx, loaded):
    L, _ = loaded
    n = L.wl.yet.n_trials
    outs = device_ylts(len(L.layers), n)
    are.are_simulate_portfolio(ctx, L.layers, L.yet, 0, n, 0, outs)
    for i, o in enumerate(outs):
        np.testing.assert_array_equal(o.cpu().numpy(), L.simulate(i, 0))


def test_batched_risk_measures(are, ctx, orc, loaded):
    L, refs = loaded
    n = L.wl.yet.n_trials
    outs = device_ylts(len(L.layers), n)
    are.are_simulate_portfolio(ctx, L.layers, L.yet, 0, n, 0, outs)
    rps, lv = [100.0, 250.0, 10.0], [0.99, 0.95]
    pml, tv = are.are_risk_measures_batch(ctx, outs, n, rps, lv)
    for i, o in enumerate(outs):
        p1, t1 = are.are_risk_measures(ctx, o, n, rps, lv)
        np.testing.assert_array_equal(pml[i], p1)
        assert rel_close(tv[i], t1, 1e-13)
        rp, rt = orc.risk_measures(refs[i].ylt, rps, lv)
        assert rel_close(pml[i], rp, 1e-12) and rel_close(tv[i], rt, 1e-12)
    many = [o for o in outs] * 3                      # a bigger batch: the scratch grows
    pml3, _ = are.are_risk_measures_batch(ctx, many, n, rps, [])
    np.testing.assert_array_equal(pml3[: len(outs)], pml)
    with pytest.raises(are.AreError):
        are.are_risk_measures_batch(ctx, [refs[0].ylt], n, rps, lv)   # host memory


@pytest.mark.parametrize("precision", [1, 2])
def test_autotune_and_tuning_file(are, ctx, loaded, tmp_path, precision):
    L, refs = loaded
    n = L.wl.yet.n_trials
    multi = are.are_autotune(ctx, L.layers, L.yet, precision)
    assert multi["kernel"] in (0, 1) and multi["ms"] > 0 and multi["trials_per_item"] > 0
    single = are.are_autotune(ctx, L.layers[:1], L.yet, precision)
    assert single["kernel"] in (0, 1, 2) and single["ms"] > 0
    outs = device_ylts(len(L.layers), n)
    are.are_simulate_portfolio(ctx, L.layers, L.yet, 0, n, precision, outs)
    for i, (o, ref) in enumerate(zip(outs, refs)):
        ok, st = mixed_check(o.cpu().numpy(), ref.ylt, trial_bound(L.wl, i), RTOL[precision])
        assert ok, st
    ok, st = mixed_check(L.simulate(0, precision), refs[0].ylt, trial_bound(L.wl, 0),
                         RTOL[precision])
    assert ok, st
    path = str(tmp_path / "tune.jsonl")
    are.are_tune_save(ctx, path)
    text = open(path).read()
    assert "_multi" in text and "_single" in text
    c2 = are.are_create(0)
    try:
        are.are_tune_load(c2, path)
        bad = tmp_path / "bad.jsonl"
        bad.write_text("not json\n")
        with pytest.raises(are.AreError):
            are.are_tune_load(c2, str(bad))
    finally:
        are.are_destroy(c2)


def test_portfolio_argument_errors(are, ctx, loaded):
    L, _ = loaded
    n = L.wl.yet.n_trials
    outs = device_ylts(len(L.layers), n)
    with pytest.raises(are.AreError):
        are.are_simulate_portfolio(ctx, L.layers, L.yet, 0, n + 1, 1, outs)
    with pytest.raises(are.AreError):
        are.are_simulate_portfolio(ctx, L.layers[:2], L.yet, 0, n, 1,
                                   [outs[0], np.zeros(n)])       # host output
    with pytest.raises(are.AreError) as e:
        are.are_simulate_portfolio(ctx, [L.layers[0], 99999], L.yet, 0, n, 1, outs[:2])
    assert e.value.status == are.ARE_ENOTFOUND


def test_portfolio_full_size(are, ctx, orc):
    """200,000 ragged trials (Poisson 1000), 64 layers of 1..32 ELTs from a
    pool of 256: sampled trials of every layer, and PML/TVaR of 8 layers
    through their tail trials, for every precision."""
    wl = W.portfolio()
    L = Loaded(are, ctx, wl, timestamps=False)
    n = wl.yet.n_trials
    rng = np.random.default_rng(2)
    try:
        for p in PRECISIONS:
            outs = device_ylts(len(L.layers), n)
            are.are_simulate_portfolio(ctx, L.layers, L.yet, 0, n, p, outs)
            rps, lv = [100.0, 250.0], [0.99]
            pml, tv = are.are_risk_measures_batch(ctx, outs, n, rps, lv)
            for i, o in enumerate(outs):
                got = o.cpu().numpy()
                assert np.all(got >= 0)
                sample = np.sort(rng.choice(n, 60, replace=False))
                ref = orc.simulate_layer(wl, i, trials=sample)
                ok, st = mixed_check(got[sample], ref.ylt, trial_bound(wl, i, sample), RTOL[p])
                assert ok, (p, i, st)
                if i % 8 == 0:
                    m_max = orc.rank_for_level(n, 0.99)
                    cand = tail_candidates(got, m_max, margin=m_max // 4 + 50)
                    rc = orc.simulate_layer(wl, i, trials=cand)
                    gap = np.sort(rc.ylt)[::-1][m_max - 1] - got[cand[-1]]
                    assert np.abs(got[cand] - rc.ylt).max() < gap or gap == 0
                    full = np.zeros(n)
                    full[cand] = rc.ylt
                    rp, rt = orc.risk_measures(full, rps, lv)
                    assert rel_close(pml[i], rp, RTOL[p]), (p, i, pml[i], rp)
                    assert rel_close(tv[i], rt, RTOL[p]), (p, i, tv[i], rt)
    finally:
        L.release()
