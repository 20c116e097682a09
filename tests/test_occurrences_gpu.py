"""Per-occurrence outputs (are_simulate_occurrences) and every kernel choice
of the analysis stage, against the oracle."""
import json
import math

import numpy as np
import pytest

import workloads as W
from gpu_support import Loaded, RTOL, mixed_check, running_bound, trial_bound

pytestmark = pytest.mark.gpu
INF = math.inf
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


def occurrences(are, ctx, L, layer, p, begin=0, n=None):
    import torch
    y = L.wl.yet
    n = y.n_trials - begin if n is None else n
    first = y.bounds(begin)[0] if n else 0
    last = y.bounds(begin + n - 1)[1] if n else 0
    marg = torch.full((max(1, last - first),), -7.0, dtype=torch.float64, device="cuda")
    omax = torch.full((n,), -7.0, dtype=torch.float64, device="cuda")
    ylt = torch.full((n,), -7.0, dtype=torch.float64, device="cuda")
    are.are_simulate_occurrences(ctx, L.layers[layer], L.yet, begin, n, p, marg, omax, ylt)
    return marg.cpu().numpy()[: last - first], omax.cpu().numpy(), ylt.cpu().numpy()


def check_against_oracle(orc, L, layer, p, marg, omax, ylt, trials=None):
    ref = orc.simulate_layer(L.wl, layer, trials=trials, marginals=True)
    bound = trial_bound(L.wl, layer, trials)
    ok, st = mixed_check(ylt, ref.ylt, bound, RTOL[p])
    assert ok, ("ylt", p, st)
    ok, st = mixed_check(omax, ref.occ_max, bound, RTOL[p])
    assert ok, ("occ_max", p, st)
    if p == 0:   # the event loss is formed in the oracle's order: occurrence losses are exact
        np.testing.assert_array_equal(omax, ref.occ_max)
    ok, st = mixed_check(marg, ref.marginals, running_bound(L.wl, layer, trials), RTOL[p])
    assert ok, ("marginals", p, st)
    return ref


@pytest.mark.parametrize("p", PRECISIONS)
def test_tiny_workload_occurrences(are, ctx, orc, p):
    wl = W.plain_tiny()
    wl.layers.append(W.Layer([0, 1, 2, 3], 5e4, 2e6, 1e5, INF))
    L = Loaded(are, ctx, wl)
    try:
        for layer in (0, 1):
            marg, omax, ylt = occurrences(are, ctx, L, layer, p)
            ref = check_against_oracle(orc, L, layer, p, marg, omax, ylt)
            # the marginals of a trial add up to its loss
            per_trial = marg.reshape(wl.yet.n_trials, wl.yet.k).sum(axis=1)
            np.testing.assert_allclose(per_trial, ylt, rtol=1e-9, atol=1e-6)
            # a sub-range writes the same values from its own first event on
            m2, o2, y2 = occurrences(are, ctx, L, layer, p, begin=1234, n=4321)
            np.testing.assert_array_equal(m2, marg[1234 * 100:(1234 + 4321) * 100])
            np.testing.assert_array_equal(o2, omax[1234:1234 + 4321])
            np.testing.assert_array_equal(y2, ylt[1234:1234 + 4321])
            assert np.all(marg >= 0)        # the clamped running total never decreases
    finally:
        L.release()


@pytest.mark.parametrize("J", [1, 3, 8, 9, 13, 16, 20, 24, 27, 32])
def test_ragged_occurrences_every_width(are, ctx, orc, J):
    g = np.random.Generator(np.random.PCG64(300 + J))
    yet = W.yet_poisson(g, 2500, 40, 3000)
    elts = []
    for j in range(J):
        e = W.percentile_terms(W.elt_lognormal(g, 3000, 200), int(g.integers(0, 300)), 990)
        e.share = float(g.choice([1.0, 0.5]))
        elts.append(e)
    pooled = np.concatenate([e.losses for e in elts])
    layer = W.Layer(list(range(J)), W.nearest_rank(pooled, 200), INF, W.nearest_rank(pooled, 600),
                    W.nearest_rank(pooled, 990) * 20)
    wl = W.Workload("occ", yet, elts, [layer])
    L = Loaded(are, ctx, wl, timestamps=False)
    try:
        for p in PRECISIONS:
            marg, omax, ylt = occurrences(are, ctx, L, 0, p)
            check_against_oracle(orc, L, 0, p, marg, omax, ylt)
    finally:
        L.release()


def test_empty_trials(are, ctx, orc):
    g = np.random.Generator(np.random.PCG64(9))
    yet = W.yet_poisson(g, 3000, 2, 500)
    elts = [W.percentile_terms(W.elt_lognormal(g, 500, 100)) for _ in range(5)]
    wl = W.Workload("e", yet, elts, [W.Layer(list(range(5)), 1e4, INF, 1e4, INF)])
    L = Loaded(are, ctx, wl, timestamps=False)
    try:
        for p in PRECISIONS:
            marg, omax, ylt = occurrences(are, ctx, L, 0, p)
            empty = yet.counts() == 0
            assert empty.sum() > 100
            assert np.all(ylt[empty] == 0) and np.all(omax[empty] == 0)
            check_against_oracle(orc, L, 0, p, marg, omax, ylt)
    finally:
        L.release()


def test_occurrence_arguments(are, ctx):
    import torch
    wl = W.plain_tiny(n_trials=100)
    L = Loaded(are, ctx, wl)
    try:
        with pytest.raises(are.AreError):
            are.are_simulate_occurrences(ctx, L.layers[0], L.yet, 0, 100, 0, np.zeros(10_000))
        with pytest.raises(are.AreError):
            are.are_simulate_occurrences(ctx, L.layers[0], L.yet, 50, 51, 0,
                                         torch.zeros(10_000, dtype=torch.float64, device="cuda"))
    finally:
        L.release()


@pytest.mark.parametrize("p", PRECISIONS)
def test_every_kernel_choice(are, ctx, orc, tmp_path, p):
    """Each single-layer kernel the tuner can pick gives oracle results: the
    tuning file written by the library is edited to force each choice."""
    wl = W.plain_tiny(n_trials=3000)
    L = Loaded(are, ctx, wl)
    try:
        ref = orc.simulate_layer(wl)
        are.are_autotune(ctx, L.layers[:1], L.yet, p)
        path = tmp_path / "t.jsonl"
        are.are_tune_save(ctx, str(path))
        entries = [json.loads(l) for l in open(path) if l.strip()]
        key = [e for e in entries if e["key"].startswith(f"p{p}_") and e["key"].endswith("_single")]
        assert key
        kinds = [1, 2] + ([0] if p != 0 else [3])
        for kind in kinds:
            for u in (1, 2):
                path.write_text("".join(json.dumps(dict(e, kernel=kind, rows_in_flight=u,
                                                        trials_per_item=3)) + "\n" for e in key))
                are.are_tune_load(ctx, str(path))
                ok, st = mixed_check(L.simulate(0, p), ref.ylt, trial_bound(wl, 0), RTOL[p])
                assert ok, (kind, u, st)
    finally:
        L.release()


@pytest.mark.parametrize("with_share", [False, True])
def test_fp64_kernels_with_and_without_share_factors(are, ctx, orc, tmp_path, with_share):
    """Each FP64 kernel the tuner can pick (staged, register, screened) gives
    the oracle's trial losses on a ragged 16-ELT layer, both when every
    share is 1 (each lane clamps its own columns) and when some are not (the
    warp-wide list of marked entries)."""
    g = np.random.Generator(np.random.PCG64(41 + with_share))
    yet = W.yet_poisson(g, 3000, 70, 4000)
    elts = []
    for j in range(16):
        e = W.percentile_terms(W.elt_lognormal(g, 4000, 400), int(g.integers(0, 300)), 990)
        if with_share:
            e.share = float(g.choice([1.0, 0.5, 0.35]))
        elts.append(e)
    pooled = np.concatenate([e.losses for e in elts])
    occ_r = W.nearest_rank(pooled, 200)
    wl = W.Workload("fp64_kernels", yet, elts,
                    [W.Layer(list(range(16)), occ_r, W.nearest_rank(pooled, 990) * 5, occ_r * 3, INF)])
    L = Loaded(are, ctx, wl)
    try:
        ref = orc.simulate_layer(wl)
        are.are_autotune(ctx, L.layers[:1], L.yet, 0)
        path = tmp_path / "t.jsonl"
        are.are_tune_save(ctx, str(path))
        entries = [json.loads(l) for l in open(path) if l.strip()]
        key = [e for e in entries if e["key"].startswith("p0_") and e["key"].endswith("_single")]
        assert key
        for kind in (1, 2, 3):
            path.write_text("".join(json.dumps(dict(e, kernel=kind)) + "\n" for e in key))
            are.are_tune_load(ctx, str(path))
            ok, st = mixed_check(L.simulate(0, 0), ref.ylt, trial_bound(wl, 0), RTOL[0])
            assert ok, (kind, st)
    finally:
        L.release()
