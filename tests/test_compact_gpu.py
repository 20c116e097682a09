"""The compact layer table (are_set_table_layout ARE_LAYOUT_COMPACT): a row
index over the catalog and rows only for the events present in some ELT.
The staged kernel reads the same values in the same order through it, so the
YLT must equal the direct layout's on the same kernel bit for bit (the
direct run is pinned to the staged kernel through the tuning file); the
FP32 results are also checked against the oracle."""
import json
import math
import os
import tempfile

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


def pin_staged(are, ctx, L, layer, p):
    """Make the direct layout's analysis of this layer run on the staged
    kernel, with the compact layout's events per lane (2 with Kahan sums,
    1 with FP64 sums): every single-layer entry of this precision in the
    tuning table is set to it."""
    are.are_autotune(ctx, [L.layers[layer]], L.yet, p)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "t.jsonl")
        are.are_tune_save(ctx, path)
        entries = [json.loads(x) for x in open(path) if x.strip()]
        pinned = [dict(e, kernel=1, rows_in_flight=2 if p == 1 else 1) for e in entries
                  if e["key"].startswith(f"p{p}_") and e["key"].endswith("_single")]
        assert pinned
        with open(path, "w") as f:
            f.write("".join(json.dumps(e) + "\n" for e in pinned))
        are.are_tune_load(ctx, path)


def both_layouts(are, ctx, L, layer, p):
    h = L.layers[layer]
    are.are_set_table_layout(ctx, h, are.ARE_LAYOUT_DIRECT)
    pin_staged(are, ctx, L, layer, p)
    direct = L.simulate(layer, p)
    are.are_set_table_layout(ctx, h, are.ARE_LAYOUT_COMPACT)
    are.are_prepare(ctx, h, L.yet, p)
    compact = L.simulate(layer, p)
    are.are_set_table_layout(ctx, h, are.ARE_LAYOUT_DIRECT)
    return direct, compact


@pytest.mark.parametrize("p", [1, 2])
def test_tiny_workload_same_as_direct_and_oracle(are, ctx, orc, p):
    wl = W.plain_tiny()
    wl.layers.append(W.Layer([3, 1, 0, 2], 5e4, 2e6, 1e5, INF))
    L = Loaded(are, ctx, wl, timestamps=False)
    try:
        for layer in (0, 1):
            direct, compact = both_layouts(are, ctx, L, layer, p)
            np.testing.assert_array_equal(compact, direct)
            ref = orc.simulate_layer(wl, layer)
            ok, st = mixed_check(compact, ref.ylt, trial_bound(wl, layer), RTOL[p])
            assert ok, st
    finally:
        L.release()


@pytest.mark.parametrize("J", [1, 5, 16, 32])
def test_large_sparse_catalog(are, ctx, J):
    """2,000,000-event catalog, ragged trials, Pareto ELTs (the precision
    stress shape, fewer trials)."""
    g = np.random.Generator(np.random.PCG64(70 + J))
    C = 2_000_000
    yet = W.yet_poisson(g, 3000, 300, C, timestamps=False)
    elts = [W.elt_pareto(g, C, int(g.integers(5000, 20000))) for _ in range(J)]
    for e in elts:
        e.share = float(g.choice([1.0, 0.5]))
    wl = W.Workload("sparse", yet, elts, [W.Layer(list(range(J)), 1e3, 1e8, 0.0, INF)])
    L = Loaded(are, ctx, wl, timestamps=False)
    try:
        for p in (1, 2):
            direct, compact = both_layouts(are, ctx, L, 0, p)
            np.testing.assert_array_equal(compact, direct)
            assert (compact > 0).mean() > 0.01   # not a degenerate all-zero case
    finally:
        L.release()


def test_empty_elts_streamed_and_arguments(are, ctx):
    import torch
    g = np.random.Generator(np.random.PCG64(77))
    C = 50_000
    yet = W.yet_fixed(g, 2000, 200, C, timestamps=False)
    empty = W.ELT(ids=np.zeros(0, np.int32), losses=np.zeros(0))
    elts = [W.elt_lognormal(g, C, 3000), empty, W.elt_lognormal(g, C, 500)]
    wl = W.Workload("e", yet, elts, [W.Layer([0, 1, 2], 1e3, INF, 0.0, INF), W.Layer([1], 0.0, INF, 0.0, INF)])
    L = Loaded(are, ctx, wl, timestamps=False)
    try:
        direct, compact = both_layouts(are, ctx, L, 0, 1)
        np.testing.assert_array_equal(compact, direct)
        _, only_empty = both_layouts(are, ctx, L, 1, 1)
        assert np.all(only_empty == 0)
        # the streamed analysis through the compact table
        are.are_set_table_layout(ctx, L.layers[0], are.ARE_LAYOUT_COMPACT)
        out = torch.full((2000,), -1.0, dtype=torch.float64, device="cuda")
        are.are_simulate_streamed(ctx, L.layers[0], C, 2000, None, 200, yet.ids, 1, out, chunk_events=50_000)
        np.testing.assert_array_equal(out.cpu().numpy(), direct)
        # FP64 keeps the direct layout
        f64 = L.simulate(0, 0)
        are.are_set_table_layout(ctx, L.layers[0], are.ARE_LAYOUT_DIRECT)
        np.testing.assert_array_equal(L.simulate(0, 0), f64)
        with pytest.raises(are.AreError):
            are.are_set_table_layout(ctx, L.layers[0], 7)
    finally:
        L.release()
