"""are_simulate_streamed: the analysis over a host-resident YET, copied to
the device chunk by chunk while earlier chunks are analysed (ids as int32,
or packed a few bits each by are_pack_ids).  Each trial is
computed by the same kernel as are_simulate, so the YLTs must be equal bit
for bit, whatever the chunking; the FP64 result is also checked against the
oracle."""
import math

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


def streamed(are, ctx, L, layer, p, chunk, pinned=True, host_out=False):
    import torch
    y = L.wl.yet
    ids = torch.from_numpy(y.ids).pin_memory() if pinned else y.ids
    off = None if y.offsets is None else y.offsets
    if host_out:
        out = np.full(y.n_trials, -1.0)
    else:
        out = torch.full((y.n_trials,), -1.0, dtype=torch.float64, device="cuda")
    are.are_simulate_streamed(ctx, L.layers[layer], y.catalog, y.n_trials, off, y.k or 0, ids, p,
                              out, chunk_events=chunk)
    return out if host_out else out.cpu().numpy()


@pytest.mark.parametrize("p", [0, 1, 2])
def test_fixed_yet_equals_resident_analysis(are, ctx, orc, p):
    wl = W.plain_tiny()
    L = Loaded(are, ctx, wl, timestamps=False)
    try:
        ref = L.simulate(0, p)
        for chunk, pinned, host_out in ((0, True, False), (3000, True, True), (777, False, False)):
            np.testing.assert_array_equal(streamed(are, ctx, L, 0, p, chunk, pinned, host_out), ref)
        if p == 0:
            o = orc.simulate_layer(wl, 0)
            ok, st = mixed_check(ref, o.ylt, trial_bound(wl, 0), RTOL[0])
            assert ok, st
    finally:
        L.release()


def test_ragged_yet_with_long_and_empty_trials(are, ctx):
    g = np.random.Generator(np.random.PCG64(12))
    counts = g.choice([0, 1, 5, 300, 2000, 5000], size=800)
    off = np.zeros(801, np.int64)
    np.cumsum(counts, out=off[1:])
    C = 6000
    ids = g.integers(0, C, size=int(off[-1]), dtype=np.int32)
    elts = [W.percentile_terms(W.elt_lognormal(g, C, 900)) for _ in range(11)]
    wl = W.Workload("r", W.YET(catalog=C, n_trials=800, ids=ids, offsets=off), elts,
                    [W.Layer(list(range(11)), 1e4, 1e6, 5e4, 5e8)])
    L = Loaded(are, ctx, wl, timestamps=False)
    try:
        for p in (0, 1, 2):
            ref = L.simulate(0, p)
            for chunk in (0, 1000, 4096):   # 1000: trials of 2000 and 5000 ids form chunks alone
                np.testing.assert_array_equal(streamed(are, ctx, L, 0, p, chunk), ref)
    finally:
        L.release()


def test_invalid_ids_and_arguments(are, ctx):
    import torch
    wl = W.plain_tiny(n_trials=500)
    L = Loaded(are, ctx, wl, timestamps=False)
    try:
        bad = wl.yet.ids.copy()
        bad[12345] = wl.yet.catalog          # one id past the catalog
        out = torch.zeros(500, dtype=torch.float64, device="cuda")
        with pytest.raises(are.AreError) as e:
            are.are_simulate_streamed(ctx, L.layers[0], wl.yet.catalog, 500, None, 100, bad, 1, out,
                                      chunk_events=2000)
        assert e.value.status == are.ARE_EINVAL
        # the context still works
        np.testing.assert_array_equal(streamed(are, ctx, L, 0, 1, 0), L.simulate(0, 1))
        dev_ids = torch.from_numpy(wl.yet.ids).cuda()
        with pytest.raises(are.AreError):
            are.are_simulate_streamed(ctx, L.layers[0], wl.yet.catalog, 500, None, 100, dev_ids, 1, out)
        with pytest.raises(are.AreError):
            are.are_simulate_streamed(ctx, L.layers[0], wl.yet.catalog, 500, None, 0, wl.yet.ids, 1, out)
    finally:
        L.release()


def pack_bits(ids, bits):
    """The packed layout written out independently: id i in bits
    i*bits .. (i+1)*bits-1 of a little-endian stream of 32-bit words."""
    n = len(ids)
    words = np.zeros((n * bits + 31) // 32 + 1, np.uint64)
    for i, v in enumerate(ids.astype(np.uint64)):
        b = i * bits
        w, sh = b // 32, b % 32
        x = int(v) << sh
        words[w] |= np.uint64(x & 0xFFFFFFFF)
        words[w + 1] |= np.uint64(x >> 32)
    return words[: (n * bits + 31) // 32].astype(np.uint32)


def test_pack_ids_layout(are, ctx):
    g = np.random.default_rng(21)
    for bits in (1, 7, 13, 20, 31, 32):
        n = 1000 + bits
        hi = min(1 << bits, 2**31 - 1)
        ids = g.integers(0, hi, size=n, dtype=np.int64).astype(np.int32)
        np.testing.assert_array_equal(are.are_pack_ids(ctx, ids, bits), pack_bits(ids, bits))
    with pytest.raises(are.AreError) as e:
        are.are_pack_ids(ctx, np.array([0, 8], np.int32), 3)      # 8 needs 4 bits
    assert e.value.status == are.ARE_EINVAL
    assert are.are_pack_ids(ctx, np.zeros(0, np.int32), 20).size == 0


@pytest.mark.parametrize("bits", [None, 32, 20])
def test_packed_ids_equal_plain_streaming(are, ctx, bits):
    """Ids packed in the fewest bits the catalog needs (or 20, or 32): the
    same YLT as the resident analysis, fixed and ragged YETs, every chunking;
    ids past the catalog that the bits can hold are reported."""
    import torch
    g = np.random.Generator(np.random.PCG64(15))
    counts = g.choice([0, 1, 5, 33, 300, 2000], size=700)
    off = np.zeros(701, np.int64)
    np.cumsum(counts, out=off[1:])
    C = 6000
    need = int(np.ceil(np.log2(C)))
    b = need if bits is None else bits
    ids = g.integers(0, C, size=int(off[-1]), dtype=np.int32)
    elts = [W.percentile_terms(W.elt_lognormal(g, C, 900)) for _ in range(11)]
    for offsets, k in ((off, 0), (None, None)):
        if offsets is None:   # a fixed YET over the same ids
            k = 97
            n_trials = len(ids) // k
            yet = W.YET(catalog=C, n_trials=n_trials, ids=ids[: n_trials * k].copy(), k=k)
        else:
            yet = W.YET(catalog=C, n_trials=700, ids=ids, offsets=offsets)
        wl = W.Workload("p", yet, elts, [W.Layer(list(range(11)), 1e4, 1e6, 5e4, 5e8)])
        L = Loaded(are, ctx, wl, timestamps=False)
        try:
            words = are.are_pack_ids(ctx, yet.ids, b)
            pinned = torch.from_numpy(words.view(np.int32)).pin_memory()
            for p in (0, 1):
                ref = L.simulate(0, p)
                for chunk in (0, 1000, 4099):
                    out = torch.full((yet.n_trials,), -1.0, dtype=torch.float64, device="cuda")
                    are.are_simulate_streamed_packed(ctx, L.layers[0], C, yet.n_trials, yet.offsets,
                                                     k or 0, pinned.data_ptr(), b, p, out,
                                                     chunk_events=chunk)
                    np.testing.assert_array_equal(out.cpu().numpy(), ref)
            if b > need:   # an id the bits can hold but the catalog does not
                bad = yet.ids.copy()
                bad[len(bad) // 2] = C
                out = torch.zeros(yet.n_trials, dtype=torch.float64, device="cuda")
                with pytest.raises(are.AreError) as e:
                    are.are_simulate_streamed_packed(ctx, L.layers[0], C, yet.n_trials, yet.offsets,
                                                     k or 0, are.are_pack_ids(ctx, bad, b), b, 1, out)
                assert e.value.status == are.ARE_EINVAL
        finally:
            L.release()
    with pytest.raises(are.AreError) as e:
        are.are_simulate_streamed_packed(ctx, 0, C, 1, None, 5, np.zeros(4, np.uint32), 0, 1,
                                         np.zeros(1))
    assert e.value.status == are.ARE_EINVAL


def test_device_offsets_and_caller_stream(are, ctx):
    """Offsets given in device memory, the analysis enqueued after other work
    on a caller stream: the same YLT as the resident analysis."""
    import torch
    g = np.random.Generator(np.random.PCG64(13))
    yet = W.yet_poisson(g, 1500, 150, 8000, timestamps=False)
    elts = [W.percentile_terms(W.elt_lognormal(g, 8000, 700)) for _ in range(6)]
    wl = W.Workload("d", yet, elts, [W.Layer(list(range(6)), 1e4, 1e6, 2e4, INF)])
    L = Loaded(are, ctx, wl, timestamps=False)
    try:
        ref = L.simulate(0, 1)
        s = torch.cuda.Stream()
        off = torch.from_numpy(yet.offsets).cuda()
        out = torch.full((1500,), -1.0, dtype=torch.float64, device="cuda")
        with torch.cuda.stream(s):
            out.fill_(-2.0)                   # queued before the analysis on the same stream
        are.are_simulate_streamed(ctx, L.layers[0], yet.catalog, 1500, off, 0, yet.ids, 1, out,
                                  chunk_events=20_000, stream=s)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), ref)
    finally:
        L.release()


def test_gather_ceiling(are, ctx):
    """The measurement helper: a positive rate for each row size, argument checks."""
    import torch
    g = np.random.Generator(np.random.PCG64(14))
    yet = W.yet_fixed(g, 4000, 500, 100_000, timestamps=False)
    h = are.are_load_yet(ctx, yet.catalog, yet.n_trials, None, yet.k, torch.from_numpy(yet.ids).cuda())
    try:
        for rb in (32, 64, 128):
            rate, shapes = are.are_gather_ceiling(ctx, h, rb, 0, yet.n_trials, reps=1, shapes=True)
            assert rate > 1e8
            # every kind of shape was timed, and the best of them is the rate
            assert {k for k, _, _, _ in shapes} == {0, 1, 2}
            assert rate == max(r for _, _, _, r in shapes)
            assert all(b >= 1 for _, _, b, _ in shapes)
        with pytest.raises(are.AreError):
            are.are_gather_ceiling(ctx, h, 48, 0, yet.n_trials)
        with pytest.raises(are.AreError):
            are.are_gather_ceiling(ctx, h, 64, 0, yet.n_trials + 1)
    finally:
        are.are_free_yet(ctx, h)
