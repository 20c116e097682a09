"""The pricing server (continuous batching) through the C ABI: results
against the oracle, the same alone and in a mix, memory-based admission,
one-at-a-time mode, bounded waits, cancellation, a full queue and argument
errors.  Faults are injected on the host only (a stalled scheduler, a
cancelled request); nothing here makes the GPU fault or hang."""
import math
import time

import numpy as np
import pytest

import workloads as W
from gpu_support import rel_close

pytestmark = pytest.mark.gpu
N_TRIALS, K, CATALOG = 20_000, 100, 20_000
RPS, LEVELS = (100.0, 250.0, 20.0), (0.99, 0.9)


@pytest.fixture(scope="module")
def are():
    import torch
    assert torch.cuda.is_available()
    import paper_1308_2066_gb300 as are
    are.lib()
    return are


@pytest.fixture(scope="module")
def pool():
    g = np.random.Generator(np.random.PCG64(44))
    yet = W.yet_fixed(g, N_TRIALS, K, CATALOG, timestamps=False)
    elts = [W.percentile_terms(W.elt_lognormal(g, CATALOG, int(g.integers(300, 1500))))
            for _ in range(24)]
    return yet, elts


@pytest.fixture()
def served(are, pool):
    """A context with the pool loaded; yields (ctx, yet handle, elt handles)."""
    yet, elts = pool
    ctx = are.are_create(0)
    y = are.are_load_yet(ctx, CATALOG, N_TRIALS, None, K, yet.ids)
    hs = [are.are_load_elt(ctx, e.ids, e.losses, e.fx, e.ded, e.lim, e.share) for e in elts]
    yield ctx, y, hs
    are.are_destroy(ctx)


def requests(seed, n, max_j=16):
    g = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        j = int(g.integers(1, max_j + 1))
        members = [int(x) for x in g.choice(24, j, replace=False)]
        occ_r = float(g.uniform(1e4, 1e5))
        out.append(dict(members=members, occ_r=occ_r, occ_l=occ_r * float(g.uniform(5, 50)),
                        agg_r=occ_r * float(g.uniform(1, 4)),
                        agg_l=float(g.choice([math.inf, occ_r * 200])),
                        n_trials=int(g.integers(500, N_TRIALS + 1))))
    return out


def submit(are, ctx, hs, r):
    return are.are_submit(ctx, [hs[m] for m in r["members"]], r["occ_r"], r["occ_l"], r["agg_r"],
                          r["agg_l"], r["n_trials"], RPS, LEVELS)


def oracle_measures(orc, pool, r):
    yet, elts = pool
    wl = W.Workload("req", yet, elts, [W.Layer(r["members"], r["occ_r"], r["occ_l"], r["agg_r"],
                                               r["agg_l"])])
    res = orc.simulate_layer(wl, trials=np.arange(r["n_trials"]))
    return orc.risk_measures(res.ylt, RPS, LEVELS)


def test_results_match_oracle_in_a_mix(are, orc, pool, served):
    ctx, y, hs = served
    are.are_server_start(ctx, y, max_inflight=8, events_per_launch=3_000_000)
    reqs = requests(1, 30)
    tickets = [submit(are, ctx, hs, r) for r in reqs]
    for r, t in zip(reqs, tickets):
        res = are.are_wait(ctx, t, 60_000_000)
        assert res["status"] == are.ARE_OK and res["n_trials"] == r["n_trials"]
        pml, tv = oracle_measures(orc, pool, r)
        assert rel_close(res["pml"], pml, 1e-5), (res["pml"], pml)
        assert rel_close(res["tvar"], tv, 1e-5), (res["tvar"], tv)
        assert res["total_us"] >= res["run_us"] >= 0 and res["queue_us"] >= 0
    are.are_server_stop(ctx)


def test_same_result_alone_and_in_the_mix(are, served):
    ctx, y, hs = served
    probe = requests(7, 1)[0]
    are.are_server_start(ctx, y, max_inflight=1)
    alone = are.are_wait(ctx, submit(are, ctx, hs, probe), 60_000_000)
    are.are_server_stop(ctx)
    # many small launches, the probe surrounded by other requests
    are.are_server_start(ctx, y, max_inflight=16, events_per_launch=400_000, trials_per_item=4)
    others = requests(8, 40)
    tickets = [submit(are, ctx, hs, r) for r in others[:20]]
    tp = submit(are, ctx, hs, probe)
    tickets += [submit(are, ctx, hs, r) for r in others[20:]]
    mixed = are.are_wait(ctx, tp, 60_000_000)
    for t in tickets:
        assert are.are_wait(ctx, t, 60_000_000)["status"] == are.ARE_OK
    are.are_server_stop(ctx)
    assert alone["pml"] == mixed["pml"] and alone["tvar"] == mixed["tvar"]
    # and the same again when every request runs alone, whole, in order
    are.are_server_start(ctx, y, max_inflight=4, one_at_a_time=True)
    seq = are.are_wait(ctx, submit(are, ctx, hs, probe), 60_000_000)
    are.are_server_stop(ctx)
    assert seq["pml"] == alone["pml"] and seq["tvar"] == alone["tvar"]


@pytest.fixture(scope="module")
def long_yet(are, pool):
    """A 1M x 200 YET over the pool's catalog, for requests of 2e8 events."""
    g = np.random.Generator(np.random.PCG64(46))
    return W.yet_fixed(g, 1_000_000, 200, CATALOG, timestamps=False)


@pytest.mark.parametrize("least_work_first", [False, True])
def test_budget_order(are, pool, long_yet, least_work_first):
    """Each launch's event budget goes to the admitted requests in arrival
    order, or with least_work_first to the least remaining work first (less
    the time waited).  A large request (2e8 events, ten launches' budget)
    submitted just before small ones: in arrival order the small ones wait
    for its last slice; least work first they finish long before it."""
    import torch
    _, elts = pool
    ctx = are.are_create(0)
    try:
        y = are.are_load_yet(ctx, CATALOG, long_yet.n_trials, None, long_yet.k,
                             torch.from_numpy(long_yet.ids).cuda())
        hs = [are.are_load_elt(ctx, e.ids, e.losses, e.fx, e.ded, e.lim, e.share) for e in elts[:8]]
        are.are_server_start(ctx, y, max_inflight=8, events_per_launch=20_000_000,
                             least_work_first=least_work_first)
        big = dict(members=[0, 1, 2], occ_r=1e4, occ_l=1e6, agg_r=0.0, agg_l=math.inf,
                   n_trials=long_yet.n_trials)
        small = [dict(big, members=[3 + i], n_trials=200) for i in range(4)]
        tb = submit(are, ctx, hs, big)
        ts = [submit(are, ctx, hs, r) for r in small]
        rb = are.are_wait(ctx, tb, 60_000_000)
        rs = [are.are_wait(ctx, t, 60_000_000) for t in ts]
        are.are_server_stop(ctx)
        assert rb["status"] == are.ARE_OK and all(r["status"] == are.ARE_OK for r in rs)
        if least_work_first:
            assert max(r["total_us"] for r in rs) < 0.5 * rb["total_us"], (rb, rs)
        else:
            assert min(r["total_us"] for r in rs) > 0.5 * rb["total_us"], (rb, rs)
    finally:
        are.are_destroy(ctx)


def test_admission_by_memory(are, served):
    ctx, y, hs = served
    table16 = CATALOG * 16 * 4
    # room for one 16-wide table and its YLT at a time
    are.are_server_start(ctx, y, max_inflight=8, arena_bytes=table16 + 8 * N_TRIALS + 4096)
    reqs = [dict(r, members=r["members"][:16]) for r in requests(3, 6)]
    tickets = [submit(are, ctx, hs, r) for r in reqs]
    out = [are.are_wait(ctx, t, 60_000_000) for t in tickets]
    assert all(o["status"] == are.ARE_OK for o in out)
    are.are_server_stop(ctx)


def test_bounded_wait_cancel_and_full_queue(are, served):
    ctx, y, hs = served
    are.are_server_start(ctx, y, max_inflight=2, max_pending=3, stall_us=300_000)
    r = requests(5, 6)
    t0 = submit(are, ctx, hs, r[0])
    with pytest.raises(are.AreError) as e:
        are.are_wait(ctx, t0, 1000)                     # the scheduler stalls: times out
    assert e.value.status == are.ARE_ETIMEOUT
    t1, t2, t3 = (submit(are, ctx, hs, x) for x in r[1:4])
    busy = None
    for x in r[4:]:
        try:
            submit(are, ctx, hs, x)
        except are.AreError as err:
            busy = err
    assert busy is not None and busy.status == are.ARE_EBUSY
    are.are_cancel(ctx, t3)
    with pytest.raises(are.AreError) as e:
        are.are_wait(ctx, t3, 0)
    assert e.value.status == are.ARE_ENOTFOUND
    for t in (t0, t1, t2):
        assert are.are_wait(ctx, t, 120_000_000)["status"] == are.ARE_OK
    with pytest.raises(are.AreError):
        are.are_wait(ctx, t0, 0)                        # a result is handed over once
    are.are_server_stop(ctx)


def test_server_argument_errors(are, served):
    ctx, y, hs = served
    with pytest.raises(are.AreError):
        are.are_submit(ctx, [hs[0]], 0, 1, 0, 1, 10)   # no server yet
    are.are_server_start(ctx, y, max_inflight=2)
    with pytest.raises(are.AreError) as e:
        are.are_server_start(ctx, y)
    assert e.value.status == are.ARE_EBUSY
    for bad in (dict(elts=[hs[0]], n=N_TRIALS + 1), dict(elts=[hs[0], hs[0]], n=10),
                dict(elts=[999999], n=10)):
        with pytest.raises(are.AreError):
            are.are_submit(ctx, bad["elts"], 0, math.inf, 0, math.inf, bad["n"])
    with pytest.raises(are.AreError):
        are.are_submit(ctx, [hs[0]], 0, 1, 0, 1, 10, [2.0] * 5, [0.5] * 4)
    with pytest.raises(are.AreError) as e:
        are.are_free_yet(ctx, y)
    assert e.value.status == are.ARE_EBUSY
    t = are.are_submit(ctx, [hs[1]], 0, math.inf, 0, math.inf, 5000)
    assert are.are_wait(ctx, t, 60_000_000)["status"] == are.ARE_OK
    are.are_server_stop(ctx)
    are.are_free_yet(ctx, y)


def test_stop_drops_queued_requests(are, served):
    ctx, y, hs = served
    are.are_server_start(ctx, y, max_inflight=1, stall_us=200_000)
    tickets = [submit(are, ctx, hs, r) for r in requests(9, 5)]
    time.sleep(0.05)
    are.are_server_stop(ctx)           # finishes what was admitted, drops the queue
    are.are_server_start(ctx, y, max_inflight=2)
    with pytest.raises(are.AreError) as e:
        are.are_wait(ctx, tickets[-1], 0)
    assert e.value.status == are.ARE_ENOTFOUND
    are.are_server_stop(ctx)


@pytest.mark.parametrize("members", [[3, 1, 4, 0, 5, 9, 2, 6], [7, 3, 11, 1, 4, 0, 10, 5, 9, 2, 8, 6]],
                         ids=["j8_dense_rows", "j12_packed_rows"])
def test_large_request_on_the_single_layer_kernel(are, members):
    """A request of at least 32M events runs its slices on the single-layer
    register-rows kernel (over packed rows for the 12-ELT layer, whose ELTs
    hold few entries per catalog event): its result equals are_simulate +
    are_risk_measures on the same layer (the same kernel, rows and
    arithmetic per trial), alone and in a mix of small requests, whole
    (arrival order) or sliced into many launches (least work first)."""
    import torch
    g = np.random.Generator(np.random.PCG64(45))
    n, k, C = 80_000, 500, 20_000
    yet = W.yet_fixed(g, n, k, C, timestamps=False)
    elts = [W.percentile_terms(W.elt_lognormal(g, C, int(g.integers(300, 1500)))) for _ in range(12)]
    ctx = are.are_create(0)
    try:
        y = are.are_load_yet(ctx, C, n, None, k, torch.from_numpy(yet.ids).cuda())
        hs = [are.are_load_elt(ctx, e.ids, e.losses, e.fx, e.ded, e.lim, e.share) for e in elts]
        terms = (2e4, 1e6, 5e4, 5e7)
        layer = are.are_define_layer(ctx, [hs[m] for m in members], *terms)
        assert are.are_layer_rows(ctx, layer, y, are.ARE_FP32_KAHAN)[1] == (len(members) > 8)
        out = torch.empty(n, dtype=torch.float64, device="cuda")
        are.are_simulate(ctx, layer, y, 0, n, are.ARE_FP32_KAHAN, out)
        pml, tv = are.are_risk_measures(ctx, out, n, RPS, LEVELS)

        def big():
            return are.are_submit(ctx, [hs[m] for m in members], *terms, n, RPS, LEVELS)

        small = [dict(members=[int(x) for x in g.choice(12, int(g.integers(1, 9)), replace=False)],
                      n=int(g.integers(1000, 20_000))) for _ in range(12)]
        for mix, lwf in ((False, False), (True, False), (True, True)):
            are.are_server_start(ctx, y, max_inflight=16, events_per_launch=10_000_000,
                                 least_work_first=lwf)
            tickets = []
            if mix:
                tickets += [are.are_submit(ctx, [hs[m] for m in r["members"]], 1e4, 1e6, 0, math.inf,
                                           r["n"], RPS, LEVELS) for r in small[:6]]
            tb = big()
            if mix:
                tickets += [are.are_submit(ctx, [hs[m] for m in r["members"]], 1e4, 1e6, 0, math.inf,
                                           r["n"], RPS, LEVELS) for r in small[6:]]
            res = are.are_wait(ctx, tb, 120_000_000)
            for t in tickets:
                assert are.are_wait(ctx, t, 120_000_000)["status"] == are.ARE_OK
            are.are_server_stop(ctx)
            assert res["status"] == are.ARE_OK
            assert list(res["pml"]) == list(pml) and list(res["tvar"]) == list(tv), (mix, res, pml, tv)
    finally:
        are.are_destroy(ctx)


def test_folded_server_matches_oracle_alone_and_in_a_mix(are, orc, pool, served):
    """Folded tables in the server: FP64 occurrence losses and exact trial
    sums, so PML/TVaR agree with the oracle within the FP64 tolerance and a
    request's result is identical alone and in a mix."""
    ctx, y, hs = served
    reqs = requests(11, 24)
    are.are_server_start(ctx, y, max_inflight=8, events_per_launch=500_000, folded=True)
    tickets = [submit(are, ctx, hs, r) for r in reqs]
    mixed = [are.are_wait(ctx, t, 60_000_000) for t in tickets]
    are.are_server_stop(ctx)
    for r, res in zip(reqs, mixed):
        assert res["status"] == are.ARE_OK
        pml, tv = oracle_measures(orc, pool, r)
        assert rel_close(res["pml"], pml, 1e-12), (res["pml"], pml)
        assert rel_close(res["tvar"], tv, 1e-12), (res["tvar"], tv)
    are.are_server_start(ctx, y, max_inflight=1, folded=True)
    for r, res in zip(reqs[:5], mixed[:5]):
        alone = are.are_wait(ctx, submit(are, ctx, hs, r), 60_000_000)
        assert alone["pml"] == res["pml"] and alone["tvar"] == res["tvar"]
    are.are_server_stop(ctx)
