"""Pins for the FP64 CPU oracle: hand-worked cases, closed forms, invariants,
exact rational arithmetic and library special cases.  None of these recompute
the oracle's own loop; each checks it against something the paper or the
mathematics fixes (the algorithm of Section II-B, Table I's terms)."""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import workloads as W

INF = float("inf")


def _f(v):
    return INF if v == "inf" else float(v)


def run_tiny(orc, elts, terms, trials, marginals=False):
    """elts: list of dicts with ids, losses, fx, ded, lim, share; terms: 4-tuple;
    trials: list of event-id lists.  Returns the oracle's TrialResult."""
    counts = [len(t) for t in trials]
    off = np.zeros(len(trials) + 1, np.int64)
    off[1:] = np.cumsum(counts)
    ids = np.array([e for t in trials for e in t], dtype=np.int32)
    eo = np.zeros(len(elts) + 1, np.int32)
    eo[1:] = np.cumsum([len(e["ids"]) for e in elts])
    ei = np.array([i for e in elts for i in e["ids"]], dtype=np.int32)
    el = np.array([x for e in elts for x in e["losses"]], dtype=np.float64)
    fx = np.array([_f(e.get("fx", 1.0)) for e in elts])
    ded = np.array([_f(e.get("ded", 0.0)) for e in elts])
    lim = np.array([_f(e.get("lim", INF)) for e in elts])
    sh = np.array([_f(e.get("share", 1.0)) for e in elts])
    return orc.simulate(ids, len(trials), off, None, eo, ei, el, fx, ded, lim, sh,
                        *[_f(t) for t in terms], marginals=marginals)


def golden_layer(golden, name):
    L = golden["layers"][name]
    return L["elts"], (L["occ_r"], L["occ_l"], L["agg_r"], L["agg_l"])


# ---------------------------------------------------------------------------
# hand-worked cases (tests/golden/hand_cases.json)
# ---------------------------------------------------------------------------

def test_hand_cases(orc, golden):
    for case in golden["trials"]:
        elts, terms = golden_layer(golden, case["layer"])
        r = run_tiny(orc, elts, terms, [case["events"]], marginals=True)
        assert r.ylt[0] == case["ylt"], case
        assert r.s_total[0] == case["s_total"], case
        assert r.gross[0] == case["gross"], case
        assert r.n_events[0] == len(case["events"])
        assert list(r.marginals) == case["marginals"], case
        assert r.lr_literal[0] == case["ylt"]


def test_hand_cases_batched_equal_single(orc, golden):
    elts, terms = golden_layer(golden, "two_elts")
    cases = [c for c in golden["trials"] if c["layer"] == "two_elts"]
    r = run_tiny(orc, elts, terms, [c["events"] for c in cases])
    assert list(r.ylt) == [c["ylt"] for c in cases]


def test_hand_risk_measures(orc, golden):
    for case in golden["risk_measures"]:
        pml, tv = orc.risk_measures(np.array(case["ylt"]), case["return_periods"], case["levels"])
        assert list(pml) == case["pml"]
        assert list(tv) == case["tvar"]


def test_rank_definitions(orc, golden):
    for c in golden["ranks"]["cases"]:
        assert orc.rank_for_return_period(c["n"], c["rp"]) == c["m"], c
    for c in golden["ranks"]["level_cases"]:
        assert orc.rank_for_level(c["n"], c["a"]) == c["m"], c
    # a naive ceil(1e6 * (1 - 0.99)) would give 10001
    assert math.ceil(1_000_000 * (1 - 0.99)) == 10001
    assert orc.rank_for_level(1_000_000, 0.99) == 10000


def test_invalid_risk_arguments(orc):
    with pytest.raises(ValueError):
        orc.risk_measures(np.array([1.0, 2.0]), [0.5], [])
    with pytest.raises(ValueError):
        orc.risk_measures(np.array([1.0, 2.0]), [], [1.0])
    with pytest.raises(ValueError):
        orc.risk_measures(np.zeros(0), [2.0], [])


def test_duplicate_ids_in_elt_rejected(orc):
    with pytest.raises(ValueError):
        run_tiny(orc, [{"ids": [1, 1], "losses": [1.0, 2.0]}], (0, INF, 0, INF), [[1]])


# ---------------------------------------------------------------------------
# closed forms and special cases
# ---------------------------------------------------------------------------

def small_workload(seed, n_trials=200, k=30, catalog=300, n_elts=3, nnz=60, ragged=False):
    g = np.random.Generator(np.random.PCG64(seed))
    if ragged:
        yet = W.yet_poisson(g, n_trials, k, catalog, timestamps=False)
    else:
        yet = W.yet_fixed(g, n_trials, k, catalog, timestamps=False)
    elts = [W.percentile_terms(W.elt_lognormal(g, catalog, nnz)) for _ in range(n_elts)]
    return yet, elts, g


def dense_losses(elts, catalog):
    """Catalog-length loss vector per ELT (zeros where the ELT has no entry)."""
    out = np.zeros((len(elts), catalog))
    for j, e in enumerate(elts):
        out[j, e.ids] = e.losses
    return out


def sim(orc, yet, elts, layer, **kw):
    eo, ei, el, fx, ded, lim, sh = W.layer_arrays(elts, layer)
    return orc.simulate(yet.ids, yet.n_trials, yet.offsets, yet.k, eo, ei, el, fx, ded, lim, sh,
                        layer.occ_r, layer.occ_l, layer.agg_r, layer.agg_l, **kw)


@pytest.mark.parametrize("ragged", [False, True])
def test_neutral_terms_give_plain_sums(orc, ragged):
    """Zero retentions/deductibles and infinite limits: trial loss is the plain
    sum of the trial's looked-up losses over all of the layer's ELTs."""
    yet, elts, _ = small_workload(1, ragged=ragged)
    for e in elts:
        e.ded, e.lim = 0.0, INF
    layer = W.Layer(elts=[0, 1, 2])
    r = sim(orc, yet, elts, layer)
    dense = dense_losses(elts, yet.catalog).sum(axis=0)
    expect = np.array([math.fsum(dense[yet.trial(i)]) for i in range(yet.n_trials)])
    assert np.all(r.ylt > 0)
    np.testing.assert_allclose(r.ylt, expect, rtol=1e-13, atol=0)
    np.testing.assert_allclose(r.gross, expect, rtol=1e-13, atol=0)
    np.testing.assert_array_equal(r.n_events, yet.counts())


def test_single_event_trials_closed_form(orc):
    """One event per trial: the loss is the event's terms stacked once each,
    clamp_agg(clamp_occ(sum_j f_j(x_j)))."""
    yet, elts, g = small_workload(2, n_trials=300, k=1, catalog=100, nnz=40)
    for j, e in enumerate(elts):
        e.fx = [1.0, 1.25, 0.8][j]
        e.share = [1.0, 0.5, 0.75][j]
    layer = W.Layer(elts=[0, 1, 2], occ_r=5e4, occ_l=8e5, agg_r=2e4, agg_l=6e5)
    r = sim(orc, yet, elts, layer)
    dense = dense_losses(elts, yet.catalog)
    for i in range(yet.n_trials):
        e = yet.ids[i]
        g_ = 0.0
        for j, el in enumerate(elts):
            v = el.fx * dense[j, e] - el.ded
            v = min(max(v, 0.0), el.lim) * el.share
            g_ += v
        o = min(max(g_ - layer.occ_r, 0.0), layer.occ_l)
        y = min(max(o - layer.agg_r, 0.0), layer.agg_l)
        assert r.ylt[i] == y
        assert r.s_total[i] == o


def test_all_zero_elts_give_zero(orc):
    yet, elts, _ = small_workload(3)
    for e in elts:
        e.losses = np.zeros_like(e.losses)
    r = sim(orc, yet, elts, W.Layer(elts=[0, 1, 2]))
    assert np.all(r.ylt == 0) and np.all(r.s_total == 0)


def test_empty_layer_and_empty_trials(orc):
    r = run_tiny(orc, [], (0, INF, 0, INF), [[1, 2, 3], []])
    assert list(r.ylt) == [0.0, 0.0]
    r = run_tiny(orc, [{"ids": [1], "losses": [5.0]}], (0, INF, 0, INF), [[], [], [1]])
    assert list(r.ylt) == [0.0, 0.0, 5.0]


# ---------------------------------------------------------------------------
# exact rational arithmetic on tiny inputs
# ---------------------------------------------------------------------------

def exact_trial(events, elts, terms):
    """The definitions in exact rationals: lookup, terms, occurrence clamp,
    cumulative sum, aggregate clamp, marginals."""
    def clamp(v, r, l):
        v = v - r
        v = v if v > 0 else Fraction(0)
        return v if l is None or v < l else l
    occ_r, occ_l, agg_r, agg_l = terms
    occ = []
    for e in events:
        g = Fraction(0)
        for el in elts:
            x = Fraction(dict(zip(el["ids"], el["losses"])).get(e, 0.0))
            lim = None if el["lim"] == INF else Fraction(el["lim"])
            g += Fraction(el["share"]) * clamp(Fraction(el["fx"]) * x, Fraction(el["ded"]), lim)
        occ.append(clamp(g, Fraction(occ_r), None if occ_l == INF else Fraction(occ_l)))
    cum = list(itertools.accumulate(occ)) if occ else []
    agg = [clamp(s, Fraction(agg_r), None if agg_l == INF else Fraction(agg_l)) for s in cum]
    marg = [a - b for a, b in zip(agg, [Fraction(0)] + agg[:-1])]
    return (agg[-1] if agg else Fraction(0)), (cum[-1] if cum else Fraction(0)), marg


@pytest.mark.parametrize("seed", range(12))
def test_brute_force_exact_rationals(orc, seed):
    """Tiny random layers (<= 8 trials x <= 6 events, J <= 3): the FP64 oracle
    lies within a few rounding errors of the exact rational result, and the
    exact marginals telescope to the exact trial loss."""
    g = np.random.Generator(np.random.PCG64(100 + seed))
    catalog = 8
    J = int(g.integers(1, 4))
    elts = []
    for _ in range(J):
        nnz = int(g.integers(0, catalog + 1))
        elts.append({"ids": [int(i) for i in g.choice(catalog, nnz, replace=False)],
                     "losses": [float(np.round(g.lognormal(5, 1.5), 3)) for _ in range(nnz)],
                     "fx": float(g.choice([1.0, 0.5, 1.1])), "ded": float(np.round(g.uniform(0, 80), 2)),
                     "lim": float(g.choice([INF, np.round(g.uniform(50, 900), 2)])),
                     "share": float(g.choice([1.0, 0.25, 0.6]))})
    terms = (float(np.round(g.uniform(0, 200), 1)), float(g.choice([INF, 700.0])),
             float(np.round(g.uniform(0, 400), 1)), float(g.choice([INF, 1500.0])))
    trials = [[int(e) for e in g.integers(0, catalog, int(g.integers(0, 7)))]
              for _ in range(int(g.integers(1, 9)))]
    r = run_tiny(orc, elts, terms, trials, marginals=True)
    pos = 0
    for i, t in enumerate(trials):
        y, s, marg = exact_trial(t, elts, terms)
        assert sum(marg, Fraction(0)) == y
        scale = float(sum(Fraction(e["fx"]) * Fraction(x) for e in elts for x in e["losses"])) * 4 + 1e4
        tol = 64 * 2.0 ** -52 * scale
        assert abs(r.ylt[i] - float(y)) <= tol, (i, r.ylt[i], float(y))
        assert abs(r.s_total[i] - float(s)) <= tol
        for d in range(len(t)):
            assert abs(r.marginals[pos + d] - float(marg[d])) <= tol
        pos += len(t)


# ---------------------------------------------------------------------------
# invariants
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def base_case():
    yet, elts, _ = small_workload(7, n_trials=400, k=20, catalog=400, n_elts=4, nnz=30)
    layer = W.Layer(elts=[0, 1, 2, 3], occ_r=3e4, occ_l=9e5, agg_r=4e5, agg_l=1e6)
    return yet, elts, layer


def test_bounds(orc, base_case):
    yet, elts, layer = base_case
    r = sim(orc, yet, elts, layer)
    assert np.all(r.ylt >= 0) and np.all(r.ylt <= layer.agg_l)
    assert 0 < np.mean(r.ylt == layer.agg_l) < 1 and 0 < np.mean(r.ylt == 0) < 1
    assert np.all(r.ylt <= r.s_total) and np.all(r.s_total <= r.gross)
    np.testing.assert_allclose(r.lr_literal, r.ylt, rtol=1e-12, atol=1e-6)


def _with(elts, j, **kw):
    out = [W.ELT(e.ids, e.losses.copy(), e.ded, e.lim, e.fx, e.share) for e in elts]
    for k, v in kw.items():
        setattr(out[j], k, v)
    return out


def test_monotone_in_losses_and_limits(orc, base_case):
    yet, elts, layer = base_case
    y0 = sim(orc, yet, elts, layer).ylt
    up = _with(elts, 1, losses=elts[1].losses * 1.7)
    assert np.all(sim(orc, yet, up, layer).ylt >= y0)
    assert np.any(sim(orc, yet, up, layer).ylt > y0)
    assert np.all(sim(orc, yet, _with(elts, 2, lim=elts[2].lim * 3), layer).ylt >= y0)
    for name in ("occ_l", "agg_l"):
        L2 = W.Layer(layer.elts, layer.occ_r, layer.occ_l, layer.agg_r, layer.agg_l)
        setattr(L2, name, getattr(layer, name) * 2)
        y = sim(orc, yet, elts, L2).ylt
        assert np.all(y >= y0) and np.any(y > y0), name


def test_non_increasing_in_retentions(orc, base_case):
    yet, elts, layer = base_case
    y0 = sim(orc, yet, elts, layer).ylt
    y = sim(orc, yet, _with(elts, 0, ded=elts[0].ded * 5), layer).ylt
    assert np.all(y <= y0) and np.any(y < y0)
    for name in ("occ_r", "agg_r"):
        L2 = W.Layer(layer.elts, layer.occ_r, layer.occ_l, layer.agg_r, layer.agg_l)
        setattr(L2, name, getattr(layer, name) * 2 + 1)
        y = sim(orc, yet, elts, L2).ylt
        assert np.all(y <= y0) and np.any(y < y0), name


def test_trials_independent_range_split(orc, base_case):
    yet, elts, layer = base_case
    y0 = sim(orc, yet, elts, layer).ylt
    parts = [sim(orc, yet, elts, layer, trials=np.arange(a, b)).ylt
             for a, b in ((0, 137), (137, 138), (138, 400))]
    np.testing.assert_array_equal(np.concatenate(parts), y0)
    perm = np.random.default_rng(0).permutation(400)
    np.testing.assert_array_equal(sim(orc, yet, elts, layer, trials=perm).ylt, y0[perm])


def test_event_order_changes_marginals_not_trial_loss(orc, base_case):
    yet, elts, layer = base_case
    r0 = sim(orc, yet, elts, layer, marginals=True)
    g = np.random.default_rng(5)
    ids = yet.ids.copy().reshape(yet.n_trials, yet.k)
    for row in ids:
        g.shuffle(row)
    y2 = W.YET(yet.catalog, yet.n_trials, ids.reshape(-1), k=yet.k)
    r1 = sim(orc, y2, elts, layer, marginals=True)
    np.testing.assert_allclose(r1.ylt, r0.ylt, rtol=0, atol=1e-13 * r0.gross.max())
    assert not np.allclose(r1.marginals, r0.marginals)


def test_duplicated_event_adds_its_occurrence_loss(orc, base_case):
    """With neutral aggregate terms the trial loss is S_k; appending a copy of
    event e adds exactly the single-event occurrence loss of e."""
    yet, elts, layer = base_case
    L2 = W.Layer(layer.elts, layer.occ_r, layer.occ_l, 0.0, INF)
    base = sim(orc, yet, elts, L2).ylt
    ids = yet.ids.reshape(yet.n_trials, yet.k)
    extra = ids[:, 3]
    dup = W.YET(yet.catalog, yet.n_trials, np.concatenate([ids, extra[:, None]], axis=1).reshape(-1),
                k=yet.k + 1)
    single = W.YET(yet.catalog, yet.n_trials, extra.copy(), k=1)
    o = sim(orc, single, elts, L2).ylt
    np.testing.assert_allclose(sim(orc, dup, elts, L2).ylt, base + o, rtol=1e-14, atol=0)


def test_threads_do_not_change_results(orc, base_case):
    yet, elts, layer = base_case
    a = sim(orc, yet, elts, layer, threads=1)
    b = sim(orc, yet, elts, layer, threads=4)
    np.testing.assert_array_equal(a.ylt, b.ylt)
    np.testing.assert_array_equal(a.s_total, b.s_total)


# ---------------------------------------------------------------------------
# PML / TVaR against library sorting
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 7, 100, 999, 10_000, 123_457])
def test_risk_measures_vs_numpy(orc, n):
    g = np.random.default_rng(n)
    y = np.round(g.lognormal(12, 2, n), 2)
    y[g.random(n) < 0.3] = 0.0
    rps = [1.0, 2.0, 10.0, 100.0, 250.0, 1000.0]
    lv = [0.5, 0.9, 0.99, 0.995]
    pml, tv = orc.risk_measures(y, rps, lv)
    desc = np.sort(y)[::-1]
    for i, rp in enumerate(rps):
        m = min(n, max(1, math.ceil(Fraction(n) / Fraction(rp))))
        assert pml[i] == desc[m - 1]
    for i, a in enumerate(lv):
        m = max(1, math.ceil(Fraction(n) * (1 - Fraction(str(a)))))
        assert tv[i] == pytest.approx(math.fsum(desc[:m]) / m, rel=1e-13)
        assert np.partition(y, n - m)[n - m] == desc[m - 1]
    assert np.all(np.diff(pml) >= 0)          # non-decreasing in RP
    for i, a in enumerate(lv):                # PML at the same rank <= TVaR <= max
        m = orc.rank_for_level(n, a)
        assert desc[m - 1] <= tv[i] <= desc[0]


def test_risk_measures_with_ties(orc):
    y = np.array([3.0] * 50 + [1.0] * 50)
    pml, tv = orc.risk_measures(y, [2.0, 1.0], [0.3])
    assert list(pml) == [3.0, 1.0]
    assert tv[0] == pytest.approx((50 * 3 + 20 * 1) / 70)


# ---------------------------------------------------------------------------
# tiny workload recipe sanity
# ---------------------------------------------------------------------------

def test_tiny_workload_shape(orc):
    w = W.plain_tiny()
    y = w.yet
    assert y.n_trials == 10_000 and y.k == 100 and y.ids.min() >= 0 and y.ids.max() < 10_000
    assert np.all(np.diff(y.timestamps.reshape(10_000, 100), axis=1) >= 0)
    assert [len(e.ids) for e in w.elts] == [2000] * 4
    for e in w.elts:
        assert len(np.unique(e.ids)) == 2000
        s = np.sort(e.losses)
        assert e.ded == s[199] and e.lim == s[1979]
    r = orc.simulate_layer(w)
    assert np.all(r.ylt <= 1e7)
