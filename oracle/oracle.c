/*
 * oracle.c -- plain, slow, FP64 CPU oracle for aggregate risk analysis.
 *
 * TEST INFRASTRUCTURE.  This file is the yardstick the GPU library is checked
 * against.  Only the tests, the smoke check and the benchmark's CPU-baseline
 * leg load it; the library never does.  It shares no code, header, table or
 * constant with the GPU library.
 *
 * Source: A. Bahl, O. Baltzer, A. Rau-Chaplin, B. Varghese, "Parallel
 * Simulations for Analysing Portfolios of Catastrophic Event Risk",
 * arXiv 1308.2066.  Section II-A defines the inputs (YET, ELT, layer), the
 * "Basic Algorithm for Aggregate Risk Analysis" box of Section II-B gives the
 * analysis stage, Table I the four layer terms, Section II-C the output.
 *
 * What it computes, for one layer and each trial with events e_1..e_k in
 * stored order (written from the definitions of Sections II-A to II-C):
 *   - an event's loss in ELT j is its entry there (0 if the ELT has none),
 *     looked up by binary search in a sorted private copy of the ELT, not
 *     through a direct-access table;
 *   - its loss net of ELT j's financial terms is
 *     f_j(x) = share_j * min(max(fx_j * x - D_j, 0), Lim_j);
 *   - the event loss g_d is the sum of f_j over the layer's ELTs, added in
 *     layer order;
 *   - the occurrence loss is o_d = min(max(g_d - OccR, 0), OccL) (Table I);
 *   - the running total S_d = o_1 + ... + o_d, its aggregate-clamped value
 *     A_d = min(max(S_d - AggR, 0), AggL) (Table I), and the marginal
 *     m_d = A_d - A_{d-1} with A_0 = 0;
 *   - the trial loss A_k, beside S_k and the literal sum of the marginals.
 * Each trial is one pass over its occurrences in stored order.
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - the financial terms I of an ELT are (fx, D, Lim, share) applied as
 *     f_j above;
 *   - the marginal of an occurrence is taken between the clamped running
 *     totals A_d and A_{d-1} (the de-cumulation of the paper's step 4 read
 *     with the clamped cumulative values), with A_0 = 0;
 *   - the trial loss written to the YLT is A_k; because every o_d >= 0 the
 *     marginals telescope and their literal sum equals A_k up to rounding;
 *     it is returned beside A_k as a self-check;
 *   - a trial with no events has loss 0;
 *   - PML at return period RP is the m-th largest trial loss with
 *     m = ceil(N / RP); TVaR at level a is the mean of the m largest trial
 *     losses with m = ceil(N * (1 - a)); RP is read to the nearest 1e-6 and a
 *     to the nearest 1e-9 so that m is an exact integer.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fopenmp -fPIC -shared.
 * -ffp-contract=off keeps fx*x - D as a rounded product then a rounded
 * difference on every host.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_EINVAL (-1)
#define OR_ENOMEM (-2)
#define OR_EDUP (-3)

/* ------------------------------------------------------------------------ */
/* ELT: a dictionary from event id to loss (Section II-A, item 2).           */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t id;
    double loss;
} or_pair;

typedef struct {
    int32_t n;
    or_pair *p; /* sorted by id */
} or_dict;

static int cmp_pair(const void *a, const void *b)
{
    const or_pair *x = (const or_pair *)a, *y = (const or_pair *)b;
    return (x->id > y->id) - (x->id < y->id);
}

static int dict_build(or_dict *t, int32_t n, const int32_t *ids, const double *loss)
{
    t->n = n;
    t->p = (or_pair *)malloc(sizeof(or_pair) * (size_t)(n > 0 ? n : 1));
    if (!t->p)
        return OR_ENOMEM;
    for (int32_t i = 0; i < n; ++i) {
        t->p[i].id = ids[i];
        t->p[i].loss = loss[i];
    }
    qsort(t->p, (size_t)n, sizeof(or_pair), cmp_pair);
    for (int32_t i = 1; i < n; ++i)
        if (t->p[i].id == t->p[i - 1].id)
            return OR_EDUP;
    return OR_OK;
}

/* x = loss of event e in this ELT, 0 when the ELT has no entry for e. */
static double dict_lookup(const or_dict *t, int32_t e)
{
    int32_t lo = 0, hi = t->n - 1;
    while (lo <= hi) {
        int32_t mid = lo + (hi - lo) / 2;
        int32_t id = t->p[mid].id;
        if (id == e)
            return t->p[mid].loss;
        if (id < e)
            lo = mid + 1;
        else
            hi = mid - 1;
    }
    return 0.0;
}

/* min(max(v - r, 0), l): the shape of every retention/limit pair in Table I. */
static double net_of(double v, double r, double l)
{
    double a = v - r;
    if (!(a > 0.0))
        a = 0.0;
    if (a > l)
        a = l;
    return a;
}

/* ------------------------------------------------------------------------ */
/* Analysis stage for one trial (Section II-B).                              */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t n_elts;
    const or_dict *elt;
    const double *fx, *ded, *lim, *share;
    double occ_r, occ_l, agg_r, agg_l;
} or_layer;

typedef struct {
    double ylt;    /* A_k: trial loss net of all terms */
    double s;      /* S_k: cumulative occurrence loss before aggregate terms */
    double gross;  /* sum over the occurrences and ELTs of fx_j * x (event by event) */
    double lr;     /* literal sum of the marginals m_d */
    double occ_max;/* largest occurrence loss o_d */
} or_trial_out;

/* One trial's occurrences in stored order.  marg: NULL or k doubles. */
static void simulate_trial(const or_layer *L, const int32_t *ev, int64_t k, double *marg,
                           or_trial_out *out)
{
    double gross = 0.0, occ_max = 0.0, lr = 0.0;
    double S = 0.0;     /* running total of the occurrence losses */
    double A = 0.0;     /* its aggregate-clamped value */
    double prev = 0.0;  /* the aggregate-clamped total before this occurrence */
    for (int64_t d = 0; d < k; ++d) {
        /* the event loss: each ELT's entry net of its financial terms,
           added over the ELTs in layer order */
        double g = 0.0;
        for (int32_t j = 0; j < L->n_elts; ++j) {
            const double x = L->elt[j].n ? dict_lookup(&L->elt[j], ev[d]) : 0.0;
            const double conv = L->fx[j] * x;
            gross += conv;
            g += L->share[j] * net_of(conv, L->ded[j], L->lim[j]);
        }
        /* the occurrence loss (occurrence terms of Table I) */
        const double o = net_of(g, L->occ_r, L->occ_l);
        if (o > occ_max)
            occ_max = o;
        /* the running total, its aggregate terms, the marginal */
        S += o;
        A = net_of(S, L->agg_r, L->agg_l);
        const double m = A - prev;
        prev = A;
        if (marg)
            marg[d] = m;
        lr += m;
    }
    out->ylt = A;
    out->s = S;
    out->gross = gross;
    out->lr = lr;
    out->occ_max = occ_max;
}

/*
 * or_simulate -- the analysis stage for one layer over a set of trials.
 *
 * YET: n_trials trials; offsets (n_trials+1 int64, CSR) or NULL with every
 *      trial holding k_fixed events; ids: event ids in stored order.
 * Layer: n_elts ELTs concatenated in layer order, ELT j occupying entries
 *      elt_off[j] .. elt_off[j+1]-1 of elt_ids/elt_loss; per-ELT terms
 *      fx/ded/lim/share[j]; layer terms occ_r, occ_l, agg_r, agg_l.
 * Trials: sel[0..n_sel-1] (trial indices) or NULL for 0..n_trials-1.
 * Outputs (n_sel each, any may be NULL): ylt, s_total, gross, lr_literal,
 *      occ_max, n_events.  marg: NULL, or per-occurrence marginals written at
 *      marg[marg_off[s] + d] for selected trial s.
 * n_threads <= 0 uses the OpenMP default.
 * Returns 0, or OR_EINVAL / OR_ENOMEM / OR_EDUP (duplicate id inside an ELT).
 */
int or_simulate(int64_t n_trials, const int64_t *offsets, int32_t k_fixed,
                const int32_t *ids, int32_t n_elts, const int32_t *elt_off,
                const int32_t *elt_ids, const double *elt_loss, const double *fx,
                const double *ded, const double *lim, const double *share,
                double occ_r, double occ_l, double agg_r, double agg_l,
                int64_t n_sel, const int64_t *sel, double *ylt, double *s_total,
                double *gross, double *lr_literal, double *occ_max,
                int64_t *n_events, double *marg, const int64_t *marg_off,
                int32_t n_threads)
{
    if (n_trials < 0 || n_elts < 0 || (!offsets && k_fixed < 0))
        return OR_EINVAL;
    if (!sel)
        n_sel = n_trials;
    or_dict *dicts = (or_dict *)calloc((size_t)(n_elts > 0 ? n_elts : 1), sizeof(or_dict));
    if (!dicts)
        return OR_ENOMEM;
    int rc = OR_OK;
    for (int32_t j = 0; j < n_elts && rc == OR_OK; ++j)
        rc = dict_build(&dicts[j], elt_off[j + 1] - elt_off[j], elt_ids + elt_off[j],
                        elt_loss + elt_off[j]);
    for (int64_t s = 0; s < n_sel && rc == OR_OK; ++s) {
        int64_t t = sel ? sel[s] : s;
        if (t < 0 || t >= n_trials)
            rc = OR_EINVAL;
    }
    if (rc == OR_OK) {
        or_layer L = {n_elts, dicts, fx, ded, lim, share, occ_r, occ_l, agg_r, agg_l};
#ifdef _OPENMP
        if (n_threads <= 0)
            n_threads = omp_get_max_threads();
#else
        n_threads = 1;
#endif
#pragma omp parallel for num_threads(n_threads) schedule(dynamic, 16)
        for (int64_t s = 0; s < n_sel; ++s) {
            int64_t t = sel ? sel[s] : s;
            int64_t b = offsets ? offsets[t] : t * (int64_t)k_fixed;
            int64_t k = offsets ? offsets[t + 1] - b : k_fixed;
            or_trial_out o;
            simulate_trial(&L, ids + b, k, marg ? marg + marg_off[s] : NULL, &o);
            if (ylt) ylt[s] = o.ylt;
            if (s_total) s_total[s] = o.s;
            if (gross) gross[s] = o.gross;
            if (lr_literal) lr_literal[s] = o.lr;
            if (occ_max) occ_max[s] = o.occ_max;
            if (n_events) n_events[s] = k;
        }
    }
    for (int32_t j = 0; j < n_elts; ++j)
        free(dicts[j].p);
    free(dicts);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Filters on the YLT (Section II-C): PML and TVaR.                          */
/* ------------------------------------------------------------------------ */

static int cmp_desc(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x < y) - (x > y);
}

/* m = ceil(N / RP), RP read to the nearest 1e-6. */
int64_t or_rank_for_return_period(int64_t n, double rp)
{
    int64_t rp_micro = llround(rp * 1e6);
    if (rp_micro < 1000000)
        return -1;
    return (n * 1000000 + rp_micro - 1) / rp_micro;
}

/* m = ceil(N * (1 - a)), a read to the nearest 1e-9. */
int64_t or_rank_for_level(int64_t n, double a)
{
    int64_t a_nano = llround(a * 1e9);
    if (a_nano <= 0 || a_nano >= 1000000000)
        return -1;
    int64_t q = 1000000000 - a_nano;
    return (n * q + 999999999) / 1000000000;
}

/*
 * or_risk_measures -- PML at each return period and TVaR at each level, from
 * a full descending sort of the YLT.  Returns 0 or OR_EINVAL / OR_ENOMEM.
 */
int or_risk_measures(const double *ylt, int64_t n, const double *rps, int32_t n_rp,
                     double *pml, const double *levels, int32_t n_tv, double *tvar)
{
    if (n <= 0)
        return OR_EINVAL;
    double *v = (double *)malloc(sizeof(double) * (size_t)n);
    if (!v)
        return OR_ENOMEM;
    memcpy(v, ylt, sizeof(double) * (size_t)n);
    qsort(v, (size_t)n, sizeof(double), cmp_desc);
    int rc = OR_OK;
    for (int32_t r = 0; r < n_rp; ++r) {
        int64_t m = or_rank_for_return_period(n, rps[r]);
        if (m < 1 || m > n) {
            rc = OR_EINVAL;
            break;
        }
        pml[r] = v[m - 1];
    }
    for (int32_t r = 0; r < n_tv && rc == OR_OK; ++r) {
        int64_t m = or_rank_for_level(n, levels[r]);
        if (m < 1 || m > n) {
            rc = OR_EINVAL;
            break;
        }
        double acc = 0.0;
        for (int64_t i = 0; i < m; ++i)
            acc += v[i];
        tvar[r] = acc / (double)m;
    }
    free(v);
    return rc;
}

int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
