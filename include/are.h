/*
 * are.h -- C ABI of libare, a GB300 (sm_103a) engine for the aggregate risk
 * analysis of Bahl, Baltzer, Rau-Chaplin and Varghese, "Parallel Simulations
 * for Analysing Portfolios of Catastrophic Event Risk" (arXiv 1308.2066).
 *
 * The calls follow the paper's statement of the problem: load a Year Event
 * Table and Event Loss Tables with their financial terms (Section II-A),
 * define layers (Section II-A item 3, Table I), run the analysis stage to a
 * Year Loss Table (Section II-B, Basic Algorithm) and read PML and TVaR from
 * it (Section I and II-C).
 *
 * Conventions shared by every call
 *   - Every call returns an are_status and never aborts the process.  On a
 *     failure are_last_error() returns a message for the calling thread.
 *   - Array arguments are plain pointers.  Unless a call says otherwise a
 *     pointer may address host memory (pageable or pinned) or device memory
 *     of the context's GPU; the library asks the CUDA runtime which it is.
 *   - Inputs are copied: the caller keeps ownership and may free or reuse
 *     its buffers when the call returns.
 *   - Handles (YET, ELT, layer) are small positive integers owned by the
 *     context; are_destroy() frees everything they refer to.
 *   - Outputs go to caller-allocated buffers.
 *   - "stream" is a cudaStream_t passed as void*.  With a stream the call
 *     only enqueues its work there: device inputs must be ready in that
 *     stream's order and device outputs are ready when the stream reaches
 *     the call.  NULL means: wait for all earlier work on the device, run on
 *     the context's own stream and finish before returning.  A call that
 *     returns values in host memory always waits for them.
 *   - The load calls (are_load_*) are synchronous; when given device
 *     pointers they first wait for all earlier work on the device.
 *   - Event ids are 0-based in [0, catalog_size).  Loss values, deductibles
 *     and retentions are finite and >= 0; limits are >= 0 and may be +inf.
 */
#ifndef ARE_H
#define ARE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define ARE_API __attribute__((visibility("default")))
#else
#define ARE_API
#endif

typedef struct are_ctx are_ctx;

typedef int32_t are_status;
#define ARE_OK 0
#define ARE_EINVAL 1    /* bad argument or malformed input data */
#define ARE_ENOMEM 2    /* over the context's memory budget, or the GPU is full */
#define ARE_ECUDA 3     /* a CUDA runtime call failed */
#define ARE_ETIMEOUT 4  /* a bounded wait ran out */
#define ARE_EBUSY 5     /* the serving queue is full */
#define ARE_ENOTFOUND 6 /* unknown handle or ticket */

/* Largest number of ELTs in one layer (the paper's layers cover 3 to 30,
 * Section II-A item 3). */
#define ARE_MAX_ELTS_PER_LAYER 32

/* Financial terms I of one ELT (Section II-A item 2: currency exchange rate
 * and terms applied to each event loss).  The loss net of terms of an event
 * with loss x is  share * min(max(fx * x - deductible, 0), limit).
 * fx > 0 finite; deductible >= 0 finite; limit >= 0 (+inf = none);
 * 0 <= share <= 1. */
typedef struct {
    double fx;
    double deductible;
    double limit;
    double share;
} are_fin_terms;

/* Layer terms T of Table I: occurrence retention/limit, applied to each
 * event occurrence; aggregate retention/limit, applied to the running sum of
 * occurrence losses within a trial.  Retentions >= 0 finite; limits >= 0
 * (+inf = none). */
typedef struct {
    double occ_ret;
    double occ_lim;
    double agg_ret;
    double agg_lim;
} are_layer_terms;

/* Arithmetic of the analysis stage.
 *   ARE_FP64          terms and sums in FP64; an event's terms are added in
 *                     the layer's ELT order.
 *   ARE_FP32_KAHAN    terms in FP32, per-event sums over ELTs in FP32, the
 *                     trial's running sum in FP32 with Kahan compensation
 *                     (the lanes' compensated pairs merged by exact two-sum
 *                     steps).
 *   ARE_FP32_FP64AGG  terms and per-event sums in FP32, the trial's running
 *                     sum in FP64.
 * In every mode an ELT's financial term of an event,
 * share * min(max(fx * loss - deductible, 0), limit), is formed in FP64 (in
 * that order of operations) when the layer's table is built and rounded once
 * to the mode's type.  The order of the FP32 sums over ELTs is not fixed.
 * The paper does not state its precision; its losses are doubles
 * (Section III-B, data structure iii). */
typedef enum {
    ARE_FP64 = 0,
    ARE_FP32_KAHAN = 1,
    ARE_FP32_FP64AGG = 2
} are_precision;

/* ------------------------------------------------------------------------ */
/* Context                                                                   */
/* ------------------------------------------------------------------------ */

/* Create a context on CUDA device `device`.  mem_budget_bytes caps the
 * device memory the context allocates for YETs, ELTs, tables and scratch
 * (0 = no cap); a load that would exceed it fails with ARE_ENOMEM and leaves
 * the context unchanged.  *out receives the context.  ARE_ECUDA if the device
 * cannot be used. */
ARE_API are_status are_create(are_ctx **out, int device, size_t mem_budget_bytes);

/* Free every device buffer and handle of the context, then the context.
 * NULL is accepted.  The caller must not use the context afterwards. */
ARE_API are_status are_destroy(are_ctx *ctx);

/* Message of the last failed call made by the calling thread on `ctx`
 * ("" if none); with ctx NULL, of its last failed are_risk_measures_static
 * call.  The string stays valid until that thread's next call. */
ARE_API const char *are_last_error(const are_ctx *ctx);

/* Device memory the context holds now, in bytes (budget accounting). */
ARE_API are_status are_memory_used(const are_ctx *ctx, size_t *bytes);

/* Number of CUDA kernels the context has launched since it was created
 * (every launch of every call, validation included). */
ARE_API are_status are_launch_count(const are_ctx *ctx, uint64_t *launches);

/* ------------------------------------------------------------------------ */
/* Inputs (Section II-A)                                                     */
/* ------------------------------------------------------------------------ */

/* Load a Year Event Table: n_trials trials, each an ordered sequence of
 * event ids (Section II-A item 1; the paper stores ids and trial boundaries,
 * Section III-B data structures i and ii).
 *   catalog_size      number of events in the catalog, > 0; ids in [0, C).
 *   offsets           int64[n_trials + 1], offsets[0] = 0, non-decreasing;
 *                     trial i is event_ids[offsets[i] .. offsets[i+1]).
 *                     NULL when every trial holds events_per_trial events.
 *   events_per_trial  > 0 when offsets is NULL, ignored otherwise.
 *   event_ids         int32[total events], in stored (time-stamp) order.
 *   timestamps        NULL, or float32[total events]; when given they must
 *                     be non-decreasing within each trial.  They are checked
 *                     and not kept: the method uses the stored order.
 * Ids, offsets and timestamps are validated on the device; a violation
 * returns ARE_EINVAL and loads nothing.  *yet_handle receives the handle. */
ARE_API are_status are_load_yet(are_ctx *ctx, int32_t catalog_size, int64_t n_trials,
                        const int64_t *offsets, int32_t events_per_trial,
                        const int32_t *event_ids, const float *timestamps,
                        int32_t *yet_handle);

/* Load an Event Loss Table: n_entries (event id, loss) pairs (Section II-A
 * item 2) with its financial terms.  Ids >= 0 and distinct within the ELT
 * (duplicates are ARE_EINVAL); losses finite and >= 0.  n_entries may be 0.
 * *elt_handle receives the handle. */
ARE_API are_status are_load_elt(are_ctx *ctx, int32_t n_entries, const int32_t *event_ids,
                        const double *losses, const are_fin_terms *terms,
                        int32_t *elt_handle);

/* Define a layer: 1..ARE_MAX_ELTS_PER_LAYER ELT handles (the same ELT may not
 * appear twice) and its layer terms (Section II-A item 3, Table I).  The
 * order of elt_handles fixes the order in which per-ELT losses are summed.
 * *layer_handle receives the handle. */
ARE_API are_status are_define_layer(are_ctx *ctx, const int32_t *elt_handles, int32_t n_elts,
                            const are_layer_terms *terms, int32_t *layer_handle);

/* Release a YET, an ELT (ARE_EINVAL while a layer uses it) or a layer,
 * with any tables built for it.  ARE_ENOTFOUND for an unknown handle. */
ARE_API are_status are_free_yet(are_ctx *ctx, int32_t yet_handle);
ARE_API are_status are_free_elt(are_ctx *ctx, int32_t elt_handle);
ARE_API are_status are_free_layer(are_ctx *ctx, int32_t layer_handle);

/* ------------------------------------------------------------------------ */
/* Analysis stage (Section II-B)                                             */
/* ------------------------------------------------------------------------ */

/* Table layout of a layer for the FP32 analysis (are_prepare, are_simulate,
 * are_simulate_streamed).  ARE_LAYOUT_DIRECT (the default): the direct-access
 * layout of Section III-B, one row per catalog event.  ARE_LAYOUT_COMPACT: a
 * row index over the catalog (4 bytes per event, -1 for an event in none of
 * the layer's ELTs) and rows only for the events present in some ELT, for
 * large catalogs and sparse ELTs; an event without a row has a zero loss in
 * every ELT, so its row is not read.  The results are the same bit for bit.
 * FP64 analyses, portfolios, per-occurrence outputs and the server use the
 * direct layout. */
#define ARE_LAYOUT_DIRECT 0
#define ARE_LAYOUT_COMPACT 1
ARE_API are_status are_set_table_layout(are_ctx *ctx, int32_t layer, int32_t layout);

/* The table rows an analysis of `layer` over `yet` reads (Section III-B's
 * direct access, one row per event occurrence), for reporting: *row_bytes
 * receives the bytes of one row and *packed 1 where the rows are packed (the
 * column mask and the non-zero terms of each event, built when the layer's
 * entries per catalog event are few), else 0.  kernel: a kernel choice as in
 * are_tune_result (0 .. 3), or -1 for the one a single-layer are_simulate of
 * this kind of work uses now (tuned, or the default).  Nothing is built or
 * launched.  ARE_ENOTFOUND for an unknown handle, ARE_EINVAL for a bad
 * kernel or a NULL output. */
ARE_API are_status are_layer_rows(are_ctx *ctx, int32_t layer, int32_t yet, are_precision precision,
                                  int32_t kernel, int32_t *row_bytes, int32_t *packed);

/* Preprocessing (Section II-B, stage 1; Section III-B's direct access
 * tables): (re)build the layer's event-major direct-access table for the
 * YET's catalog in the given precision, on `stream`.  are_simulate builds
 * the table on first use; calling this first keeps that cost out of it. */
ARE_API are_status are_prepare(are_ctx *ctx, int32_t layer, int32_t yet, are_precision precision,
                       void *stream);

/* Analysis stage for one layer (Basic Algorithm, Section II-B): for trials
 * trial_begin .. trial_begin + n_trials - 1 of the YET, look up every event
 * in every ELT of the layer, apply the financial terms, sum over ELTs, apply
 * the occurrence terms, accumulate the trial's running sum and apply the
 * aggregate terms; ylt[i] receives the loss of trial trial_begin + i
 * (double[n_trials], host or device).  Trials are independent, so a run split
 * into trial ranges gives the same YLT as one run.  Enqueued on `stream`;
 * when ylt is host memory the call copies it back and synchronises. */
ARE_API are_status are_simulate(are_ctx *ctx, int32_t layer, int32_t yet, int64_t trial_begin,
                        int64_t n_trials, are_precision precision, double *ylt,
                        void *stream);

/* Analysis stage for n_layers layers over the same trials (the Basic
 * Algorithm's outer loop over layers; the portfolio analysis of Section IV).
 * ylts[i] (device memory, double[n_trials]) receives layer layers[i]'s YLT.
 * With FP32 tables the tuned configuration decides between persistent
 * launches (one per table width) whose warps claim (layer, trial tile) work
 * items layer by layer, and one single-layer launch per layer, back to back;
 * FP64 runs one launch per layer.  The first call with a given set of layers, YET, trial
 * range, precision, output pointers and tuned configuration builds the
 * layers' tables, a work list and a CUDA graph; identical later calls replay
 * the graph.  Replays of one plan must not overlap on the GPU. */
ARE_API are_status are_simulate_portfolio(are_ctx *ctx, const int32_t *layers, int32_t n_layers,
                                          int32_t yet, int64_t trial_begin, int64_t n_trials,
                                          are_precision precision, double *const *ylts,
                                          void *stream);

/* ------------------------------------------------------------------------ */
/* Launch tuning                                                             */
/* ------------------------------------------------------------------------ */

/* The launch configuration the autotuner picked for one kind of work. */
typedef struct {
    int32_t kernel;          /* 0 persistent work items, 1 staged rows (one event per lane),
                                2 register rows (rows read straight into registers by a
                                warp per block of trials: a packed row of the non-zero
                                terms behind their column mask, 32 bytes where the layer
                                holds few entries per catalog event, else 64, or in FP32
                                the dense row of up to 16 ELTs; are_layer_rows tells which;
                                FP64 with exact trial sums), 3 (FP64) staged rows of an
                                FP32 screen with the marked entries read from the FP64
                                table */
    int32_t rows_in_flight;  /* register rows and persistent kernel: groups of 32 events
                                per batch, 1 or 2; staged kernel: events per lane per
                                batch, 1 or 2; 0 (in a loaded tuning file): the
                                kernel's default */
    int32_t trials_per_item; /* trials per work item (persistent kernel) */
    int32_t blocks_per_sm;   /* 0 = as many as fit */
    double ms;               /* measured time of one pass */
} are_tune_result;

/* Time every candidate launch configuration on these layers and this YET
 * (one layer: the single-layer kernels and persistent-kernel settings;
 * several: back-to-back single-layer launches, or the persistent kernel with
 * its rows in flight and trials per work item)
 * and keep the fastest for this kind of work: precision, YET layout, widest
 * table row, mean events per trial and one layer vs several.  Later
 * are_simulate and are_simulate_portfolio calls of that kind use it.
 * Untuned work runs the register-rows kernel with one group of 32 events per
 * batch over 32-byte FP32 rows and two over wider rows and FP64 rows.
 * *best (may be NULL) receives the winner.  Runs on `stream` and waits. */
ARE_API are_status are_autotune(are_ctx *ctx, const int32_t *layers, int32_t n_layers,
                                int32_t yet, are_precision precision, void *stream,
                                are_tune_result *best);

/* Write / read the context's tuning table (one JSON object per line). */
ARE_API are_status are_tune_save(are_ctx *ctx, const char *path);
ARE_API are_status are_tune_load(are_ctx *ctx, const char *path);

/* The same analysis stage with per-occurrence outputs (step 4 of the
 * Basic Algorithm before its final sum): for every event occurrence of the
 * trials, in stored order, marginals[e - first] = m_d = A_d - A_{d-1}, the
 * aggregate-clamped running total's increment at that occurrence (the
 * year-event loss table of the layer), where `first` is the first event of
 * trial trial_begin; occ_max[i] (may be NULL) = the largest occurrence loss
 * (after occurrence terms) of trial trial_begin + i, the input of an
 * occurrence-exceedance PML; ylt[i] (may be NULL) = the trial loss.  All
 * three are device memory.  The running totals come from warp-shuffle
 * prefix scans; the precision argument selects the table and term
 * arithmetic as for are_simulate, the running totals are FP64. */
ARE_API are_status are_simulate_occurrences(are_ctx *ctx, int32_t layer, int32_t yet,
                                            int64_t trial_begin, int64_t n_trials,
                                            are_precision precision, double *marginals,
                                            double *occ_max, double *ylt, void *stream);

/* Folded layer table -- a variant of the analysis stage, not the per-ELT
 * lookup of the Basic Algorithm.  Steps 1-3 of Section II-B (lookup,
 * financial terms, sum over ELTs, occurrence terms) depend on the event and
 * the layer only, since occurrence terms apply to each occurrence on its
 * own.  are_prepare_folded computes, once per catalog event e and in FP64,
 * the occurrence loss h[e] (the same operations in the same ELT order as
 * are_simulate's FP64 path, so equal to it bit for bit), a bitmap of
 * h[e] > 0 and the largest h, from the ELTs' entries (one pass per ELT, in
 * layer order).  Memory: 8 B per catalog event + catalog / 8 B, held until
 * the layer is freed.  Enqueued on `stream`. */
ARE_API are_status are_prepare_folded(are_ctx *ctx, int32_t layer, int32_t yet, void *stream);

/* Trial pass over the folded table: ylt[i] (double[n_trials], host or
 * device) = min(max(S - AggR, 0), AggL) for trial trial_begin + i, with S the
 * sum of h over the trial's occurrences.  S is formed exactly (h scaled by
 * a power of two taken from the largest h and added as integers; any h of at
 * least 2^-52 of the largest converts without error) and rounded to double
 * once, so it does not depend on the order of the occurrences or on how the
 * trials are split.  Builds the folded table on first use.  Same stream and
 * host-memory rules as are_simulate. */
ARE_API are_status are_simulate_folded(are_ctx *ctx, int32_t layer, int32_t yet,
                                       int64_t trial_begin, int64_t n_trials, double *ylt,
                                       void *stream);

/* Analysis stage for one layer over a YET held in host memory (Section
 * II-B with the YET of Section II-A item 1 left where it is): the same
 * result as are_load_yet + are_simulate, without a device copy of the whole
 * YET.  The trials are cut into chunks of whole trials of about
 * chunk_events ids (0: 64M; a longer trial forms a chunk alone); the copy of
 * each chunk to the device (the host-to-device link, pinned memory at full
 * speed) overlaps the analysis of the one before, in two device buffers of
 * one chunk each.  Arguments as for are_load_yet (offsets: n_trials + 1
 * int64, host or device, or NULL with events_per_trial > 0; event_ids: host
 * memory, read until the call returns) and are_simulate (ylt: double[n_trials],
 * host or device).  Ids are checked on the device as they arrive: an id
 * outside [0, catalog_size) is read as 0 and the call returns ARE_EINVAL,
 * with ylt not valid.  Waits for completion, also with a caller stream
 * (then it runs after the work already queued on that stream). */
ARE_API are_status are_simulate_streamed(are_ctx *ctx, int32_t layer, int32_t catalog_size,
                                         int64_t n_trials, const int64_t *offsets,
                                         int32_t events_per_trial, const int32_t *event_ids,
                                         int64_t chunk_events, are_precision precision,
                                         double *ylt, void *stream);

/* are_simulate_streamed over a host YET whose event ids are packed id_bits
 * bits each (1 .. 32; ceil(log2(catalog_size)) is enough): id i occupies
 * bits i * id_bits .. (i + 1) * id_bits - 1 of the stream of 32-bit words
 * packed_ids (bit b of the stream is bit b % 32 of word b / 32), as
 * are_pack_ids writes it: ceil(n_events * id_bits / 32) words of host
 * memory.  Only those words cross the host-to-device link (2.5 bytes per id
 * for a catalog of up to 2^20 events, against 4); the ids are unpacked and
 * checked on the device as each chunk arrives.  Same results, arguments,
 * stream and error behaviour as are_simulate_streamed otherwise. */
ARE_API are_status are_simulate_streamed_packed(are_ctx *ctx, int32_t layer, int32_t catalog_size,
                                                int64_t n_trials, const int64_t *offsets,
                                                int32_t events_per_trial, const uint32_t *packed_ids,
                                                int32_t id_bits, int64_t chunk_events,
                                                are_precision precision, double *ylt, void *stream);

/* Packs n event ids (host memory, each in [0, 2^id_bits)) id_bits bits each
 * into ceil(n * id_bits / 32) 32-bit words of host memory, the layout
 * are_simulate_streamed_packed reads.  Host work only; ARE_EINVAL for an id
 * that does not fit. */
ARE_API are_status are_pack_ids(are_ctx *ctx, const int32_t *ids, int64_t n, int32_t id_bits,
                                uint32_t *out);

/* One launch shape of the gather ceiling and its measured rate. */
typedef struct {
    int32_t kind;            /* 0: 16-byte loads, row_bytes/16 lanes per row, each lane
                                reading its row's id; 1: 32-byte loads, row_bytes/32 lanes
                                per row, ids read once per 32 events and passed by shuffles
                                (the FP32 register-rows kernel's shape); 2: whole rows
                                copied into shared memory by 16-byte cp.async (the staged
                                kernels' shape) */
    int32_t rows_in_flight;  /* kind 0: rows per lane; kinds 1 and 2: groups of 32 events */
    int32_t blocks_per_sm;   /* 256-thread blocks per SM */
    double rows_per_s;
} are_ceiling_shape;

/* Gather ceiling -- a measurement helper, not a step of the method.  Reads,
 * for every event occurrence of trials trial_begin .. trial_begin +
 * n_trials - 1 of the YET, its id and one row of row_bytes bytes (32, 64 or
 * 128) of a zero table with one row per catalog event, as the analysis
 * kernels do, and nothing else; the table is allocated and freed inside the
 * call (against the memory budget).  Every shape of are_ceiling_shape is
 * timed with 2 to 16 rows per lane (or 1 to 4 groups of 32 events) in flight
 * and 3, 4, 6 and 8 blocks per SM (those that fit, or as many as fit when that
 * is fewer than 3), the best of `reps` timed
 * passes (1..100) each.  *rows_per_s receives the best rate of all: the bound
 * that the table-row reads put on any analysis kernel for this YET and row
 * size.  shapes (may be NULL) receives up to max_shapes of the shapes timed
 * and *n_shapes (may be NULL) how many were timed.  Blocks the caller. */
ARE_API are_status are_gather_ceiling(are_ctx *ctx, int32_t yet, int32_t row_bytes,
                                      int64_t trial_begin, int64_t n_trials, int32_t reps,
                                      double *rows_per_s, are_ceiling_shape *shapes,
                                      int32_t max_shapes, int32_t *n_shapes);

/* ------------------------------------------------------------------------ */
/* Filters on the YLT (Section II-C): PML and TVaR                           */
/* ------------------------------------------------------------------------ */

/* From a YLT of n > 0 trial losses (host or device):
 *   pml_out[r]  = the m-th largest loss, m = ceil(n / return_periods[r]),
 *                 return period read to the nearest 1e-6 and >= 1;
 *   tvar_out[r] = the mean of the m largest losses,
 *                 m = ceil(n * (1 - tvar_levels[r])), level read to the
 *                 nearest 1e-9 and strictly between 0 and 1.
 * The paper names these measures without defining them (Section I,
 * Section II-C); this is the reading the library takes.
 * pml_out and tvar_out are both host arrays (the call synchronises
 * `stream`) or both device arrays (ylt must then be device memory: the call
 * only enqueues the selection and the copies into them, and returns; the
 * values are there when `stream` reaches that point).  The selection's
 * scratch belongs to the context, so selections of one context on
 * different streams must not overlap.  Mixed host and device outputs, or
 * device outputs with a host YLT, are ARE_EINVAL. */
ARE_API are_status are_risk_measures(are_ctx *ctx, const double *ylt, int64_t n,
                             const double *return_periods, int32_t n_rp, double *pml_out,
                             const double *tvar_levels, int32_t n_tv, double *tvar_out,
                             void *stream);

/* are_risk_measures for n_ylt YLTs of n losses each (ylts: host array of
 * device pointers), selected together: pml_out[y * n_rp + r] and
 * tvar_out[y * n_tv + r] are host arrays.  Synchronises `stream`. */
ARE_API are_status are_risk_measures_batch(are_ctx *ctx, const double *const *ylts, int32_t n_ylt,
                                           int64_t n, const double *return_periods, int32_t n_rp,
                                           double *pml_out, const double *tvar_levels,
                                           int32_t n_tv, double *tvar_out, void *stream);

/* ------------------------------------------------------------------------ */
/* Pricing server: continuous batching of requests                           */
/* ------------------------------------------------------------------------ */

/* The paper's real-time pricing scenario (Section I, Section IV: an
 * underwriter prices a contract while on the phone) as a server over one
 * resident YET and the context's resident ELTs.  A scheduler thread inside
 * the library admits queued requests while request slots and arena memory
 * are free, hands each iteration's budget of events_per_launch to the
 * admitted requests in arrival order, the oldest whole (or, with
 * least_work_first, in order of least remaining work less the time waited,
 * so short requests overtake long ones), and runs the slices of small
 * requests in one persistent
 * launch and those of large ones on the single-layer kernel; a request
 * arriving while others run joins at the next iteration, and the next
 * iteration is always queued behind the running one.  When a request's last
 * slice is done its PML/TVaR are selected and its result posted.  All
 * device waits are bounded. */
typedef struct {
    int32_t max_inflight;      /* requests admitted at once, 1..256 */
    int32_t max_pending;       /* queued requests; a submit beyond is ARE_EBUSY */
    size_t arena_bytes;        /* device memory for admitted requests' tables and YLTs */
    int64_t events_per_launch; /* events of one batched launch (0 = 2e8) */
    int32_t trials_per_item;   /* trials per work item (0 = 8) */
    int32_t one_at_a_time;     /* 1: no batching; each request runs alone, whole, in order */
    are_precision precision;   /* ARE_FP32_KAHAN or ARE_FP32_FP64AGG */
    int64_t stall_us;          /* test hook: the scheduler sleeps this long before each launch */
    int32_t folded;            /* nonzero: price each request on its folded table (FP64
                                  occurrence loss per catalog event, exact trial sums, one
                                  lookup per occurrence -- the variant of are_simulate_folded);
                                  precision is then not used */
    int32_t least_work_first;  /* 0: arrival order -- the oldest admitted request runs whole
                                  and the ones behind it share the budget (nothing overtakes,
                                  which gives the lowest tail latency when request sizes are
                                  bounded); 1: the budget goes in order of least remaining
                                  work less the time waited (short requests overtake long
                                  ones, which are cut into slices) */
} are_server_cfg;

/* One pricing request: a layer of the context's ELTs with its own layer terms,
 * priced over trials 0 .. n_trials-1 of the server's YET.  Everything is
 * copied at submission. */
typedef struct {
    const int32_t *elt_handles;
    int32_t n_elts;               /* 1 .. ARE_MAX_ELTS_PER_LAYER */
    are_layer_terms terms;
    int64_t n_trials;             /* 1 .. trials in the YET */
    const double *return_periods; /* PML return periods, n_rp of them */
    int32_t n_rp;
    const double *tvar_levels;    /* TVaR levels, n_tv of them; n_rp + n_tv <= 8 */
    int32_t n_tv;
} are_request;

typedef struct {
    are_status status;   /* ARE_OK, or why the request failed */
    int32_t n_rp, n_tv;
    double pml[8];
    double tvar[8];
    int64_t n_trials;
    double queue_us;     /* submission -> admission */
    double run_us;       /* admission -> result posted */
    double total_us;     /* submission -> result posted */
} are_result;

/* Start the server on `yet` (ARE_EBUSY if one runs).  While it runs the YET
 * and every ELT cannot be freed. */
ARE_API are_status are_server_start(are_ctx *ctx, int32_t yet, const are_server_cfg *cfg);
/* Queue a request; *ticket identifies it.  ARE_EBUSY when max_pending
 * requests are queued. */
ARE_API are_status are_submit(are_ctx *ctx, const are_request *req, int64_t *ticket);
/* Wait up to timeout_us (< 0: no limit) for a request's result and hand it
 * over (a ticket's result can be taken once).  ARE_ETIMEOUT if it is not
 * ready in time; ARE_ENOTFOUND for an unknown, taken or cancelled ticket. */
ARE_API are_status are_wait(are_ctx *ctx, int64_t ticket, int64_t timeout_us, are_result *out);
/* Cancel a queued or running request; its slot and memory are freed at the
 * next launch boundary. */
ARE_API are_status are_cancel(are_ctx *ctx, int64_t ticket);
/* Finish the admitted requests, cancel the queued ones, stop the scheduler
 * and free the server's memory. */
ARE_API are_status are_server_stop(are_ctx *ctx);

/* ------------------------------------------------------------------------ */
/* Allocation-free PML/TVaR                                                  */
/* ------------------------------------------------------------------------ */

/* Size of the device scratch array behind are_risk_measures_static. */
#define ARE_STATIC_SCRATCH_BYTES (256u * 1024u)

/* PML and TVaR of a device-resident YLT without a context and without any
 * allocation.  The paper has no counterpart: this exists for callers that
 * cannot allocate device memory -- code running under another framework's
 * memory pool or a fixed memory reservation (a real-time pricing service
 * that sizes everything up front), or code that must not create a context.
 *
 * Same definitions and results as are_risk_measures, with these limits:
 *   - ylt must be device memory of the current CUDA device (host memory is
 *     ARE_EINVAL: copying it in would need a device buffer);
 *   - n_rp + n_tv <= 8 (more is ARE_EINVAL); n < 2^32 - 1;
 *   - pml_out and tvar_out are host arrays; the call synchronises `stream`
 *     (NULL = the legacy default stream) before returning.
 * The kernels' scratch (histograms, selection state, per-block partial sums,
 * results) is one file-scope device array of ARE_STATIC_SCRATCH_BYTES
 * (256 KiB) that every GPU loading the library holds until the process
 * exits.  The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress, with the device current) and caches it: make that
 * first call before any stream capture.  Every call shares the one array and
 * reinitialises what must start at zero; calls whose work overlaps on the
 * GPU (other streams or other threads on the same device) race on it and
 * must be serialised by the caller.  Nothing is allocated: no cudaMalloc,
 * no cudaFree, no allocating library routine.  On failure, are_last_error(NULL)
 * returns the calling thread's message. */
ARE_API are_status are_risk_measures_static(const double *ylt, int64_t n,
                                            const double *return_periods, int32_t n_rp,
                                            double *pml_out, const double *tvar_levels,
                                            int32_t n_tv, double *tvar_out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* ARE_H */
