// are_internal.cuh -- context state and kernel entry points shared by the
// translation units of libare.  Not part of the public ABI (include/are.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "are.h"

namespace are {

constexpr int kMaxElts = ARE_MAX_ELTS_PER_LAYER;
constexpr int kMaxTargets = 8;  // PML/TVaR ranks selected in one pass

// ---------------------------------------------------------------------------
// status helpers
// ---------------------------------------------------------------------------

void set_error(const are_ctx *ctx, const std::string &msg);

struct Server;
// Device allocation charged to the context's budget (throws Error).
void *ctx_alloc(are_ctx *ctx, size_t bytes);
void ctx_free(are_ctx *ctx, void *p, size_t bytes);
void server_destroy(are_ctx *ctx);   // stops and frees a running server

struct Error {
    are_status code;
    std::string msg;
};

#define ARE_CUDA_TRY(expr)                                                          \
    do {                                                                            \
        cudaError_t e__ = (expr);                                                   \
        if (e__ != cudaSuccess)                                                     \
            throw ::are::Error{e__ == cudaErrorMemoryAllocation ? ARE_ENOMEM        \
                                                                : ARE_ECUDA,        \
                               std::string(#expr) + ": " + cudaGetErrorString(e__)}; \
    } while (0)

#define ARE_CHECK(cond, code, msg)                      \
    do {                                                \
        if (!(cond)) throw ::are::Error{(code), (msg)}; \
    } while (0)

// ---------------------------------------------------------------------------
// device-resident inputs
// ---------------------------------------------------------------------------

struct Yet {
    int32_t catalog = 0;
    int64_t n_trials = 0;
    int32_t k = 0;                 // events per trial when fixed, else 0
    int64_t n_events = 0;
    int64_t *d_off = nullptr;      // n_trials + 1 (ragged only)
    int32_t *d_ids = nullptr;      // n_events, padded by kIdPad zero ids
    size_t bytes = 0;
};
constexpr int64_t kIdPad = 64;     // zero ids after the last event (vector over-read)

struct Elt {
    int32_t n = 0;
    int32_t max_id = -1;
    double max_loss = 0.0;         // largest loss of the ELT
    int32_t *d_ids = nullptr;
    double *d_loss = nullptr;
    are_fin_terms terms{};
    size_t bytes = 0;
    int users = 0;                 // layers referring to it
};

// Event-major direct-access table of one layer: row e holds, for each of the
// layer's ELTs in layer order, event e's financial term
// share * min(max(fx * loss - D, 0), Lim) (zero where the ELT has no entry
// for e), jp columns (j >= J are zero).
struct Table {
    int32_t catalog = -1;
    int jp = 0;
    void *d = nullptr;
    size_t bytes = 0;
};

// Folded table of one layer: the FP64 occurrence loss h[e] of every catalog
// event as a 128-bit fixed-point integer F[e] = h[e] * 2^s (s from the
// largest h), a bitmap of h > 0 and the largest h (its bits), in one
// allocation laid out [hmax | 248 B pad][bits: words x 4 B][F: catalog x 16 B].
struct Folded {
    int32_t catalog = -1;
    int32_t words = 0;
    void *d = nullptr;
    size_t bytes = 0;
    unsigned long long *hmax() const { return static_cast<unsigned long long *>(d); }
    uint32_t *bits() const { return reinterpret_cast<uint32_t *>(static_cast<char *>(d) + 256); }
    ulonglong2 *F() const
    {
        return reinterpret_cast<ulonglong2 *>(static_cast<char *>(d) + 256 +
                                              (((size_t)words * 4 + 255) & ~(size_t)255));
    }
};

// Compact FP32 table of one layer: row_of[catalog] (-1: no row) and rows
// for the events present in some ELT, in one allocation laid out
// [row_of | scan scratch | rows: max_rows x jp floats].
struct Compact {
    int32_t catalog = -1;
    int jp = 0;
    int64_t max_rows = 0;
    void *d = nullptr;
    size_t bytes = 0;
    size_t counts_off = 0, rows_off = 0;
    int32_t *row_of() const { return static_cast<int32_t *>(d); }
    int32_t *counts() const { return reinterpret_cast<int32_t *>(static_cast<char *>(d) + counts_off); }
    float *rows() const { return reinterpret_cast<float *>(static_cast<char *>(d) + rows_off); }
};

// Packed table of one layer: catalog rows of 32 or 64 bytes holding each
// event's non-zero terms in column order behind the mask of their columns,
// a counter and the overflow terms, in one allocation laid out [rows |
// counter (256 B) | overflow].  FP64 (built from the ELT entries by
// launch_pack64_direct):
// rw = 4 or 8 64-bit words per row, the mask and the overflow offset in word
// 0, up to rw - 1 terms inline and every term of a longer row in the
// overflow.  FP32 (built from the ELT entries by launch_pack32_direct):
// rw = 8 or 16 32-bit words, the mask in word 0, up to rw - 1 terms inline;
// a longer row keeps rw - 2 inline and the offset of the rest in its last
// word.  The row size follows the layer's entries per catalog event
// (packed_row_words).
struct Packed {
    int32_t catalog = -1;
    int rw = 0;
    void *d = nullptr;
    size_t bytes = 0;
    size_t rows_bytes = 0;
    void *rows() const { return d; }
    unsigned long long *used() const
    {
        return reinterpret_cast<unsigned long long *>(static_cast<char *>(d) + rows_bytes);
    }
    void *ovf() const { return static_cast<char *>(d) + rows_bytes + 256; }
};

struct Layer {
    std::vector<int32_t> elts;
    are_layer_terms terms{};
    Table t32, t64;
    Table t32u;              // FP32 screen of t64: its values rounded up
    Packed p64;              // packed FP64 rows of t64
    Packed p32;              // packed FP32 rows of t32 (layers of more than 8 ELTs)
    Folded fold;
    int layout = 0;          // ARE_LAYOUT_DIRECT or ARE_LAYOUT_COMPACT (FP32 analysis)
    Compact comp;
    uint64_t generation = 0;   // bumped whenever a table is (re)allocated or freed
};

// ---------------------------------------------------------------------------
// kernel parameter blocks (passed by value; they live in the constant bank)
// ---------------------------------------------------------------------------

// The layer's occurrence terms (Table I); the per-ELT terms are in the table.
struct TermsF32 {
    float occ_r, occ_l;
};
struct TermsF64 {
    double occ_r, occ_l;
};

struct SimArgs {
    const int32_t *ids;      // YET event ids
    const int64_t *off;      // ragged offsets or nullptr
    int32_t k;               // fixed events per trial
    int64_t trial_begin;
    int64_t n_trials;
    const void *table;       // [catalog][jp]
    const void *table2;      // screened FP64: the FP32 screen [catalog][jp32];
                             // compact FP32 (kernel 4): the row index row_of[catalog]
    int32_t jp64;            // screened FP64: columns of the FP64 table
    int32_t n_elts;          // ELTs of the layer
    double agg_r, agg_l;
    double *ylt;             // n_trials (may be null when occurrences are written)
    int kernel;              // 1 staged, 2 register rows, 3 (FP64) staged screen
    int epl;                 // staged FP32 kernel: events per lane per batch (1 or 2);
                             // register-rows kernel: groups of 32 events per batch (1 or 2);
                             // 0: the kernel's default (one event per lane; one group over
                             // 32-byte FP32 rows, two over wider rows and FP64 rows)
    double *marg;            // per-occurrence marginals, or null
    double *occ_max;         // largest occurrence loss per trial, or null
    int64_t marg_base;       // event index of marg[0]
};

// The trial pass over a folded table.
struct FoldArgs {
    const int32_t *ids;
    const int64_t *off;      // ragged offsets or nullptr
    int32_t k;
    int64_t trial_begin;
    int64_t n_trials;
    int64_t n_events;        // of the whole YET (the id array's extent)
    const ulonglong2 *F;     // [catalog] occurrence losses h * 2^s, 128-bit (x low, y high)
    const uint32_t *bits;    // [words] bit e set iff h[e] > 0
    int32_t words;
    const unsigned long long *hmax;   // bits of the largest h
    double agg_r, agg_l;
    double *ylt;             // n_trials
};

// The layer's ELTs and their financial terms, as the table builders read them.
struct ScatterArgs {
    const int32_t *ids[kMaxElts];
    const double *loss[kMaxElts];
    int32_t n[kMaxElts];
    double fx[kMaxElts];
    double ded[kMaxElts];
    double lim[kMaxElts];
    double share[kMaxElts];
    int32_t n_elts;
    int32_t jp;
};

// A layer table entry: the financial term share * min(max(fx * x - D, 0), Lim)
// of a loss x in FP64, operation by operation (Section II-B step 2).
__device__ __forceinline__ double fin_term(double x, double fx, double ded, double lim, double share)
{
    double e = __dsub_rn(__dmul_rn(fx, x), ded);
    e = e > 0.0 ? e : 0.0;
    e = e > lim ? lim : e;
    return __dmul_rn(share, e);
}

// One layer of a persistent multi-layer launch (FP32 tables).
struct LayerF32 {
    const float *table;      // [catalog][jp] terms
    double *ylt;             // n_trials losses
    float occ_r, occ_l;
    double agg_r, agg_l;
    int32_t jp;              // 8, 16 or 32
    int64_t item_begin;      // index of the layer's first work item
    int64_t t0, nt;          // the layer's trials: t0 .. t0 + nt - 1 (ylt indexed by trial)
};

// Work of a persistent launch: every layer's trials cut into items of
// trials_per_item trials, numbered layer by layer.
struct ItemWork {
    const int32_t *ids;
    const int64_t *off;      // ragged offsets or nullptr (k events per trial)
    int32_t k;
    int64_t trial_begin, n_trials;
    int32_t trials_per_item;
    int32_t n_layers;
    int64_t n_items;
    const LayerF32 *layers;            // device array of n_layers, or nullptr: use `one`
    unsigned long long *counter;       // device, zero before the launch; nullptr: static split
    LayerF32 one;                      // the layer when there is exactly one
};

// Tunables of the persistent kernel.
struct ItemConfig {
    int rows_in_flight = 2;  // U: groups of 32 events per batch (1 or 2)
    int trials_per_item = 8; // trials per work item
    int blocks_per_sm = 0;   // 256-thread blocks per SM (0 = as many as fit)
};

// A tuned launch configuration of the analysis stage.
struct TuneEntry {
    int kernel = 0;            // 0 persistent items, 1 staged, 2 register
    ItemConfig cfg;
    double ms = 0.0;
};

// A cached multi-layer launch: work list and CUDA graph.
struct Plan {
    std::vector<int32_t> layers;
    std::vector<uint64_t> generations;
    std::vector<double *> ylts;
    int32_t yet = 0;
    int64_t trial_begin = 0, n_trials = 0;
    int precision = 0;
    int kernel = 0;
    ItemConfig cfg;
    void *d_work = nullptr;    // LayerF32 records by table width, then the item counters
    size_t work_bytes = 0;
    uint64_t launches = 0;     // kernels per replay
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

// ---------------------------------------------------------------------------
// launchers (one per translation unit); each returns the number of kernels
// it launched, which the context adds to its launch count
// ---------------------------------------------------------------------------

// repack.cu
int launch_scatter_table(void *table, bool fp32, const ScatterArgs &a, cudaStream_t s,
                         bool round_up = false);
int launch_screen64(const SimArgs &a, int jp32, const TermsF64 &t, int num_sms, cudaStream_t s);
int64_t compact_scan_blocks(int32_t catalog);
int launch_build_compact(int32_t *row_of, int32_t *counts, float *rows, size_t rows_bytes,
                         int32_t catalog, const ScatterArgs &a, cudaStream_t s);
int32_t folded_words(int32_t catalog);
bool folded_bits_in_smem(int32_t words);
int launch_fold(const ScatterArgs &elts, double occ_r, double occ_l, int32_t catalog, ulonglong2 *F,
                uint32_t *bits, unsigned long long *hmax, int num_sms, cudaStream_t s);
int launch_folded(const FoldArgs &a, int num_sms, cudaStream_t s);
// One launch shape of the gather ceiling and its rate (ceiling.cu).
struct CeilingShape {
    int kind;              // 0 16-byte loads, 1 32-byte loads with shuffled ids, 2 cp.async staging
    int rows_in_flight;    // rows per lane (0) or groups of 32 events (1, 2) in flight
    int blocks_per_sm;     // 256-thread blocks per SM
    double rows_per_s;
};
std::vector<CeilingShape> gather_ceiling(const int32_t *ids, int64_t n, int row_bytes, int reps,
                                         int num_sms, const void *table, float *out, cudaStream_t s,
                                         uint64_t &launches);
int table_jp(int n_elts, bool fp32);
int packed_row_words(int n_elts, double terms_per_event, bool fp32);
int launch_pack64_direct(const ScatterArgs &a, int32_t catalog, int rw, unsigned long long *rows, double *ovf,
                         unsigned long long *ovf_used, cudaStream_t s);
int launch_pack32_direct(const ScatterArgs &a, int32_t catalog, int pw, uint32_t *rows, float *ovf,
                         unsigned long long *ovf_used, cudaStream_t s);

// api.cu: how many blocks of `kern` (threads per block, bytes of dynamic
// shared memory) fit on one SM of the current device.  On the first call for
// a device it also raises the kernel's dynamic shared-memory limit to `smem`
// on that device; the answer is kept per (kernel, device, shape) under a
// lock, so contexts on several devices and threads may share the library.
int fit_blocks(const void *kern, int threads, size_t smem);

// validate.cu: each sets *flag (device int, zeroed by the caller) non-zero on a violation
int launch_check_ids(const int32_t *ids, int64_t n, int32_t catalog, int *flag, cudaStream_t s);
int launch_sanitize_ids(int32_t *ids, int64_t n, int32_t catalog, int *flag, cudaStream_t s);
// ids of `bits` bits each packed into 32-bit words (id j at bit bit0 + j *
// bits; one word past the last id readable) -> int32, checked against the
// catalog like launch_sanitize_ids.
int launch_unpack_ids(const uint32_t *words, int64_t bit0, int bits, int64_t n, int32_t catalog, int32_t *out,
                      int *flag, cudaStream_t s);
int launch_check_offsets(const int64_t *off, int64_t n_trials, int64_t n_events, int *flag,
                          cudaStream_t s);
int launch_check_timestamps(const float *ts, const int64_t *off, int64_t n_trials, int32_t k,
                             int *flag, cudaStream_t s);

// sim_items.cu
// All of w's layers must have table width jp (8, 16 or 32 floats).
int launch_items(const ItemWork &w, int jp, const ItemConfig &cfg, are_precision prec,
                 int num_sms, cudaStream_t s);

// staged64.cu: one event per lane, FP64 rows staged in shared memory.
int launch_staged64(const SimArgs &a, int jp, const TermsF64 &t, int num_sms, cudaStream_t s);

// rows64.cu: the FP64 register-rows kernel over the packed FP64 table
// (a.table, row_words words per row; a.table2: its overflow terms); `scale`
// is the fixed-point scale of its exact running sums (every occurrence loss
// times 2^scale below 2^126).
// rows_occ.cu: the per-occurrence outputs over the register-rows kernels'
// rows (form 0 packed FP64, 1 packed FP32, 2 dense FP32; a.table and
// a.table2 the rows and their overflow).
int launch_rows_occ(const SimArgs &a, int form, int row_words, const TermsF32 &t32, const TermsF64 &t64, int scale,
                    int num_sms, cudaStream_t s);
int launch_rows64(const SimArgs &a, int row_words, const TermsF64 &t, int scale, int num_sms,
                  cudaStream_t s);

// simulate.cu
int launch_simulate(const SimArgs &a, are_precision prec, int jp, const TermsF32 *t32,
                     const TermsF64 *t64, int num_sms, cudaStream_t s);

// select.cu
struct SelectScratch {
    uint32_t *hist = nullptr;       // 3 * kMaxTargets * 256
    unsigned long long *state = nullptr;  // per target: prefix, remaining rank
    unsigned int *ctrl = nullptr;   // 4 words: blocks arrived, top word of the largest |value|
    unsigned long long *acc = nullptr;    // per target: integer tail sums and count (7 words)
    double *result = nullptr;       // per target: value, tail mean
    unsigned long long *app = nullptr;    // single-YLT selection, per target: keys kept
    unsigned long long *cand = nullptr;   // per target: the kept keys of its bucket
    int max_blocks = 0;
};
void select_alloc(SelectScratch &s, int num_sms);
// Ranks of the risk measures (definitions in include/are.h); -1 when the
// return period or level is out of range.
int64_t rank_for_return_period(int64_t n, double rp);
int64_t rank_for_level(int64_t n, double a);
// Message of the calling thread's last failed are_risk_measures_static call.
const char *static_last_error();
void select_free(SelectScratch &s);
constexpr int kSelectLaunches = 1 + 8 + 1;    // the multi-YLT and allocation-free selections
inline int select_max_blocks(int num_sms) { return num_sms * 4; }
// ranks[t] (1-based, descending order) for n_targets <= kMaxTargets; writes
// result[2*t] = m-th largest value, result[2*t+1] = mean of the m largest.
cudaError_t select_enqueue(const double *ylt, int64_t n, const int64_t *ranks, int nt,
                           const SelectScratch &s, cudaStream_t st);
// The same for n_ylt YLTs of n losses each (device array of pointers); the
// scratch must be sized by select_multi_bytes.  Results: result[(y*8+t)*2].
size_t select_multi_bytes(int n_ylt, int64_t n, int num_sms);
int launch_select_multi(const double *const *ylts, int n_ylt, int64_t n, const int64_t *ranks,
                        int nt, void *scratch, int num_sms, cudaStream_t st, double **result);
int launch_select(const double *ylt, int64_t n, const int64_t *ranks, int n_targets,
                   SelectScratch &s, int num_sms, cudaStream_t st);

}  // namespace are

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------

struct are_ctx {
    int device = 0;
    int num_sms = 0;
    size_t budget = 0;
    size_t used = 0;
    cudaStream_t stream = nullptr;
    std::recursive_mutex mu;
    int32_t next_handle = 1;
    std::map<int32_t, are::Yet> yets;
    std::map<int32_t, are::Elt> elts;
    std::map<int32_t, are::Layer> layers;
    int *d_flag = nullptr;   // validation flag
    int *h_flag = nullptr;   // pinned mirror
    are::SelectScratch sel;
    double *h_result = nullptr;  // pinned, 2 * kMaxTargets
    uint64_t launches = 0;       // kernels launched by this context
    cudaStream_t capture = nullptr;           // stream used to capture plans
    std::map<std::string, are::TuneEntry> tune;
    std::vector<are::Plan> plans;
    void *d_multi = nullptr;     // batched-selection scratch and pointer array
    size_t multi_bytes = 0;
    double *h_multi = nullptr;   // pinned results of a batched selection
    size_t h_multi_count = 0;
    are::Server *server = nullptr;  // running pricing server, if any
    // device blocks released by the library and kept for reuse: size -> block
    std::multimap<size_t, void *> cache;
    std::map<void *, size_t> block_size;   // every live or cached block's allocated size
    size_t cached = 0;                     // bytes held in `cache`
    cudaStream_t copy_stream = nullptr;    // host-to-device copies of streamed analyses
};
