// api.cu -- host implementation of the C ABI declared in include/are.h:
// context and handle management, input validation, memory-budget
// accounting, the per-layer table cache and kernel dispatch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <tuple>
#include <unordered_map>

#include <nvtx3/nvToolsExt.h>

#include "are_internal.cuh"

namespace are {

namespace {
thread_local std::unordered_map<const are_ctx *, std::string> t_errors;
}

void set_error(const are_ctx *ctx, const std::string &msg) { t_errors[ctx] = msg; }

namespace {

// Runs fn, mapping exceptions to a status and a thread-local message.
template <typename F>
are_status guarded(are_ctx *ctx, F &&fn)
{
    if (!ctx) return ARE_EINVAL;
    std::lock_guard<std::recursive_mutex> lock(ctx->mu);
    t_errors[ctx].clear();
    try {
        ARE_CUDA_TRY(cudaSetDevice(ctx->device));
        fn();
        return ARE_OK;
    } catch (const Error &e) {
        set_error(ctx, e.msg);
        return e.code;
    } catch (const std::bad_alloc &) {
        set_error(ctx, "host allocation failed");
        return ARE_ENOMEM;
    }
}

bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// The stream a call runs on.  A caller's stream is used as given and the call
// only enqueues work.  NULL means: wait for all earlier work on the device
// (the caller's inputs may come from any stream), run on the context's own
// stream, and finish before returning.
// NVTX range over one library call (named in profilers' timelines; free
// when no profiler is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

struct CallStream {
    cudaStream_t s;
    bool own;
    CallStream(are_ctx *ctx, void *user)
    {
        own = user == nullptr;
        if (own) ARE_CUDA_TRY(cudaDeviceSynchronize());
        s = own ? ctx->stream : static_cast<cudaStream_t>(user);
    }
    void finish() const
    {
        if (own) ARE_CUDA_TRY(cudaStreamSynchronize(s));
    }
};

// Device inputs of the load calls may still be in flight on another stream.
void fence_device_inputs(std::initializer_list<const void *> ptrs)
{
    for (const void *p : ptrs)
        if (is_device_ptr(p)) {
            ARE_CUDA_TRY(cudaDeviceSynchronize());
            return;
        }
}

// Device allocation charged to the context's budget.  Blocks the library
// releases are kept in a per-context cache and handed out again for requests
// of up to 5/4 of their size (cudaMalloc and cudaFree of gigabyte blocks cost
// milliseconds and cudaFree synchronises the device); the cache is emptied
// when an allocation fails or the budget needs the room, and at are_destroy.
void release_cache(are_ctx *ctx)
{
    for (auto &kv : ctx->cache) {
        ctx->block_size.erase(kv.second);
        cudaFree(kv.second);
    }
    ctx->cache.clear();
    ctx->cached = 0;
}

void *dalloc(are_ctx *ctx, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    ARE_CHECK(ctx->budget == 0 || ctx->used + bytes <= ctx->budget, ARE_ENOMEM,
              "memory budget exceeded: need " + std::to_string(bytes) + " bytes, " +
                  std::to_string(ctx->budget - ctx->used) + " left");
    auto it = ctx->cache.lower_bound(bytes);
    if (it != ctx->cache.end() && it->first <= bytes + bytes / 4) {
        void *p = it->second;
        ctx->cached -= it->first;
        ctx->cache.erase(it);
        ctx->used += bytes;
        return p;
    }
    if (ctx->budget && ctx->used + ctx->cached + bytes > ctx->budget) release_cache(ctx);
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e == cudaErrorMemoryAllocation && !ctx->cache.empty()) {
        cudaGetLastError();
        release_cache(ctx);
        e = cudaMalloc(&p, bytes);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw Error{e == cudaErrorMemoryAllocation ? ARE_ENOMEM : ARE_ECUDA,
                    std::string("cudaMalloc: ") + cudaGetErrorString(e)};
    }
    ctx->block_size[p] = bytes;
    ctx->used += bytes;
    return p;
}

// Returns a block to the cache once no device work can still use it (the
// same device-wide wait that cudaFree makes).
void dfree(are_ctx *ctx, void *p, size_t bytes)
{
    if (!p) return;
    if (bytes == 0) bytes = 16;
    ctx->used -= std::min(ctx->used, bytes);
    auto it = ctx->block_size.find(p);
    if (it == ctx->block_size.end()) {   // not from dalloc
        cudaFree(p);
        return;
    }
    cudaDeviceSynchronize();
    ctx->cache.emplace(it->second, p);
    ctx->cached += it->second;
}

// Copy n bytes from src (host or device) into device memory dst.
void copy_in(void *dst, const void *src, size_t n, cudaStream_t s)
{
    if (n == 0) return;
    ARE_CUDA_TRY(cudaMemcpyAsync(dst, src, n, cudaMemcpyDefault, s));
}

template <typename T>
std::vector<T> to_host(const T *src, size_t n, cudaStream_t s)
{
    std::vector<T> v(n);
    if (n == 0) return v;
    if (is_device_ptr(src)) {
        ARE_CUDA_TRY(cudaMemcpyAsync(v.data(), src, n * sizeof(T), cudaMemcpyDeviceToHost, s));
        ARE_CUDA_TRY(cudaStreamSynchronize(s));
    } else {
        std::memcpy(v.data(), src, n * sizeof(T));
    }
    return v;
}

bool nonneg_finite(double x) { return std::isfinite(x) && x >= 0.0; }
bool nonneg_limit(double x) { return !std::isnan(x) && x >= 0.0; }

// A layer's terms with -0.0 read as +0.0: the kernels compare non-negative
// doubles by their bit patterns.
are_layer_terms positive_zeros(are_layer_terms t)
{
    for (double *x : {&t.occ_ret, &t.occ_lim, &t.agg_ret, &t.agg_lim})
        if (*x == 0.0) *x = 0.0;
    return t;
}

int check_flag(are_ctx *ctx, cudaStream_t s)
{
    ARE_CUDA_TRY(cudaMemcpyAsync(ctx->h_flag, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    ARE_CUDA_TRY(cudaStreamSynchronize(s));
    return *ctx->h_flag;
}

void free_table(are_ctx *ctx, Table &t)
{
    dfree(ctx, t.d, t.bytes);
    t = Table{};
}

void free_packed(are_ctx *ctx, Packed &p)
{
    dfree(ctx, p.d, p.bytes);
    p = Packed{};
}

void free_folded(are_ctx *ctx, Folded &f)
{
    dfree(ctx, f.d, f.bytes);
    f = Folded{};
}

// Build (or rebuild) the layer's table for `catalog` in fp32 or fp64.
ScatterArgs scatter_args(are_ctx *ctx, const Layer &L, int32_t catalog, int jp)
{
    ScatterArgs a{};
    a.n_elts = (int32_t)L.elts.size();
    a.jp = jp;
    for (size_t j = 0; j < L.elts.size(); ++j) {
        const Elt &e = ctx->elts.at(L.elts[j]);
        ARE_CHECK(e.max_id < catalog, ARE_EINVAL,
                  "ELT " + std::to_string(L.elts[j]) + " holds event id " + std::to_string(e.max_id) +
                      " outside the YET's catalog of " + std::to_string(catalog));
        a.ids[j] = e.d_ids;
        a.loss[j] = e.d_loss;
        a.n[j] = e.n;
        a.fx[j] = e.terms.fx;
        a.ded[j] = e.terms.deductible;
        a.lim[j] = e.terms.limit;
        a.share[j] = e.terms.share;
    }
    return a;
}

// (Re)allocate table t for catalog x jp columns of elem bytes.
void size_table(are_ctx *ctx, Layer &L, Table &t, int32_t catalog, int jp, size_t elem)
{
    const size_t bytes = (size_t)catalog * jp * elem;
    if (t.d && (t.catalog != catalog || t.jp != jp)) free_table(ctx, t);
    if (!t.d) {
        ++L.generation;
        t.d = dalloc(ctx, bytes);
        t.bytes = bytes;
        t.catalog = catalog;
        t.jp = jp;
    }
}

void free_compact(are_ctx *ctx, Compact &c)
{
    dfree(ctx, c.d, c.bytes);
    c = Compact{};
}

// Build (or rebuild) the layer's compact FP32 table for `catalog`: room for
// as many rows as the ELTs hold entries (or the catalog, if smaller).
Compact &build_compact(are_ctx *ctx, Layer &L, int32_t catalog, cudaStream_t s)
{
    Compact &c = L.comp;
    const int jp = table_jp((int)L.elts.size(), true);
    const ScatterArgs a = scatter_args(ctx, L, catalog, jp);
    int64_t entries = 0;
    for (int j = 0; j < a.n_elts; ++j) entries += a.n[j];
    const int64_t max_rows = std::max<int64_t>(1, std::min<int64_t>(catalog, entries));
    if (c.d && (c.catalog != catalog || c.jp != jp || c.max_rows < max_rows)) free_compact(ctx, c);
    if (!c.d) {
        ++L.generation;
        auto up256 = [](size_t x) { return (x + 255) & ~(size_t)255; };
        c.counts_off = up256(sizeof(int32_t) * (size_t)catalog);
        c.rows_off = c.counts_off + up256(sizeof(int32_t) * (size_t)compact_scan_blocks(catalog));
        c.bytes = c.rows_off + sizeof(float) * (size_t)max_rows * jp;
        c.d = dalloc(ctx, c.bytes);
        c.catalog = catalog;
        c.jp = jp;
        c.max_rows = max_rows;
    }
    ctx->launches += launch_build_compact(c.row_of(), c.counts(), c.rows(),
                                          sizeof(float) * (size_t)c.max_rows * jp, catalog, a, s);
    return c;
}

// The tables an analysis of layer L in `precision` reads, built if missing.
void ensure_tables(are_ctx *ctx, Layer &L, const Yet &y, are_precision precision, cudaStream_t s,
                   bool rebuild);
TuneEntry tuned(are_ctx *ctx, are_precision p, const Yet &y, int jp, bool multi);

// Build (or rebuild) the layer's table for `catalog` in fp32 or fp64.
Table &build_table(are_ctx *ctx, Layer &L, int32_t catalog, bool fp32, cudaStream_t s)
{
    Table &t = fp32 ? L.t32 : L.t64;
    const int jp = table_jp((int)L.elts.size(), fp32);
    const ScatterArgs a = scatter_args(ctx, L, catalog, jp);
    size_table(ctx, L, t, catalog, jp, fp32 ? 4 : 8);
    ARE_CUDA_TRY(cudaMemsetAsync(t.d, 0, t.bytes, s));
    ctx->launches += launch_scatter_table(t.d, fp32, a, s);
    return t;
}

// The FP32 screen of the layer's FP64 table (values rounded up), read by the
// screened FP64 kernel only: built when that kernel is the tuned choice, so
// the other FP64 kernels do not pay for it (its 64 MB would also push the
// FP64 table out of L2 before the analysis).
Table &build_screen(are_ctx *ctx, Layer &L, int32_t catalog, cudaStream_t s)
{
    Table &u = L.t32u;
    const int jp = table_jp((int)L.elts.size(), true);
    const ScatterArgs a = scatter_args(ctx, L, catalog, jp);
    size_table(ctx, L, u, catalog, jp, 4);
    ARE_CUDA_TRY(cudaMemsetAsync(u.d, 0, u.bytes, s));
    ctx->launches += launch_scatter_table(u.d, true, a, s, true);
    return u;
}

// (Re)allocates packed table p for `catalog` rows of `row_bytes` and an
// overflow of `ovf_bytes`.
void size_packed(are_ctx *ctx, Layer &L, Packed &p, int32_t catalog, int rw, size_t row_bytes,
                 size_t ovf_bytes)
{
    const size_t rows_bytes = (size_t)catalog * row_bytes;
    const size_t need = rows_bytes + 256 + std::max<size_t>(ovf_bytes, 8);
    if (p.d && (p.catalog != catalog || p.rw != rw || p.bytes < need)) free_packed(ctx, p);
    if (!p.d) {
        ++L.generation;
        p.d = dalloc(ctx, need);
        p.bytes = need;
        p.rows_bytes = rows_bytes;
        p.catalog = catalog;
        p.rw = rw;
    }
}

int64_t layer_entries(are_ctx *ctx, const Layer &L)
{
    int64_t entries = 0;
    for (int32_t h : L.elts) entries += ctx->elts.at(h).n;
    ARE_CHECK(entries < (1LL << 32), ARE_EINVAL, "a layer's ELTs hold 2^32 or more entries");
    return entries;
}

// Words per packed row of the layer over a catalog of `catalog` events (0:
// the dense FP32 row), from its ELT entries per catalog event.
int row_words(are_ctx *ctx, const Layer &L, int32_t catalog, bool fp32)
{
    const double tpe = catalog > 0 ? (double)layer_entries(ctx, L) / (double)catalog : 0.0;
    return packed_row_words((int)L.elts.size(), tpe, fp32);
}

// The packed FP64 rows of the layer, built straight from its ELT entries (no
// dense table), read by the FP64 register-rows kernel.
Packed &build_packed64(are_ctx *ctx, Layer &L, int32_t catalog, cudaStream_t s)
{
    Packed &p = L.p64;
    const int rw = row_words(ctx, L, catalog, false);
    size_packed(ctx, L, p, catalog, rw, rw * sizeof(unsigned long long),
                sizeof(double) * (size_t)layer_entries(ctx, L));
    const ScatterArgs a = scatter_args(ctx, L, catalog, table_jp((int)L.elts.size(), false));
    ctx->launches += launch_pack64_direct(a, catalog, rw, static_cast<unsigned long long *>(p.rows()),
                                          static_cast<double *>(p.ovf()), p.used(), s);
    return p;
}

// The packed FP32 rows (pw words each) built straight from the layer's ELT
// entries, with no dense table: what the FP32 register-rows kernel reads.
Packed &build_packed32_direct(are_ctx *ctx, Layer &L, int32_t catalog, int pw, cudaStream_t s)
{
    Packed &p = L.p32;
    const ScatterArgs a = scatter_args(ctx, L, catalog, table_jp((int)L.elts.size(), true));
    size_packed(ctx, L, p, catalog, pw, pw * sizeof(float), sizeof(float) * (size_t)layer_entries(ctx, L));
    ctx->launches += launch_pack32_direct(a, catalog, pw, static_cast<uint32_t *>(p.rows()),
                                          static_cast<float *>(p.ovf()), p.used(), s);
    return p;
}

// The table beside a layer's dense FP64 table that a kernel choice reads:
// the FP32 screen (kernel 3).  `fresh`: the layer's table was just rebuilt.
// (The packed rows of the register-rows kernels are built from the ELT
// entries: build_packed32_direct, build_packed64.)
void ensure_aux(are_ctx *ctx, Layer &L, int32_t catalog, bool fp32, int kernel, bool fresh, cudaStream_t s)
{
    if (!fp32 && kernel == 3 && (fresh || !L.t32u.d || L.t32u.catalog != catalog)) build_screen(ctx, L, catalog, s);
}

// The packed rows a register-rows analysis (kernel 2) of the layer reads,
// built if missing (or always, with rebuild); false where it reads the
// dense FP32 table instead.
bool ensure_packed(are_ctx *ctx, Layer &L, int32_t catalog, bool fp32, cudaStream_t s, bool rebuild)
{
    const int w = row_words(ctx, L, catalog, fp32);
    if (!w) return false;
    Packed &p = fp32 ? L.p32 : L.p64;
    if (rebuild || !p.d || p.catalog != catalog || p.rw != w) {
        if (fp32)
            build_packed32_direct(ctx, L, catalog, w, s);
        else
            build_packed64(ctx, L, catalog, s);
    }
    return true;
}

void ensure_tables(are_ctx *ctx, Layer &L, const Yet &y, are_precision precision, cudaStream_t s,
                   bool rebuild)
{
    const bool fp32 = precision != ARE_FP64;
    const int32_t catalog = y.catalog;
    if (fp32 && L.layout == ARE_LAYOUT_COMPACT) {
        if (rebuild || !L.comp.d || L.comp.catalog != catalog) build_compact(ctx, L, catalog, s);
        return;
    }
    const int jp = table_jp((int)L.elts.size(), fp32);
    const int kernel = tuned(ctx, precision, y, jp, false).kernel;
    // packed rows straight from the ELT entries; a dense table only when a kernel needs one
    if (kernel == 2 && ensure_packed(ctx, L, catalog, fp32, s, rebuild)) return;
    const Table &t = fp32 ? L.t32 : L.t64;
    const bool fresh = rebuild || !t.d || t.catalog != catalog;
    if (fresh) build_table(ctx, L, catalog, fp32, s);
    ensure_aux(ctx, L, catalog, fp32, kernel, fresh, s);
}

Layer &layer_of(are_ctx *ctx, int32_t h)
{
    auto it = ctx->layers.find(h);
    if (it == ctx->layers.end()) throw Error{ARE_ENOTFOUND, "unknown layer handle " + std::to_string(h)};
    return it->second;
}
Yet &yet_of(are_ctx *ctx, int32_t h)
{
    auto it = ctx->yets.find(h);
    if (it == ctx->yets.end()) throw Error{ARE_ENOTFOUND, "unknown YET handle " + std::to_string(h)};
    return it->second;
}

void check_precision(are_precision p)
{
    ARE_CHECK(p == ARE_FP64 || p == ARE_FP32_KAHAN || p == ARE_FP32_FP64AGG, ARE_EINVAL,
              "unknown precision " + std::to_string((int)p));
}

void fill_terms(const Layer &L, TermsF32 &t32, TermsF64 &t64)
{
    t64.occ_r = L.terms.occ_ret;
    t64.occ_l = L.terms.occ_lim;
    t32.occ_r = (float)L.terms.occ_ret;
    t32.occ_l = (float)L.terms.occ_lim;
}

// (Re)build the layer's folded table for `catalog` from its ELTs.
Folded &build_folded(are_ctx *ctx, Layer &L, int32_t catalog, cudaStream_t s)
{
    Folded &f = L.fold;
    const int32_t words = folded_words(catalog);
    if (f.d && f.catalog != catalog) free_folded(ctx, f);
    if (!f.d) {
        f.words = words;
        f.bytes = 256 + (((size_t)words * 4 + 255) & ~(size_t)255) + (size_t)catalog * 16;
        f.d = dalloc(ctx, f.bytes);
        f.catalog = catalog;
    }
    const ScatterArgs a = scatter_args(ctx, L, catalog, 0);
    ctx->launches += launch_fold(a, L.terms.occ_ret, L.terms.occ_lim, catalog, f.F(), f.bits(),
                                 f.hmax(), ctx->num_sms, s);
    return f;
}

void fill_layer_f32(const Layer &L, LayerF32 &o)
{
    std::memset(&o, 0, sizeof o);
    o.table = static_cast<const float *>(L.t32.d);
    o.jp = L.t32.jp;
    o.occ_r = (float)L.terms.occ_ret;
    o.occ_l = (float)L.terms.occ_lim;
    o.agg_r = L.terms.agg_ret;
    o.agg_l = L.terms.agg_lim;
}

// Key of the tuning table: precision, YET layout, widest table row, mean
// events per trial (power-of-two bucket) and one layer vs several.
std::string tune_key(are_precision p, const Yet &y, int jp, bool multi)
{
    const double mean = y.n_trials ? (double)y.n_events / (double)y.n_trials : 0.0;
    int bucket = 1;
    while (bucket < mean && bucket < (1 << 20)) bucket <<= 1;
    return "p" + std::to_string((int)p) + (y.d_off ? "_ragged" : "_fixed") + "_jp" +
           std::to_string(jp) + "_ev" + std::to_string(bucket) + (multi ? "_multi" : "_single");
}

ItemWork item_work(const Yet &y, int64_t trial_begin, int64_t n_trials, const ItemConfig &cfg)
{
    ItemWork w;
    std::memset(&w, 0, sizeof w);
    w.ids = y.d_ids;
    w.off = y.d_off;
    w.k = y.k;
    w.trial_begin = trial_begin;
    w.n_trials = n_trials;
    w.trials_per_item = cfg.trials_per_item > 0 ? cfg.trials_per_item : 8;
    return w;
}

// The fixed-point scale of the FP64 register-rows kernel's exact running
// sums: s = 125 - floor(log2(B)) for an upper bound B of every occurrence
// loss of the layer -- min(OccL, the sum over its ELTs of the largest term),
// the largest term being the term of the ELT's largest loss (a term is
// non-decreasing in the loss), with a margin for the rounding of that sum.
int fixed_scale(are_ctx *ctx, const Layer &L)
{
    double g = 0.0;
    for (int32_t h : L.elts) {
        const Elt &e = ctx->elts.at(h);
        if (e.n == 0) continue;
        double x = e.terms.fx * e.max_loss - e.terms.deductible;
        x = x > 0.0 ? x : 0.0;
        x = x > e.terms.limit ? e.terms.limit : x;
        g += e.terms.share * x;
    }
    double b = std::min(g, L.terms.occ_lim) * (1.0 + 1e-9);
    if (!(b > 0.0)) return 0;
    int ex = 0;
    std::frexp(b, &ex);          // b = f * 2^ex, 0.5 <= f < 1: floor(log2 b) = ex - 1
    return 125 - (ex - 1);
}

// One layer's analysis stage with a given kernel choice.
int run_single(are_ctx *ctx, const Layer &L, const Yet &y, int64_t trial_begin, int64_t n_trials,
               are_precision precision, double *d_out, const TuneEntry &te, cudaStream_t s)
{
    const bool fp32 = precision != ARE_FP64;
    if (fp32 && te.kernel == 0) {
        ItemWork w = item_work(y, trial_begin, n_trials, te.cfg);
        fill_layer_f32(L, w.one);
        w.one.ylt = d_out;
        w.one.t0 = 0;
        w.one.nt = n_trials;
        w.n_layers = 1;
        w.n_items = (n_trials + w.trials_per_item - 1) / w.trials_per_item;
        return launch_items(w, L.t32.jp, te.cfg, precision, ctx->num_sms, s);
    }
    const bool compact = fp32 && L.layout == ARE_LAYOUT_COMPACT && L.comp.d && L.comp.catalog == y.catalog;
    const Table &t = fp32 ? L.t32 : L.t64;
    SimArgs a{};
    a.ids = y.d_ids;
    a.off = y.d_off;
    a.k = y.k;
    a.trial_begin = trial_begin;
    a.n_trials = n_trials;
    a.table = t.d;
    a.agg_r = L.terms.agg_ret;
    a.agg_l = L.terms.agg_lim;
    a.ylt = d_out;
    a.kernel = te.kernel;
    a.epl = te.cfg.rows_in_flight;   // 0 (untuned): the kernel's default
    TermsF32 t32;
    TermsF64 t64;
    fill_terms(L, t32, t64);
    a.n_elts = (int32_t)L.elts.size();
    if (fp32 && !compact && te.kernel == 2 && L.p32.d && L.p32.catalog == y.catalog &&
        L.p32.rw == row_words(ctx, L, y.catalog, true)) {
        a.table = L.p32.rows();   // register rows over the packed FP32 rows
        a.table2 = L.p32.ovf();
        a.kernel = 5;
        return launch_simulate(a, precision, L.p32.rw, &t32, &t64, ctx->num_sms, s);
    }
    if (compact) {   // the staged kernel, through the row index
        a.table = L.comp.rows();
        a.table2 = L.comp.row_of();
        a.kernel = 4;
        return launch_simulate(a, precision, L.comp.jp, &t32, &t64, ctx->num_sms, s);
    }
    if (!fp32) {
        if (te.kernel == 2 && L.p64.d && L.p64.catalog == y.catalog) {   // packed FP64 rows
            a.table = L.p64.rows();
            a.table2 = L.p64.ovf();
            return launch_rows64(a, L.p64.rw, t64, fixed_scale(ctx, L), ctx->num_sms, s);
        }
        if (te.kernel == 3 && L.t32u.d && L.t32u.catalog == y.catalog) {   // the FP32 screen
            a.table2 = L.t32u.d;
            a.jp64 = t.jp;
            return launch_screen64(a, L.t32u.jp, t64, ctx->num_sms, s);
        }
        return launch_staged64(a, t.jp, t64, ctx->num_sms, s);   // (or an aux table not built)
    }
    return launch_simulate(a, precision, t.jp, &t32, &t64, ctx->num_sms, s);
}

TuneEntry tuned(are_ctx *ctx, are_precision p, const Yet &y, int jp, bool multi)
{
    auto it = ctx->tune.find(tune_key(p, y, jp, multi));
    if (it != ctx->tune.end()) return it->second;
    TuneEntry d;   // untuned: the register-rows kernels with their default batch
    d.kernel = 2;
    d.cfg.rows_in_flight = 0;
    return d;
}

int64_t rank_rp(int64_t n, double rp)
{
    const int64_t m = rank_for_return_period(n, rp);
    ARE_CHECK(m >= 1, ARE_EINVAL, "return period must be finite and >= 1");
    return m;
}
int64_t rank_level(int64_t n, double a)
{
    const int64_t m = rank_for_level(n, a);
    ARE_CHECK(m >= 1, ARE_EINVAL, "TVaR level must be finite and lie in (0, 1)");
    return m;
}

}  // namespace

// Integer ranks of the risk measures (the definitions in include/are.h).
int64_t rank_for_return_period(int64_t n, double rp)
{
    if (!std::isfinite(rp) || rp > 1e12) return -1;
    const long long micro = std::llround(rp * 1e6);
    if (micro < 1000000) return -1;
    return (n * 1000000 + micro - 1) / micro;
}
int64_t rank_for_level(int64_t n, double a)
{
    if (!std::isfinite(a)) return -1;
    const long long nano = std::llround(a * 1e9);
    if (nano <= 0 || nano >= 1000000000) return -1;
    return (n * (1000000000 - nano) + 999999999) / 1000000000;
}

namespace {

void free_plan(are_ctx *ctx, Plan &p)
{
    if (p.exec) cudaGraphExecDestroy(p.exec);
    if (p.graph) cudaGraphDestroy(p.graph);
    dfree(ctx, p.d_work, p.work_bytes);
    p = Plan{};
}

constexpr int kWidths[3] = {8, 16, 32};

// Layers of a multi-layer launch grouped by FP32 table width: group g holds
// the LayerF32 records of width kWidths[g] at d_work + offset[g].
struct Groups {
    std::vector<LayerF32> rec[3];
    size_t offset[3] = {0, 0, 0};
    size_t counters = 0;
    size_t bytes = 0;
};

Groups group_layers(are_ctx *ctx, const std::vector<int32_t> &layers,
                    const std::vector<double *> &ylts, int64_t n_trials, int tpi)
{
    Groups g;
    for (size_t i = 0; i < layers.size(); ++i) {
        const Layer &L = ctx->layers.at(layers[i]);
        LayerF32 r;
        fill_layer_f32(L, r);
        r.ylt = ylts[i];
        const int gi = r.jp == 8 ? 0 : r.jp == 16 ? 1 : 2;
        r.item_begin = 0;
        g.rec[gi].push_back(r);
    }
    const int64_t per_layer = (n_trials + tpi - 1) / tpi;
    size_t off = 0;
    for (int gi = 0; gi < 3; ++gi) {
        int64_t next = 0;
        for (LayerF32 &r : g.rec[gi]) {
            r.item_begin = next;
            r.t0 = 0;
            r.nt = n_trials;
            next += per_layer;
        }
        g.offset[gi] = off;
        off += (sizeof(LayerF32) * g.rec[gi].size() + 255) / 256 * 256;
    }
    g.counters = off;
    g.bytes = off + 3 * sizeof(unsigned long long);
    return g;
}

// Enqueues the analysis stage of several layers.  FP32: one persistent
// launch per table width over a device work list at d_work (which must hold
// the Groups layout); FP64: one launch per layer.
int enqueue_multi(are_ctx *ctx, const std::vector<int32_t> &layers,
                  const std::vector<double *> &ylts, const Yet &y, int64_t trial_begin,
                  int64_t n_trials, are_precision prec, const TuneEntry &te, const Groups *g,
                  void *d_work, cudaStream_t s)
{
    int launches = 0;
    if (prec == ARE_FP64 || te.kernel != 0) {
        // one single-layer launch per layer, back to back (one table hot in L2 at a time)
        for (size_t i = 0; i < layers.size(); ++i)
            launches += run_single(ctx, ctx->layers.at(layers[i]), y, trial_begin, n_trials, prec,
                                   ylts[i], te, s);
        return launches;
    }
    unsigned char *base = static_cast<unsigned char *>(d_work);
    for (int gi = 0; gi < 3; ++gi) {
        if (g->rec[gi].empty()) continue;
        ItemWork w = item_work(y, trial_begin, n_trials, te.cfg);
        w.layers = reinterpret_cast<const LayerF32 *>(base + g->offset[gi]);
        w.n_layers = (int32_t)g->rec[gi].size();
        w.n_items = (int64_t)g->rec[gi].size() * ((n_trials + w.trials_per_item - 1) / w.trials_per_item);
        w.counter = reinterpret_cast<unsigned long long *>(base + g->counters) + gi;
        ARE_CUDA_TRY(cudaMemsetAsync(w.counter, 0, sizeof(unsigned long long), s));
        launches += launch_items(w, kWidths[gi], te.cfg, prec, ctx->num_sms, s);
    }
    return launches;
}

void check_multi_args(are_ctx *ctx, const int32_t *layers, int32_t n_layers, const Yet &y,
                      int64_t trial_begin, int64_t n_trials, double *const *ylts)
{
    ARE_CHECK(layers && n_layers >= 1, ARE_EINVAL, "need at least one layer");
    ARE_CHECK(trial_begin >= 0 && n_trials >= 1 && trial_begin + n_trials <= y.n_trials, ARE_EINVAL,
              "trial range outside the YET");
    for (int32_t i = 0; i < n_layers; ++i) {
        layer_of(ctx, layers[i]);
        if (ylts) {
            ARE_CHECK(ylts[i] && is_device_ptr(ylts[i]), ARE_EINVAL,
                      "every YLT of a multi-layer launch must be device memory");
        }
    }
}

// Every layer's table and the tables beside it that `kernel` reads (0: none).
void ensure_tables(are_ctx *ctx, const int32_t *layers, int32_t n_layers, const Yet &y, bool fp32,
                   cudaStream_t s, int kernel = 0)
{
    for (int32_t i = 0; i < n_layers; ++i) {
        Layer &L = layer_of(ctx, layers[i]);
        if (kernel == 2 && ensure_packed(ctx, L, y.catalog, fp32, s, false)) continue;   // packed rows
        const Table &t = fp32 ? L.t32 : L.t64;
        const bool fresh = !t.d || t.catalog != y.catalog;
        if (fresh) build_table(ctx, L, y.catalog, fp32, s);
        ensure_aux(ctx, L, y.catalog, fp32, kernel, fresh, s);
    }
}

int max_width(are_ctx *ctx, const int32_t *layers, int32_t n_layers, bool fp32)
{
    int jp = 0;
    for (int32_t i = 0; i < n_layers; ++i)
        jp = std::max(jp, table_jp((int)layer_of(ctx, layers[i]).elts.size(), fp32));
    return jp;
}

}  // namespace

int fit_blocks(const void *kern, int threads, size_t smem)
{
    static std::mutex mu;
    static std::map<std::tuple<const void *, int, int, size_t>, int> known;
    int dev = 0;
    ARE_CUDA_TRY(cudaGetDevice(&dev));
    const auto key = std::make_tuple(kern, dev, threads, smem);
    std::lock_guard<std::mutex> lock(mu);
    auto it = known.find(key);
    if (it != known.end()) return it->second;
    if (smem > 48 * 1024)
        ARE_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    ARE_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    if (per_sm < 1) per_sm = 1;
    known[key] = per_sm;
    return per_sm;
}

void *ctx_alloc(are_ctx *ctx, size_t bytes) { return dalloc(ctx, bytes); }
void ctx_free(are_ctx *ctx, void *p, size_t bytes) { dfree(ctx, p, bytes); }

}  // namespace are

using namespace are;

extern "C" {

are_status are_create(are_ctx **out, int device, size_t mem_budget_bytes)
{
    if (!out) return ARE_EINVAL;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return ARE_ECUDA;
    }
    are_ctx *ctx = new (std::nothrow) are_ctx();
    if (!ctx) return ARE_ENOMEM;
    ctx->device = device;
    ctx->budget = mem_budget_bytes;
    are_status st = guarded(ctx, [&] {
        ARE_CUDA_TRY(cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device));
        ARE_CUDA_TRY(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
        ARE_CUDA_TRY(cudaStreamCreateWithFlags(&ctx->capture, cudaStreamNonBlocking));
        ARE_CUDA_TRY(cudaMalloc(&ctx->d_flag, sizeof(int)));
        ARE_CUDA_TRY(cudaMallocHost(&ctx->h_flag, sizeof(int)));
        ARE_CUDA_TRY(cudaMallocHost(&ctx->h_result, sizeof(double) * 2 * kMaxTargets));
        select_alloc(ctx->sel, ctx->num_sms);
    });
    if (st != ARE_OK) {
        are_destroy(ctx);
        return st;
    }
    *out = ctx;
    return ARE_OK;
}

are_status are_destroy(are_ctx *ctx)
{
    if (!ctx) return ARE_OK;
    server_destroy(ctx);   // before taking the lock: its thread may be waiting for it
    {
        std::lock_guard<std::recursive_mutex> lock(ctx->mu);
        cudaSetDevice(ctx->device);
        if (ctx->stream) cudaStreamSynchronize(ctx->stream);
        for (auto &kv : ctx->layers) {
            free_table(ctx, kv.second.t32);
            free_table(ctx, kv.second.t64);
            free_table(ctx, kv.second.t32u);
            free_packed(ctx, kv.second.p64);
            free_packed(ctx, kv.second.p32);
            free_folded(ctx, kv.second.fold);
            free_compact(ctx, kv.second.comp);
        }
        for (auto &kv : ctx->elts) {
            dfree(ctx, kv.second.d_ids, 0);
            dfree(ctx, kv.second.d_loss, 0);
        }
        for (auto &kv : ctx->yets) {
            dfree(ctx, kv.second.d_ids, 0);
            dfree(ctx, kv.second.d_off, 0);
        }
        for (auto &p : ctx->plans) free_plan(ctx, p);
        ctx->plans.clear();
        if (ctx->d_multi) cudaFree(ctx->d_multi);
        if (ctx->h_multi) cudaFreeHost(ctx->h_multi);
        if (ctx->capture) cudaStreamDestroy(ctx->capture);
        select_free(ctx->sel);
        if (ctx->d_flag) cudaFree(ctx->d_flag);
        if (ctx->h_flag) cudaFreeHost(ctx->h_flag);
        if (ctx->h_result) cudaFreeHost(ctx->h_result);
        release_cache(ctx);
        if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
        if (ctx->stream) cudaStreamDestroy(ctx->stream);
        t_errors.erase(ctx);
    }
    delete ctx;
    return ARE_OK;
}

const char *are_last_error(const are_ctx *ctx)
{
    if (!ctx) return static_last_error();
    auto it = t_errors.find(ctx);
    return it == t_errors.end() ? "" : it->second.c_str();
}

are_status are_memory_used(const are_ctx *ctx, size_t *bytes)
{
    if (!ctx || !bytes) return ARE_EINVAL;
    *bytes = ctx->used;
    return ARE_OK;
}

are_status are_launch_count(const are_ctx *ctx, uint64_t *launches)
{
    if (!ctx || !launches) return ARE_EINVAL;
    *launches = ctx->launches;
    return ARE_OK;
}

are_status are_load_yet(are_ctx *ctx, int32_t catalog_size, int64_t n_trials,
                        const int64_t *offsets, int32_t events_per_trial,
                        const int32_t *event_ids, const float *timestamps, int32_t *yet_handle)
{
    return guarded(ctx, [&] {
        NvtxRange nvtx("are_load_yet");
        ARE_CHECK(yet_handle, ARE_EINVAL, "yet_handle is NULL");
        ARE_CHECK(catalog_size > 0, ARE_EINVAL, "catalog_size must be > 0");
        ARE_CHECK(n_trials >= 0 && n_trials < (int64_t)INT32_MAX, ARE_EINVAL,
                  "n_trials must lie in 0 .. 2^31 - 2");
        ARE_CHECK(offsets || events_per_trial > 0, ARE_EINVAL,
                  "need offsets or events_per_trial > 0");
        fence_device_inputs({offsets, event_ids, timestamps});
        cudaStream_t s = ctx->stream;
        Yet y;
        y.catalog = catalog_size;
        y.n_trials = n_trials;
        y.k = offsets ? 0 : events_per_trial;
        auto cleanup = [&] {
            dfree(ctx, y.d_ids, y.bytes);
            dfree(ctx, y.d_off, y.d_off ? sizeof(int64_t) * (n_trials + 1) : 0);
        };
        try {
            if (offsets) {
                int64_t last = 0;
                ARE_CUDA_TRY(cudaMemcpyAsync(&last, offsets + n_trials, sizeof(int64_t),
                                             cudaMemcpyDefault, s));
                ARE_CUDA_TRY(cudaStreamSynchronize(s));
                ARE_CHECK(last >= 0, ARE_EINVAL, "offsets[n_trials] must be >= 0");
                y.n_events = last;
                y.d_off = (int64_t *)dalloc(ctx, sizeof(int64_t) * (n_trials + 1));
                copy_in(y.d_off, offsets, sizeof(int64_t) * (n_trials + 1), s);
            } else {
                y.n_events = n_trials * (int64_t)events_per_trial;
            }
            ARE_CHECK(y.n_events == 0 || event_ids, ARE_EINVAL, "event_ids is NULL");
            y.bytes = sizeof(int32_t) * (y.n_events + kIdPad);
            y.d_ids = (int32_t *)dalloc(ctx, y.bytes);
            copy_in(y.d_ids, event_ids, sizeof(int32_t) * y.n_events, s);
            ARE_CUDA_TRY(cudaMemsetAsync(y.d_ids + y.n_events, 0, sizeof(int32_t) * kIdPad, s));
            ARE_CUDA_TRY(cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), s));
            if (y.d_off)
                ctx->launches += launch_check_offsets(y.d_off, n_trials, y.n_events, ctx->d_flag, s);
            ctx->launches += launch_check_ids(y.d_ids, y.n_events, catalog_size, ctx->d_flag, s);
            int f = check_flag(ctx, s);
            ARE_CHECK(!(f & 2), ARE_EINVAL,
                      "offsets must start at 0, be non-decreasing and end at the event count");
            ARE_CHECK(!(f & 1), ARE_EINVAL, "event id outside [0, catalog_size)");
            if (timestamps && y.n_events > 0) {
                float *d_ts = (float *)dalloc(ctx, sizeof(float) * y.n_events);
                try {
                    copy_in(d_ts, timestamps, sizeof(float) * y.n_events, s);
                    ctx->launches +=
                        launch_check_timestamps(d_ts, y.d_off, n_trials, y.k, ctx->d_flag, s);
                    f = check_flag(ctx, s);
                } catch (...) {
                    dfree(ctx, d_ts, sizeof(float) * y.n_events);
                    throw;
                }
                dfree(ctx, d_ts, sizeof(float) * y.n_events);
                ARE_CHECK(!(f & 4), ARE_EINVAL, "timestamps must be non-decreasing within each trial");
            }
            ARE_CUDA_TRY(cudaStreamSynchronize(s));
        } catch (...) {
            cleanup();
            throw;
        }
        const int32_t h = ctx->next_handle++;
        ctx->yets[h] = y;
        *yet_handle = h;
    });
}

are_status are_load_elt(are_ctx *ctx, int32_t n_entries, const int32_t *event_ids,
                        const double *losses, const are_fin_terms *terms, int32_t *elt_handle)
{
    return guarded(ctx, [&] {
        NvtxRange nvtx("are_load_elt");
        ARE_CHECK(elt_handle && terms, ARE_EINVAL, "elt_handle and terms must not be NULL");
        ARE_CHECK(n_entries >= 0, ARE_EINVAL, "n_entries must be >= 0");
        ARE_CHECK(n_entries == 0 || (event_ids && losses), ARE_EINVAL, "event_ids/losses are NULL");
        const are_fin_terms f = *terms;
        ARE_CHECK(std::isfinite(f.fx) && f.fx > 0.0, ARE_EINVAL, "fx must be finite and > 0");
        ARE_CHECK(nonneg_finite(f.deductible), ARE_EINVAL, "deductible must be finite and >= 0");
        ARE_CHECK(nonneg_limit(f.limit), ARE_EINVAL, "limit must be >= 0");
        ARE_CHECK(std::isfinite(f.share) && f.share >= 0.0 && f.share <= 1.0, ARE_EINVAL,
                  "share must lie in [0, 1]");
        fence_device_inputs({event_ids, losses});
        cudaStream_t s = ctx->stream;
        std::vector<int32_t> ids = to_host(event_ids, (size_t)n_entries, s);
        std::vector<double> loss = to_host(losses, (size_t)n_entries, s);
        int32_t max_id = -1;
        double max_loss = 0.0;
        for (int32_t i = 0; i < n_entries; ++i) {
            ARE_CHECK(ids[i] >= 0, ARE_EINVAL, "negative event id in ELT");
            ARE_CHECK(nonneg_finite(loss[i]), ARE_EINVAL, "ELT losses must be finite and >= 0");
            ARE_CHECK(std::isfinite(f.fx * loss[i]), ARE_EINVAL, "fx * loss overflows");
            max_id = std::max(max_id, ids[i]);
            max_loss = std::max(max_loss, loss[i]);
        }
        bool dup = false;
        if (n_entries == 0) {
        } else if (max_id < (1 << 28)) {   // bitmap of the ids seen
            std::vector<uint64_t> seen((size_t)max_id / 64 + 1, 0);
            for (int32_t i = 0; i < n_entries && !dup; ++i) {
                uint64_t &w = seen[(size_t)ids[i] >> 6];
                const uint64_t b = 1ull << (ids[i] & 63);
                dup = (w & b) != 0;
                w |= b;
            }
        } else {
            std::vector<int32_t> sorted(ids);
            std::sort(sorted.begin(), sorted.end());
            dup = std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end();
        }
        ARE_CHECK(!dup, ARE_EINVAL, "duplicate event id within one ELT");
        Elt e;
        e.n = n_entries;
        e.max_id = max_id;
        e.max_loss = max_loss;
        e.terms = f;
        try {
            e.d_ids = (int32_t *)dalloc(ctx, sizeof(int32_t) * n_entries);
            e.d_loss = (double *)dalloc(ctx, sizeof(double) * n_entries);
            copy_in(e.d_ids, ids.data(), sizeof(int32_t) * n_entries, s);
            copy_in(e.d_loss, loss.data(), sizeof(double) * n_entries, s);
            ARE_CUDA_TRY(cudaStreamSynchronize(s));
        } catch (...) {
            dfree(ctx, e.d_ids, sizeof(int32_t) * n_entries);
            dfree(ctx, e.d_loss, sizeof(double) * n_entries);
            throw;
        }
        e.bytes = (sizeof(int32_t) + sizeof(double)) * n_entries;
        const int32_t h = ctx->next_handle++;
        ctx->elts[h] = e;
        *elt_handle = h;
    });
}

are_status are_define_layer(are_ctx *ctx, const int32_t *elt_handles, int32_t n_elts,
                            const are_layer_terms *terms, int32_t *layer_handle)
{
    return guarded(ctx, [&] {
        ARE_CHECK(layer_handle && terms && elt_handles, ARE_EINVAL, "NULL argument");
        ARE_CHECK(n_elts >= 1 && n_elts <= kMaxElts, ARE_EINVAL,
                  "a layer holds 1.." + std::to_string(kMaxElts) + " ELTs");
        const are_layer_terms t = *terms;
        ARE_CHECK(nonneg_finite(t.occ_ret) && nonneg_finite(t.agg_ret), ARE_EINVAL,
                  "retentions must be finite and >= 0");
        ARE_CHECK(nonneg_limit(t.occ_lim) && nonneg_limit(t.agg_lim), ARE_EINVAL,
                  "limits must be >= 0");
        Layer L;
        for (int32_t j = 0; j < n_elts; ++j) {
            const int32_t h = elt_handles[j];
            ARE_CHECK(ctx->elts.count(h), ARE_ENOTFOUND, "unknown ELT handle " + std::to_string(h));
            ARE_CHECK(std::find(L.elts.begin(), L.elts.end(), h) == L.elts.end(), ARE_EINVAL,
                      "ELT " + std::to_string(h) + " appears twice in the layer");
            L.elts.push_back(h);
        }
        L.terms = positive_zeros(t);
        for (int32_t h : L.elts) ctx->elts[h].users++;
        const int32_t h = ctx->next_handle++;
        ctx->layers[h] = L;
        *layer_handle = h;
    });
}

are_status are_free_yet(are_ctx *ctx, int32_t h)
{
    return guarded(ctx, [&] {
        Yet &y = yet_of(ctx, h);
        ARE_CHECK(!ctx->server, ARE_EBUSY, "a pricing server is running on this context");
        ARE_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
        dfree(ctx, y.d_ids, y.bytes);
        dfree(ctx, y.d_off, y.d_off ? sizeof(int64_t) * (y.n_trials + 1) : 0);
        ctx->yets.erase(h);
    });
}

are_status are_free_elt(are_ctx *ctx, int32_t h)
{
    return guarded(ctx, [&] {
        auto it = ctx->elts.find(h);
        ARE_CHECK(it != ctx->elts.end(), ARE_ENOTFOUND, "unknown ELT handle " + std::to_string(h));
        ARE_CHECK(it->second.users == 0, ARE_EINVAL, "ELT is used by a layer");
        ARE_CHECK(!ctx->server, ARE_EBUSY, "a pricing server is running on this context");
        dfree(ctx, it->second.d_ids, sizeof(int32_t) * it->second.n);
        dfree(ctx, it->second.d_loss, sizeof(double) * it->second.n);
        ctx->elts.erase(it);
    });
}

are_status are_free_layer(are_ctx *ctx, int32_t h)
{
    return guarded(ctx, [&] {
        Layer &L = layer_of(ctx, h);
        ARE_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
        free_table(ctx, L.t32);
        free_table(ctx, L.t64);
        free_table(ctx, L.t32u);
        free_packed(ctx, L.p64);
        free_packed(ctx, L.p32);
        free_folded(ctx, L.fold);
        free_compact(ctx, L.comp);
        for (int32_t e : L.elts) ctx->elts[e].users--;
        ctx->layers.erase(h);
    });
}

are_status are_prepare(are_ctx *ctx, int32_t layer, int32_t yet, are_precision precision,
                       void *stream)
{
    return guarded(ctx, [&] {
        NvtxRange nvtx("are_prepare");
        check_precision(precision);
        Layer &L = layer_of(ctx, layer);
        Yet &y = yet_of(ctx, yet);
        CallStream cs(ctx, stream);
        ensure_tables(ctx, L, y, precision, cs.s, true);
        cs.finish();
    });
}

are_status are_simulate(are_ctx *ctx, int32_t layer, int32_t yet, int64_t trial_begin,
                        int64_t n_trials, are_precision precision, double *ylt, void *stream)
{
    return guarded(ctx, [&] {
        NvtxRange nvtx("are_simulate");
        check_precision(precision);
        Layer &L = layer_of(ctx, layer);
        Yet &y = yet_of(ctx, yet);
        ARE_CHECK(trial_begin >= 0 && n_trials >= 0 && trial_begin + n_trials <= y.n_trials,
                  ARE_EINVAL, "trial range outside the YET");
        ARE_CHECK(n_trials == 0 || ylt, ARE_EINVAL, "ylt is NULL");
        if (n_trials == 0) return;
        CallStream cs(ctx, stream);
        cudaStream_t s = cs.s;
        const bool fp32 = precision != ARE_FP64;
        ensure_tables(ctx, L, y, precision, s, false);
        const bool dev_out = is_device_ptr(ylt);
        double *d_out = ylt;
        if (!dev_out) d_out = (double *)dalloc(ctx, sizeof(double) * n_trials);
        try {
            const TuneEntry te = tuned(ctx, precision, y, table_jp((int)L.elts.size(), fp32), false);
            ctx->launches += run_single(ctx, L, y, trial_begin, n_trials, precision, d_out, te, s);
            if (!dev_out) {
                ARE_CUDA_TRY(cudaMemcpyAsync(ylt, d_out, sizeof(double) * n_trials,
                                             cudaMemcpyDeviceToHost, s));
                ARE_CUDA_TRY(cudaStreamSynchronize(s));
            }
            cs.finish();
        } catch (...) {
            if (!dev_out) dfree(ctx, d_out, sizeof(double) * n_trials);
            throw;
        }
        if (!dev_out) dfree(ctx, d_out, sizeof(double) * n_trials);
    });
}

are_status are_set_table_layout(are_ctx *ctx, int32_t layer, int32_t layout)
{
    return guarded(ctx, [&] {
        Layer &L = layer_of(ctx, layer);
        ARE_CHECK(layout == ARE_LAYOUT_DIRECT || layout == ARE_LAYOUT_COMPACT, ARE_EINVAL,
                  "layout must be ARE_LAYOUT_DIRECT or ARE_LAYOUT_COMPACT");
        if (L.layout != layout) ++L.generation;
        L.layout = layout;
    });
}

are_status are_layer_rows(are_ctx *ctx, int32_t layer, int32_t yet, are_precision precision,
                          int32_t kernel, int32_t *row_bytes, int32_t *packed)
{
    return guarded(ctx, [&] {
        ARE_CHECK(row_bytes && packed, ARE_EINVAL, "row_bytes and packed must not be NULL");
        ARE_CHECK(kernel >= -1 && kernel <= 3, ARE_EINVAL, "kernel must lie in -1 .. 3");
        check_precision(precision);
        const Layer &L = layer_of(ctx, layer);
        const Yet &y = yet_of(ctx, yet);
        const bool fp32 = precision != ARE_FP64;
        const int J = (int)L.elts.size();
        const int k = kernel >= 0 ? kernel : tuned(ctx, precision, y, table_jp(J, fp32), false).kernel;
        int rb = table_jp(J, fp32) * (fp32 ? 4 : 8), pk = 0;
        if (fp32 && L.layout != ARE_LAYOUT_COMPACT && k == 2) {
            const int pw = row_words(ctx, L, y.catalog, true);
            if (pw) {
                rb = pw * 4;
                pk = 1;
            }
        } else if (!fp32 && k == 2) {
            rb = row_words(ctx, L, y.catalog, false) * 8;
            pk = 1;
        } else if (!fp32 && k == 3) {
            rb = table_jp(J, true) * 4;   // the screen's rows (and the marked FP64 entries)
        }
        *row_bytes = rb;
        *packed = pk;
    });
}

are_status are_prepare_folded(are_ctx *ctx, int32_t layer, int32_t yet, void *stream)
{
    return guarded(ctx, [&] {
        NvtxRange nvtx("are_prepare_folded");
        Layer &L = layer_of(ctx, layer);
        Yet &y = yet_of(ctx, yet);
        CallStream cs(ctx, stream);
        build_folded(ctx, L, y.catalog, cs.s);
        cs.finish();
    });
}

are_status are_simulate_folded(are_ctx *ctx, int32_t layer, int32_t yet, int64_t trial_begin,
                               int64_t n_trials, double *ylt, void *stream)
{
    return guarded(ctx, [&] {
        NvtxRange nvtx("are_simulate_folded");
        Layer &L = layer_of(ctx, layer);
        Yet &y = yet_of(ctx, yet);
        ARE_CHECK(trial_begin >= 0 && n_trials >= 0 && trial_begin + n_trials <= y.n_trials,
                  ARE_EINVAL, "trial range outside the YET");
        ARE_CHECK(n_trials == 0 || ylt, ARE_EINVAL, "ylt is NULL");
        if (n_trials == 0) return;
        CallStream cs(ctx, stream);
        cudaStream_t s = cs.s;
        Folded &f = L.fold;
        if (!f.d || f.catalog != y.catalog) build_folded(ctx, L, y.catalog, s);
        const bool dev_out = is_device_ptr(ylt);
        double *d_out = dev_out ? ylt : (double *)dalloc(ctx, sizeof(double) * n_trials);
        try {
            FoldArgs a{};
            a.ids = y.d_ids;
            a.off = y.d_off;
            a.k = y.k;
            a.trial_begin = trial_begin;
            a.n_trials = n_trials;
            a.n_events = y.n_events;
            a.F = f.F();
            a.bits = f.bits();
            a.words = f.words;
            a.hmax = f.hmax();
            a.agg_r = L.terms.agg_ret;
            a.agg_l = L.terms.agg_lim;
            a.ylt = d_out;
            ctx->launches += launch_folded(a, ctx->num_sms, s);
            if (!dev_out) {
                ARE_CUDA_TRY(cudaMemcpyAsync(ylt, d_out, sizeof(double) * n_trials,
                                             cudaMemcpyDeviceToHost, s));
                ARE_CUDA_TRY(cudaStreamSynchronize(s));
            }
            cs.finish();
        } catch (...) {
            if (!dev_out) dfree(ctx, d_out, sizeof(double) * n_trials);
            throw;
        }
        if (!dev_out) dfree(ctx, d_out, sizeof(double) * n_trials);
    });
}

// The analysis over a host-resident YET, chunk by chunk (are_simulate_streamed
// and are_simulate_streamed_packed).  id_bits 0: event_ids is int32[n_events];
// 1 .. 32: a stream of 32-bit words holding the ids packed id_bits bits each.
static void simulate_streamed(are_ctx *ctx, int32_t layer, int32_t catalog_size, int64_t n_trials,
                       const int64_t *offsets, int32_t events_per_trial, const void *event_ids, int id_bits,
                       int64_t chunk_events, are_precision precision, double *ylt, void *stream)
{
    {
        check_precision(precision);
        Layer &L = layer_of(ctx, layer);
        ARE_CHECK(catalog_size > 0, ARE_EINVAL, "catalog_size must be > 0");
        ARE_CHECK(n_trials >= 0 && n_trials < (int64_t)INT32_MAX, ARE_EINVAL,
                  "n_trials must lie in 0 .. 2^31 - 2");
        ARE_CHECK(offsets || events_per_trial > 0, ARE_EINVAL, "need offsets or events_per_trial > 0");
        ARE_CHECK(chunk_events >= 0, ARE_EINVAL, "chunk_events must be >= 0");
        ARE_CHECK(n_trials == 0 || ylt, ARE_EINVAL, "ylt is NULL");
        if (n_trials == 0) return;
        ARE_CHECK(event_ids && !is_device_ptr(event_ids), ARE_EINVAL,
                  "event_ids must be host memory (a device-resident YET goes through are_load_yet)");
        fence_device_inputs({offsets});
        CallStream cs(ctx, stream);
        cudaStream_t s = cs.s;
        if (!ctx->copy_stream) ARE_CUDA_TRY(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
        cudaStream_t cp = ctx->copy_stream;

        // the trials' event ranges, on the host for the chunk plan
        Yet v;
        v.catalog = catalog_size;
        v.n_trials = n_trials;
        v.k = offsets ? 0 : events_per_trial;
        std::vector<int64_t> hoff;
        if (offsets) {
            hoff = to_host(offsets, (size_t)n_trials + 1, s);
            ARE_CHECK(hoff[0] == 0, ARE_EINVAL, "offsets must start at 0");
            for (int64_t t = 0; t < n_trials; ++t)
                ARE_CHECK(hoff[t + 1] >= hoff[t], ARE_EINVAL, "offsets must be non-decreasing");
            v.n_events = hoff[n_trials];
        } else {
            v.n_events = n_trials * (int64_t)events_per_trial;
        }
        auto first_event = [&](int64_t t) { return offsets ? hoff[t] : t * (int64_t)events_per_trial; };
        // chunks of whole trials, about chunk_events ids each (a longer trial is a chunk alone)
        const int64_t want = chunk_events > 0 ? chunk_events : ((int64_t)64 << 20);
        std::vector<int64_t> cut{0};
        int64_t longest = 0;
        for (int64_t t = 0; t < n_trials;) {
            const int64_t b = first_event(t);
            int64_t u = t + 1;
            if (offsets) {
                while (u < n_trials && hoff[u + 1] - b <= want) ++u;
            } else {
                const int64_t per = std::max<int64_t>(1, want / events_per_trial);
                u = std::min(n_trials, t + per);
            }
            longest = std::max(longest, first_event(u) - b);
            cut.push_back(u);
            t = u;
        }
        const size_t buf_bytes = sizeof(int32_t) * (size_t)(longest + 4 + kIdPad);
        // packed ids: the words of the longest chunk, a partial word on each
        // side and one more the unpacking may read
        const size_t wbuf_bytes = id_bits ? sizeof(uint32_t) * (size_t)((longest * id_bits + 31) / 32 + 3) : 0;

        const bool fp32 = precision != ARE_FP64;
        ensure_tables(ctx, L, v, precision, s, false);
        const int jp = table_jp((int)L.elts.size(), fp32);
        int64_t *d_off = nullptr;
        int32_t *buf[2] = {nullptr, nullptr};
        uint32_t *wbuf[2] = {nullptr, nullptr};
        const bool dev_out = is_device_ptr(ylt);
        double *d_out = nullptr;
        cudaEvent_t start = nullptr, ready[2] = {nullptr, nullptr}, done[2] = {nullptr, nullptr};
        auto cleanup = [&] {
            for (cudaEvent_t e : {start, ready[0], ready[1], done[0], done[1]})
                if (e) cudaEventDestroy(e);
            if (!dev_out) dfree(ctx, d_out, sizeof(double) * n_trials);
            for (int i = 0; i < 2; ++i) dfree(ctx, buf[i], buf_bytes);
            for (int i = 0; i < 2; ++i) dfree(ctx, wbuf[i], wbuf_bytes);
            dfree(ctx, d_off, d_off ? sizeof(int64_t) * (n_trials + 1) : 0);
        };
        try {
            if (offsets) {
                d_off = (int64_t *)dalloc(ctx, sizeof(int64_t) * (n_trials + 1));
                copy_in(d_off, hoff.data(), sizeof(int64_t) * (n_trials + 1), s);
            }
            v.d_off = d_off;
            for (int i = 0; i < 2; ++i) buf[i] = (int32_t *)dalloc(ctx, buf_bytes);
            if (id_bits)
                for (int i = 0; i < 2; ++i) {
                    wbuf[i] = (uint32_t *)dalloc(ctx, wbuf_bytes);
                    ARE_CUDA_TRY(cudaMemsetAsync(wbuf[i], 0, wbuf_bytes, s));
                }
            d_out = dev_out ? ylt : (double *)dalloc(ctx, sizeof(double) * n_trials);
            for (cudaEvent_t *e : {&start, &ready[0], &ready[1], &done[0], &done[1]})
                ARE_CUDA_TRY(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
            ARE_CUDA_TRY(cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), s));
            ARE_CUDA_TRY(cudaEventRecord(start, s));
            ARE_CUDA_TRY(cudaStreamWaitEvent(cp, start, 0));
            const TuneEntry te = tuned(ctx, precision, v, jp, false);
            for (size_t c = 0; c + 1 < cut.size(); ++c) {
                const int slot = (int)(c & 1);
                const int64_t t0 = cut[c], t1 = cut[c + 1];
                const int64_t first = first_event(t0), n = first_event(t1) - first;
                const int64_t lead = first & 3;   // keeps 16-byte vectors of ids aligned
                // the copy stream only copies, back to back; the rest of a
                // chunk's preparation runs on the analysis stream
                if (c >= 2) ARE_CUDA_TRY(cudaStreamWaitEvent(cp, done[slot], 0));
                int32_t *b = buf[slot];
                if (!id_bits) {
                    if (n)
                        ARE_CUDA_TRY(cudaMemcpyAsync(b + lead, static_cast<const int32_t *>(event_ids) + first,
                                                     sizeof(int32_t) * n, cudaMemcpyHostToDevice, cp));
                } else if (n) {   // the words that hold the chunk's ids
                    const int64_t w0 = first * id_bits / 32, w1 = ((first + n) * id_bits + 31) / 32;
                    ARE_CUDA_TRY(cudaMemcpyAsync(wbuf[slot], static_cast<const uint32_t *>(event_ids) + w0,
                                                 sizeof(uint32_t) * (w1 - w0), cudaMemcpyHostToDevice, cp));
                }
                ARE_CUDA_TRY(cudaEventRecord(ready[slot], cp));
                ARE_CUDA_TRY(cudaStreamWaitEvent(s, ready[slot], 0));
                if (lead) ARE_CUDA_TRY(cudaMemsetAsync(b, 0, sizeof(int32_t) * lead, s));
                ARE_CUDA_TRY(cudaMemsetAsync(b + lead + n, 0, sizeof(int32_t) * kIdPad, s));
                if (!id_bits)
                    ctx->launches += launch_sanitize_ids(b + lead, n, catalog_size, ctx->d_flag, s);
                else
                    ctx->launches += launch_unpack_ids(wbuf[slot], first * id_bits - first * id_bits / 32 * 32,
                                                       id_bits, n, catalog_size, b + lead, ctx->d_flag, s);
                Yet cv = v;
                cv.d_ids = b + lead - first;   // indexed by the YET's own event numbers
                ctx->launches += run_single(ctx, L, cv, t0, t1 - t0, precision, d_out + t0, te, s);
                ARE_CUDA_TRY(cudaEventRecord(done[slot], s));
            }
            if (!dev_out)
                ARE_CUDA_TRY(cudaMemcpyAsync(ylt, d_out, sizeof(double) * n_trials, cudaMemcpyDeviceToHost, s));
            const int f = check_flag(ctx, s);
            ARE_CHECK(!(f & 1), ARE_EINVAL, "event id outside [0, catalog_size) (results are not valid)");
            cs.finish();
        } catch (...) {
            cudaStreamSynchronize(s);
            cudaStreamSynchronize(cp);
            cleanup();
            throw;
        }
        cleanup();
    }
}

are_status are_simulate_streamed(are_ctx *ctx, int32_t layer, int32_t catalog_size, int64_t n_trials,
                                 const int64_t *offsets, int32_t events_per_trial,
                                 const int32_t *event_ids, int64_t chunk_events,
                                 are_precision precision, double *ylt, void *stream)
{
    return guarded(ctx, [&] {
        NvtxRange nvtx("are_simulate_streamed");
        simulate_streamed(ctx, layer, catalog_size, n_trials, offsets, events_per_trial, event_ids, 0,
                          chunk_events, precision, ylt, stream);
    });
}

are_status are_simulate_streamed_packed(are_ctx *ctx, int32_t layer, int32_t catalog_size, int64_t n_trials,
                                        const int64_t *offsets, int32_t events_per_trial,
                                        const uint32_t *packed_ids, int32_t id_bits, int64_t chunk_events,
                                        are_precision precision, double *ylt, void *stream)
{
    return guarded(ctx, [&] {
        NvtxRange nvtx("are_simulate_streamed_packed");
        ARE_CHECK(id_bits >= 1 && id_bits <= 32, ARE_EINVAL, "id_bits must lie in 1 .. 32");
        simulate_streamed(ctx, layer, catalog_size, n_trials, offsets, events_per_trial, packed_ids, id_bits,
                          chunk_events, precision, ylt, stream);
    });
}

are_status are_pack_ids(are_ctx *ctx, const int32_t *ids, int64_t n, int32_t id_bits, uint32_t *out)
{
    return guarded(ctx, [&] {
        ARE_CHECK(id_bits >= 1 && id_bits <= 32, ARE_EINVAL, "id_bits must lie in 1 .. 32");
        ARE_CHECK(n >= 0 && (n == 0 || (ids && out)), ARE_EINVAL, "NULL array");
        ARE_CHECK(!is_device_ptr(ids) && !is_device_ptr(out), ARE_EINVAL, "ids and out must be host memory");
        const uint64_t lim = id_bits == 32 ? (1ull << 32) : (1ull << id_bits);
        const int64_t words = (n * id_bits + 31) / 32;
        uint64_t acc = 0;   // bits not yet written, the lowest first
        int have = 0;
        int64_t w = 0;
        for (int64_t i = 0; i < n; ++i) {
            const int32_t v = ids[i];
            ARE_CHECK(v >= 0 && (uint64_t)v < lim, ARE_EINVAL,
                      "id " + std::to_string(v) + " does not fit in " + std::to_string(id_bits) + " bits");
            acc |= (uint64_t)(uint32_t)v << have;
            have += id_bits;
            if (have >= 32) {
                out[w++] = (uint32_t)acc;
                acc >>= 32;
                have -= 32;
            }
        }
        if (have > 0) out[w++] = (uint32_t)acc;
        ARE_CHECK(w == words, ARE_EINVAL, "internal: packed word count");
    });
}

are_status are_gather_ceiling(are_ctx *ctx, int32_t yet, int32_t row_bytes, int64_t trial_begin,
                              int64_t n_trials, int32_t reps, double *rows_per_s,
                              are_ceiling_shape *shapes, int32_t max_shapes, int32_t *n_shapes)
{
    return guarded(ctx, [&] {
        NvtxRange nvtx("are_gather_ceiling");
        Yet &y = yet_of(ctx, yet);
        ARE_CHECK(row_bytes == 32 || row_bytes == 64 || row_bytes == 128, ARE_EINVAL,
                  "row_bytes must be 32, 64 or 128");
        ARE_CHECK(reps >= 1 && reps <= 100, ARE_EINVAL, "reps must lie in 1 .. 100");
        ARE_CHECK(trial_begin >= 0 && n_trials >= 1 && trial_begin + n_trials <= y.n_trials,
                  ARE_EINVAL, "trial range outside the YET (or empty)");
        ARE_CHECK(rows_per_s, ARE_EINVAL, "rows_per_s is NULL");
        ARE_CHECK(!shapes || max_shapes >= 0, ARE_EINVAL, "max_shapes must be >= 0");
        CallStream cs(ctx, nullptr);
        int64_t first, last;
        if (y.d_off) {
            ARE_CUDA_TRY(cudaMemcpy(&first, y.d_off + trial_begin, sizeof first, cudaMemcpyDeviceToHost));
            ARE_CUDA_TRY(cudaMemcpy(&last, y.d_off + trial_begin + n_trials, sizeof last,
                                    cudaMemcpyDeviceToHost));
        } else {
            first = trial_begin * y.k;
            last = (trial_begin + n_trials) * y.k;
        }
        ARE_CHECK(last > first, ARE_EINVAL, "the trial range holds no events");
        const size_t tab_bytes = (size_t)y.catalog * row_bytes;
        const size_t out_bytes = sizeof(float) * (size_t)ctx->num_sms * 8 * 256;
        void *tab = dalloc(ctx, tab_bytes);
        float *out = nullptr;
        try {
            out = (float *)dalloc(ctx, out_bytes);
            ARE_CUDA_TRY(cudaMemsetAsync(tab, 0, tab_bytes, cs.s));
            const std::vector<CeilingShape> res = gather_ceiling(
                y.d_ids + first, last - first, row_bytes, reps, ctx->num_sms, tab, out, cs.s,
                ctx->launches);
            double best = 0.0;
            for (size_t i = 0; i < res.size(); ++i) {
                best = std::max(best, res[i].rows_per_s);
                if (shapes && (int64_t)i < max_shapes)
                    shapes[i] = are_ceiling_shape{res[i].kind, res[i].rows_in_flight,
                                                  res[i].blocks_per_sm, res[i].rows_per_s};
            }
            *rows_per_s = best;
            if (n_shapes) *n_shapes = (int32_t)res.size();
            cs.finish();
        } catch (...) {
            if (out) dfree(ctx, out, out_bytes);
            dfree(ctx, tab, tab_bytes);
            throw;
        }
        dfree(ctx, out, out_bytes);
        dfree(ctx, tab, tab_bytes);
    });
}

are_status are_simulate_occurrences(are_ctx *ctx, int32_t layer, int32_t yet, int64_t trial_begin,
                                    int64_t n_trials, are_precision precision, double *marginals,
                                    double *occ_max, double *ylt, void *stream)
{
    return guarded(ctx, [&] {
        NvtxRange nvtx("are_simulate_occurrences");
        check_precision(precision);
        Layer &L = layer_of(ctx, layer);
        Yet &y = yet_of(ctx, yet);
        ARE_CHECK(trial_begin >= 0 && n_trials >= 0 && trial_begin + n_trials <= y.n_trials,
                  ARE_EINVAL, "trial range outside the YET");
        ARE_CHECK(marginals && is_device_ptr(marginals), ARE_EINVAL,
                  "marginals must be device memory");
        ARE_CHECK(!occ_max || is_device_ptr(occ_max), ARE_EINVAL, "occ_max must be device memory");
        ARE_CHECK(!ylt || is_device_ptr(ylt), ARE_EINVAL, "ylt must be device memory");
        if (n_trials == 0) return;
        CallStream cs(ctx, stream);
        const bool fp32 = precision != ARE_FP64;
        Table &t = fp32 ? L.t32 : L.t64;
        // the rows of the register-rows form (the direct layout, whatever the
        // layer's analysis layout): packed where the layer's row size calls for them
        const bool packed = ensure_packed(ctx, L, y.catalog, fp32, cs.s, false);
        if (!packed && (!t.d || t.catalog != y.catalog)) build_table(ctx, L, y.catalog, fp32, cs.s);
        SimArgs a{};
        a.ids = y.d_ids;
        a.off = y.d_off;
        a.k = y.k;
        a.trial_begin = trial_begin;
        a.n_trials = n_trials;
        a.table = t.d;
        a.agg_r = L.terms.agg_ret;
        a.agg_l = L.terms.agg_lim;
        a.ylt = ylt;
        a.marg = marginals;
        a.occ_max = occ_max;
        if (y.d_off) {
            ARE_CUDA_TRY(cudaMemcpyAsync(&a.marg_base, y.d_off + trial_begin, sizeof(int64_t),
                                         cudaMemcpyDeviceToHost, cs.s));
            ARE_CUDA_TRY(cudaStreamSynchronize(cs.s));
        } else {
            a.marg_base = trial_begin * (int64_t)y.k;
        }
        TermsF32 t32;
        TermsF64 t64;
        fill_terms(L, t32, t64);
        if (packed) {
            const Packed &p = fp32 ? L.p32 : L.p64;
            a.table = p.rows();
            a.table2 = p.ovf();
            ctx->launches += launch_rows_occ(a, fp32 ? 1 : 0, p.rw, t32, t64, fixed_scale(ctx, L), ctx->num_sms,
                                             cs.s);
        } else {         // dense FP32 rows
            ctx->launches += launch_rows_occ(a, 2, t.jp, t32, t64, fixed_scale(ctx, L), ctx->num_sms, cs.s);
        }
        cs.finish();
    });
}

are_status are_risk_measures(are_ctx *ctx, const double *ylt, int64_t n,
                             const double *return_periods, int32_t n_rp, double *pml_out,
                             const double *tvar_levels, int32_t n_tv, double *tvar_out,
                             void *stream)
{
    return guarded(ctx, [&] {
        NvtxRange nvtx("are_risk_measures");
        ARE_CHECK(n > 0 && ylt, ARE_EINVAL, "need a YLT of n > 0 losses");
        ARE_CHECK(n < (int64_t)UINT32_MAX, ARE_EINVAL, "YLT too long for the selection counters");
        ARE_CHECK(n_rp >= 0 && n_tv >= 0, ARE_EINVAL, "negative count");
        ARE_CHECK(n_rp == 0 || (return_periods && pml_out), ARE_EINVAL, "NULL PML arrays");
        ARE_CHECK(n_tv == 0 || (tvar_levels && tvar_out), ARE_EINVAL, "NULL TVaR arrays");
        std::vector<int64_t> ranks;
        for (int32_t r = 0; r < n_rp; ++r) ranks.push_back(rank_rp(n, return_periods[r]));
        for (int32_t r = 0; r < n_tv; ++r) ranks.push_back(rank_level(n, tvar_levels[r]));
        if (ranks.empty()) return;
        // device outputs: the call only enqueues (see the header)
        const bool dev_pml = n_rp > 0 && is_device_ptr(pml_out), dev_tv = n_tv > 0 && is_device_ptr(tvar_out);
        const bool dev_out = dev_pml || dev_tv;
        if (dev_out) {
            ARE_CHECK((n_rp == 0 || dev_pml) && (n_tv == 0 || dev_tv), ARE_EINVAL,
                      "pml_out and tvar_out must both be host or both be device arrays");
            ARE_CHECK(is_device_ptr(ylt), ARE_EINVAL, "device outputs need a device YLT");
            CallStream cs(ctx, stream);
            cudaStream_t s = cs.s;
            const int32_t nr = (int32_t)ranks.size();
            for (int32_t b = 0; b < nr; b += kMaxTargets) {
                const int nt = std::min<int32_t>(kMaxTargets, nr - b);
                ctx->launches += launch_select(ylt, n, ranks.data() + b, nt, ctx->sel, ctx->num_sms, s);
                // result: (m-th largest, mean of the m largest) per target
                const int p_end = std::min(b + nt, n_rp);
                if (p_end > b)
                    ARE_CUDA_TRY(cudaMemcpy2DAsync(pml_out + b, sizeof(double), ctx->sel.result, 2 * sizeof(double),
                                                   sizeof(double), p_end - b, cudaMemcpyDeviceToDevice, s));
                const int t_begin = std::max(b, n_rp);
                if (b + nt > t_begin)
                    ARE_CUDA_TRY(cudaMemcpy2DAsync(tvar_out + (t_begin - n_rp), sizeof(double),
                                                   ctx->sel.result + 2 * (t_begin - b) + 1, 2 * sizeof(double),
                                                   sizeof(double), b + nt - t_begin, cudaMemcpyDeviceToDevice, s));
            }
            cs.finish();
            return;
        }
        CallStream cs(ctx, stream);
        cudaStream_t s = cs.s;
        const bool dev_in = is_device_ptr(ylt);
        const double *d_y = ylt;
        double *tmp = nullptr;
        if (!dev_in) {
            tmp = (double *)dalloc(ctx, sizeof(double) * n);
            d_y = tmp;
        }
        std::vector<double> res(2 * ranks.size());
        try {
            if (tmp) copy_in(tmp, ylt, sizeof(double) * n, s);
            for (size_t b = 0; b < ranks.size(); b += kMaxTargets) {
                const int nt = (int)std::min<size_t>(kMaxTargets, ranks.size() - b);
                ctx->launches += launch_select(d_y, n, ranks.data() + b, nt, ctx->sel, ctx->num_sms, s);
                ARE_CUDA_TRY(cudaMemcpyAsync(ctx->h_result, ctx->sel.result, sizeof(double) * 2 * nt,
                                             cudaMemcpyDeviceToHost, s));
                ARE_CUDA_TRY(cudaStreamSynchronize(s));
                std::memcpy(res.data() + 2 * b, ctx->h_result, sizeof(double) * 2 * nt);
            }
        } catch (...) {
            dfree(ctx, tmp, sizeof(double) * n);
            throw;
        }
        dfree(ctx, tmp, sizeof(double) * n);
        for (int32_t r = 0; r < n_rp; ++r) pml_out[r] = res[2 * r];
        for (int32_t r = 0; r < n_tv; ++r) tvar_out[r] = res[2 * (n_rp + r) + 1];
    });
}

are_status are_simulate_portfolio(are_ctx *ctx, const int32_t *layers, int32_t n_layers,
                                  int32_t yet, int64_t trial_begin, int64_t n_trials,
                                  are_precision precision, double *const *ylts, void *stream)
{
    return guarded(ctx, [&] {
        NvtxRange nvtx("are_simulate_portfolio");
        check_precision(precision);
        Yet &y = yet_of(ctx, yet);
        ARE_CHECK(ylts, ARE_EINVAL, "ylts is NULL");
        check_multi_args(ctx, layers, n_layers, y, trial_begin, n_trials, ylts);
        CallStream cs(ctx, stream);
        const bool fp32 = precision != ARE_FP64;
        const int k = tuned(ctx, precision, y, max_width(ctx, layers, n_layers, fp32), n_layers > 1).kernel;
        ensure_tables(ctx, layers, n_layers, y, fp32, cs.s, k);
        const std::vector<int32_t> lv(layers, layers + n_layers);
        const std::vector<double *> yv(ylts, ylts + n_layers);
        std::vector<uint64_t> gens;
        for (int32_t h : lv) gens.push_back(ctx->layers.at(h).generation);
        const TuneEntry te = tuned(ctx, precision, y, max_width(ctx, layers, n_layers, fp32), true);

        Plan *plan = nullptr;
        for (Plan &p : ctx->plans)
            if (p.layers == lv && p.ylts == yv && p.generations == gens && p.yet == yet &&
                p.trial_begin == trial_begin && p.n_trials == n_trials &&
                p.precision == (int)precision && p.kernel == te.kernel &&
                p.cfg.rows_in_flight == te.cfg.rows_in_flight &&
                p.cfg.trials_per_item == te.cfg.trials_per_item &&
                p.cfg.blocks_per_sm == te.cfg.blocks_per_sm)
                plan = &p;
        if (!plan) {
            if (ctx->plans.size() >= 8) {
                free_plan(ctx, ctx->plans.front());
                ctx->plans.erase(ctx->plans.begin());
            }
            Plan p;
            p.layers = lv;
            p.ylts = yv;
            p.generations = gens;
            p.yet = yet;
            p.trial_begin = trial_begin;
            p.n_trials = n_trials;
            p.precision = (int)precision;
            p.kernel = te.kernel;
            p.cfg = te.cfg;
            try {
                Groups g;
                if (fp32 && te.kernel == 0) {
                    g = group_layers(ctx, lv, yv, n_trials,
                                     te.cfg.trials_per_item > 0 ? te.cfg.trials_per_item : 8);
                    p.work_bytes = g.bytes;
                    p.d_work = dalloc(ctx, g.bytes);
                    std::vector<unsigned char> host(g.bytes, 0);
                    for (int gi = 0; gi < 3; ++gi)
                        if (!g.rec[gi].empty())
                            std::memcpy(host.data() + g.offset[gi], g.rec[gi].data(),
                                        sizeof(LayerF32) * g.rec[gi].size());
                    ARE_CUDA_TRY(cudaMemcpyAsync(p.d_work, host.data(), g.bytes,
                                                 cudaMemcpyHostToDevice, cs.s));
                    ARE_CUDA_TRY(cudaStreamSynchronize(cs.s));
                }
                ARE_CUDA_TRY(cudaStreamBeginCapture(ctx->capture, cudaStreamCaptureModeThreadLocal));
                int launches = 0;
                try {
                    launches = enqueue_multi(ctx, lv, yv, y, trial_begin, n_trials, precision, te,
                                             &g, p.d_work, ctx->capture);
                } catch (...) {
                    cudaGraph_t dead = nullptr;
                    cudaStreamEndCapture(ctx->capture, &dead);
                    if (dead) cudaGraphDestroy(dead);
                    throw;
                }
                ARE_CUDA_TRY(cudaStreamEndCapture(ctx->capture, &p.graph));
                ARE_CUDA_TRY(cudaGraphInstantiate(&p.exec, p.graph, 0));
                p.launches = (uint64_t)launches;
            } catch (...) {
                free_plan(ctx, p);
                throw;
            }
            ctx->plans.push_back(p);
            plan = &ctx->plans.back();
        }
        ARE_CUDA_TRY(cudaGraphLaunch(plan->exec, cs.s));
        ctx->launches += plan->launches;
        cs.finish();
    });
}

are_status are_risk_measures_batch(are_ctx *ctx, const double *const *ylts, int32_t n_ylt,
                                   int64_t n, const double *return_periods, int32_t n_rp,
                                   double *pml_out, const double *tvar_levels, int32_t n_tv,
                                   double *tvar_out, void *stream)
{
    return guarded(ctx, [&] {
        NvtxRange nvtx("are_risk_measures_batch");
        ARE_CHECK(ylts && n_ylt >= 1, ARE_EINVAL, "need at least one YLT");
        ARE_CHECK(n > 0 && n < (int64_t)UINT32_MAX, ARE_EINVAL, "bad YLT length");
        ARE_CHECK(n_rp >= 0 && n_tv >= 0, ARE_EINVAL, "negative count");
        ARE_CHECK(n_rp == 0 || (return_periods && pml_out), ARE_EINVAL, "NULL PML arrays");
        ARE_CHECK(n_tv == 0 || (tvar_levels && tvar_out), ARE_EINVAL, "NULL TVaR arrays");
        for (int32_t i = 0; i < n_ylt; ++i)
            ARE_CHECK(ylts[i] && is_device_ptr(ylts[i]), ARE_EINVAL, "every YLT must be device memory");
        std::vector<int64_t> ranks;
        for (int32_t r = 0; r < n_rp; ++r) ranks.push_back(rank_rp(n, return_periods[r]));
        for (int32_t r = 0; r < n_tv; ++r) ranks.push_back(rank_level(n, tvar_levels[r]));
        if (ranks.empty()) return;
        CallStream cs(ctx, stream);
        const size_t ptr_bytes = (sizeof(double *) * n_ylt + 255) / 256 * 256;
        const size_t need = ptr_bytes + select_multi_bytes(n_ylt, n, ctx->num_sms);
        if (ctx->multi_bytes < need) {
            ARE_CUDA_TRY(cudaStreamSynchronize(cs.s));
            dfree(ctx, ctx->d_multi, ctx->multi_bytes);
            ctx->d_multi = nullptr;
            ctx->multi_bytes = 0;
            ctx->d_multi = dalloc(ctx, need);
            ctx->multi_bytes = need;
        }
        const size_t count = (size_t)2 * kMaxTargets * n_ylt;
        if (ctx->h_multi_count < count) {
            if (ctx->h_multi) cudaFreeHost(ctx->h_multi);
            ctx->h_multi = nullptr;
            ctx->h_multi_count = 0;
            ARE_CUDA_TRY(cudaMallocHost(&ctx->h_multi, sizeof(double) * count));
            ctx->h_multi_count = count;
        }
        const double *const *d_ptrs = static_cast<const double *const *>(ctx->d_multi);
        ARE_CUDA_TRY(cudaMemcpyAsync(ctx->d_multi, ylts, sizeof(double *) * n_ylt,
                                     cudaMemcpyHostToDevice, cs.s));
        void *scratch = static_cast<unsigned char *>(ctx->d_multi) + ptr_bytes;
        for (size_t b = 0; b < ranks.size(); b += kMaxTargets) {
            const int nt = (int)std::min<size_t>(kMaxTargets, ranks.size() - b);
            double *d_res = nullptr;
            ctx->launches += launch_select_multi(d_ptrs, n_ylt, n, ranks.data() + b, nt, scratch,
                                                 ctx->num_sms, cs.s, &d_res);
            ARE_CUDA_TRY(cudaMemcpyAsync(ctx->h_multi, d_res, sizeof(double) * count,
                                         cudaMemcpyDeviceToHost, cs.s));
            ARE_CUDA_TRY(cudaStreamSynchronize(cs.s));
            for (int32_t y = 0; y < n_ylt; ++y)
                for (int t = 0; t < nt; ++t) {
                    const size_t gt = b + t;
                    const double *res = ctx->h_multi + (size_t)y * 2 * kMaxTargets;
                    if ((int64_t)gt < n_rp) pml_out[(size_t)y * n_rp + gt] = res[2 * t];
                    else tvar_out[(size_t)y * n_tv + (gt - n_rp)] = res[2 * t + 1];
                }
        }
        cs.finish();
    });
}

are_status are_autotune(are_ctx *ctx, const int32_t *layers, int32_t n_layers, int32_t yet,
                        are_precision precision, void *stream, are_tune_result *best)
{
    return guarded(ctx, [&] {
        NvtxRange nvtx("are_autotune");
        check_precision(precision);
        Yet &y = yet_of(ctx, yet);
        check_multi_args(ctx, layers, n_layers, y, 0, y.n_trials, nullptr);
        CallStream cs(ctx, stream);
        const bool fp32 = precision != ARE_FP64;
        ensure_tables(ctx, layers, n_layers, y, fp32, cs.s, 2);              // packed rows
        ensure_tables(ctx, layers, n_layers, y, fp32, cs.s, 1);              // dense rows
        if (!fp32) ensure_tables(ctx, layers, n_layers, y, fp32, cs.s, 3);  // FP64: the screen
        const bool multi = n_layers > 1;
        const int jp = max_width(ctx, layers, n_layers, fp32);
        const std::string key = tune_key(precision, y, jp, multi);
        std::vector<TuneEntry> cands;
        if (fp32) {
            for (int u : {1, 2}) {            // register rows, one or two groups of 32 events
                TuneEntry e;
                e.kernel = 2;
                e.cfg.rows_in_flight = u;
                cands.push_back(e);
            }
            for (int epl : {1, 2}) {          // staged rows, one or two events per lane
                TuneEntry e;
                e.kernel = 1;
                e.cfg.rows_in_flight = epl;
                cands.push_back(e);
            }
            for (int u : {1, 2})              // persistent work items
                for (int tpi : multi ? std::vector<int>{4, 8, 16, 32} : std::vector<int>{8, 32}) {
                    TuneEntry e;
                    e.kernel = 0;
                    e.cfg.rows_in_flight = u;
                    e.cfg.trials_per_item = tpi;
                    cands.push_back(e);
                }
        } else {
            for (int u : {1, 2}) {      // register rows over the packed FP64 rows
                TuneEntry e;
                e.kernel = 2;
                e.cfg.rows_in_flight = u;
                cands.push_back(e);
            }
            for (int k : {1, 3}) {      // staged FP64 rows, staged screen rows
                TuneEntry e;
                e.kernel = k;
                cands.push_back(e);
            }
        }
        const size_t out_bytes = sizeof(double) * (size_t)y.n_trials * n_layers;
        double *outs = (double *)dalloc(ctx, out_bytes);
        void *work = nullptr;
        size_t work_bytes = 0;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        TuneEntry win;
        win.ms = 1e300;
        try {
            ARE_CUDA_TRY(cudaEventCreate(&e0));
            ARE_CUDA_TRY(cudaEventCreate(&e1));
            std::vector<int32_t> lv(layers, layers + n_layers);
            std::vector<double *> yv;
            for (int32_t i = 0; i < n_layers; ++i) yv.push_back(outs + (size_t)i * y.n_trials);
            for (TuneEntry &c : cands) {
                Groups g;
                if (fp32 && c.kernel == 0) {
                    g = group_layers(ctx, lv, yv, y.n_trials, c.cfg.trials_per_item);
                    if (work_bytes < g.bytes) {
                        ARE_CUDA_TRY(cudaStreamSynchronize(cs.s));
                        dfree(ctx, work, work_bytes);
                        work = nullptr;
                        work = dalloc(ctx, g.bytes);
                        work_bytes = g.bytes;
                    }
                    std::vector<unsigned char> host(g.bytes, 0);
                    for (int gi = 0; gi < 3; ++gi)
                        if (!g.rec[gi].empty())
                            std::memcpy(host.data() + g.offset[gi], g.rec[gi].data(),
                                        sizeof(LayerF32) * g.rec[gi].size());
                    ARE_CUDA_TRY(cudaMemcpyAsync(work, host.data(), g.bytes, cudaMemcpyHostToDevice, cs.s));
                    ARE_CUDA_TRY(cudaStreamSynchronize(cs.s));
                }
                auto run = [&] {
                    if (multi)
                        ctx->launches += enqueue_multi(ctx, lv, yv, y, 0, y.n_trials, precision, c,
                                                       &g, work, cs.s);
                    else
                        ctx->launches += run_single(ctx, ctx->layers.at(lv[0]), y, 0, y.n_trials,
                                                    precision, yv[0], c, cs.s);
                };
                run();
                double best_ms = 1e300;
                for (int rep = 0; rep < 3; ++rep) {
                    ARE_CUDA_TRY(cudaEventRecord(e0, cs.s));
                    run();
                    ARE_CUDA_TRY(cudaEventRecord(e1, cs.s));
                    ARE_CUDA_TRY(cudaEventSynchronize(e1));
                    float ms = 0.f;
                    ARE_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
                    best_ms = std::min(best_ms, (double)ms);
                }
                c.ms = best_ms;
                if (best_ms < win.ms) win = c;
            }
        } catch (...) {
            cudaStreamSynchronize(cs.s);
            if (e0) cudaEventDestroy(e0);
            if (e1) cudaEventDestroy(e1);
            dfree(ctx, work, work_bytes);
            dfree(ctx, outs, out_bytes);
            throw;
        }
        ARE_CUDA_TRY(cudaStreamSynchronize(cs.s));
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        dfree(ctx, work, work_bytes);
        dfree(ctx, outs, out_bytes);
        ctx->tune[key] = win;
        if (best) {
            best->kernel = win.kernel;
            best->rows_in_flight = win.cfg.rows_in_flight;
            best->trials_per_item = win.cfg.trials_per_item;
            best->blocks_per_sm = win.cfg.blocks_per_sm;
            best->ms = win.ms;
        }
        cs.finish();
    });
}

are_status are_tune_save(are_ctx *ctx, const char *path)
{
    return guarded(ctx, [&] {
        ARE_CHECK(path, ARE_EINVAL, "path is NULL");
        FILE *f = std::fopen(path, "w");
        ARE_CHECK(f, ARE_EINVAL, std::string("cannot write ") + path);
        for (const auto &kv : ctx->tune)
            std::fprintf(f,
                         "{\"key\": \"%s\", \"kernel\": %d, \"rows_in_flight\": %d, "
                         "\"trials_per_item\": %d, \"blocks_per_sm\": %d, \"ms\": %.6f}\n",
                         kv.first.c_str(), kv.second.kernel, kv.second.cfg.rows_in_flight,
                         kv.second.cfg.trials_per_item, kv.second.cfg.blocks_per_sm, kv.second.ms);
        std::fclose(f);
    });
}

are_status are_tune_load(are_ctx *ctx, const char *path)
{
    return guarded(ctx, [&] {
        ARE_CHECK(path, ARE_EINVAL, "path is NULL");
        FILE *f = std::fopen(path, "r");
        ARE_CHECK(f, ARE_ENOTFOUND, std::string("cannot read ") + path);
        char line[512], key[256];
        int loaded = 0;
        while (std::fgets(line, sizeof line, f)) {
            TuneEntry e;
            double ms = 0;
            if (std::sscanf(line,
                            "{\"key\": \"%255[^\"]\", \"kernel\": %d, \"rows_in_flight\": %d, "
                            "\"trials_per_item\": %d, \"blocks_per_sm\": %d, \"ms\": %lf}",
                            key, &e.kernel, &e.cfg.rows_in_flight, &e.cfg.trials_per_item,
                            &e.cfg.blocks_per_sm, &ms) == 6 &&
                e.kernel >= 0 && e.kernel <= 3 && e.cfg.rows_in_flight >= 0 && e.cfg.rows_in_flight <= 2 &&
                e.cfg.trials_per_item > 0) {
                e.ms = ms;
                ctx->tune[key] = e;
                ++loaded;
            }
        }
        std::fclose(f);
        ARE_CHECK(loaded > 0, ARE_EINVAL, std::string("no tuning entries in ") + path);
    });
}

}  // extern "C"
