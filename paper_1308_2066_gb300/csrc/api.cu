// api.cu -- host implementation of the C ABI declared in include/are.h:
// context and handle management, input validation, memory-budget
// accounting, the per-layer table cache and kernel dispatch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <unordered_map>

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

// Device allocation charged to the context's budget.
void *dalloc(are_ctx *ctx, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    ARE_CHECK(ctx->budget == 0 || ctx->used + bytes <= ctx->budget, ARE_ENOMEM,
              "memory budget exceeded: need " + std::to_string(bytes) + " bytes, " +
                  std::to_string(ctx->budget - ctx->used) + " left");
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw Error{e == cudaErrorMemoryAllocation ? ARE_ENOMEM : ARE_ECUDA,
                    std::string("cudaMalloc: ") + cudaGetErrorString(e)};
    }
    ctx->used += bytes;
    return p;
}

void dfree(are_ctx *ctx, void *p, size_t bytes)
{
    if (!p) return;
    cudaFree(p);
    if (bytes == 0) bytes = 16;
    ctx->used -= std::min(ctx->used, bytes);
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

// Build (or rebuild) the layer's table for `catalog` in fp32 or fp64.
Table &build_table(are_ctx *ctx, Layer &L, int32_t catalog, bool fp32, cudaStream_t s)
{
    Table &t = fp32 ? L.t32 : L.t64;
    const int jp = table_jp((int)L.elts.size(), fp32);
    const size_t bytes = (size_t)catalog * jp * (fp32 ? 4 : 8);
    if (t.d && (t.catalog != catalog || t.jp != jp)) free_table(ctx, t);
    if (!t.d) {
        t.d = dalloc(ctx, bytes);
        t.bytes = bytes;
        t.catalog = catalog;
        t.jp = jp;
    }
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
    }
    ARE_CUDA_TRY(cudaMemsetAsync(t.d, 0, bytes, s));
    ctx->launches += launch_scatter_table(t.d, fp32, a, s);
    return t;
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

void fill_terms(are_ctx *ctx, const Layer &L, TermsF32 &t32, TermsF64 &t64, int &any_share)
{
    std::memset(&t32, 0, sizeof t32);
    std::memset(&t64, 0, sizeof t64);
    any_share = 0;
    for (int j = 0; j < kMaxElts; ++j) {
        t32.share[j] = 1.f;
        t64.share[j] = 1.0;
    }
    for (size_t j = 0; j < L.elts.size(); ++j) {
        const are_fin_terms &f = ctx->elts.at(L.elts[j]).terms;
        t64.ded[j] = f.deductible;
        t64.lim[j] = f.limit;
        t64.share[j] = f.share;
        t32.ded[j] = (float)f.deductible;
        t32.lim[j] = (float)f.limit;
        t32.share[j] = (float)f.share;
        any_share |= f.share != 1.0;
    }
    t64.occ_r = L.terms.occ_ret;
    t64.occ_l = L.terms.occ_lim;
    t32.occ_r = (float)L.terms.occ_ret;
    t32.occ_l = (float)L.terms.occ_lim;
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
    {
        std::lock_guard<std::recursive_mutex> lock(ctx->mu);
        cudaSetDevice(ctx->device);
        if (ctx->stream) cudaStreamSynchronize(ctx->stream);
        for (auto &kv : ctx->layers) {
            free_table(ctx, kv.second.t32);
            free_table(ctx, kv.second.t64);
        }
        for (auto &kv : ctx->elts) {
            dfree(ctx, kv.second.d_ids, 0);
            dfree(ctx, kv.second.d_loss, 0);
        }
        for (auto &kv : ctx->yets) {
            dfree(ctx, kv.second.d_ids, 0);
            dfree(ctx, kv.second.d_off, 0);
        }
        select_free(ctx->sel);
        if (ctx->d_flag) cudaFree(ctx->d_flag);
        if (ctx->h_flag) cudaFreeHost(ctx->h_flag);
        if (ctx->h_result) cudaFreeHost(ctx->h_result);
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
        ARE_CHECK(yet_handle, ARE_EINVAL, "yet_handle is NULL");
        ARE_CHECK(catalog_size > 0, ARE_EINVAL, "catalog_size must be > 0");
        ARE_CHECK(n_trials >= 0, ARE_EINVAL, "n_trials must be >= 0");
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
        for (int32_t i = 0; i < n_entries; ++i) {
            ARE_CHECK(ids[i] >= 0, ARE_EINVAL, "negative event id in ELT");
            ARE_CHECK(nonneg_finite(loss[i]), ARE_EINVAL, "ELT losses must be finite and >= 0");
            ARE_CHECK(std::isfinite(f.fx * loss[i]), ARE_EINVAL, "fx * loss overflows");
            max_id = std::max(max_id, ids[i]);
        }
        std::vector<int32_t> sorted(ids);
        std::sort(sorted.begin(), sorted.end());
        ARE_CHECK(std::adjacent_find(sorted.begin(), sorted.end()) == sorted.end(), ARE_EINVAL,
                  "duplicate event id within one ELT");
        Elt e;
        e.n = n_entries;
        e.max_id = max_id;
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
        L.terms = t;
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
        for (int32_t e : L.elts) ctx->elts[e].users--;
        ctx->layers.erase(h);
    });
}

are_status are_prepare(are_ctx *ctx, int32_t layer, int32_t yet, are_precision precision,
                       void *stream)
{
    return guarded(ctx, [&] {
        check_precision(precision);
        Layer &L = layer_of(ctx, layer);
        Yet &y = yet_of(ctx, yet);
        CallStream cs(ctx, stream);
        build_table(ctx, L, y.catalog, precision != ARE_FP64, cs.s);
        cs.finish();
    });
}

are_status are_simulate(are_ctx *ctx, int32_t layer, int32_t yet, int64_t trial_begin,
                        int64_t n_trials, are_precision precision, double *ylt, void *stream)
{
    return guarded(ctx, [&] {
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
        Table &t = fp32 ? L.t32 : L.t64;
        if (!t.d || t.catalog != y.catalog) build_table(ctx, L, y.catalog, fp32, s);
        const bool dev_out = is_device_ptr(ylt);
        double *d_out = ylt;
        if (!dev_out) d_out = (double *)dalloc(ctx, sizeof(double) * n_trials);
        try {
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
            TermsF32 t32;
            TermsF64 t64;
            fill_terms(ctx, L, t32, t64, a.any_share);
            ctx->launches += launch_simulate(a, precision, t.jp, &t32, &t64, ctx->num_sms, s);
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

are_status are_risk_measures(are_ctx *ctx, const double *ylt, int64_t n,
                             const double *return_periods, int32_t n_rp, double *pml_out,
                             const double *tvar_levels, int32_t n_tv, double *tvar_out,
                             void *stream)
{
    return guarded(ctx, [&] {
        ARE_CHECK(n > 0 && ylt, ARE_EINVAL, "need a YLT of n > 0 losses");
        ARE_CHECK(n < (int64_t)UINT32_MAX, ARE_EINVAL, "YLT too long for the selection counters");
        ARE_CHECK(n_rp >= 0 && n_tv >= 0, ARE_EINVAL, "negative count");
        ARE_CHECK(n_rp == 0 || (return_periods && pml_out), ARE_EINVAL, "NULL PML arrays");
        ARE_CHECK(n_tv == 0 || (tvar_levels && tvar_out), ARE_EINVAL, "NULL TVaR arrays");
        std::vector<int64_t> ranks;
        for (int32_t r = 0; r < n_rp; ++r) ranks.push_back(rank_rp(n, return_periods[r]));
        for (int32_t r = 0; r < n_tv; ++r) ranks.push_back(rank_level(n, tvar_levels[r]));
        if (ranks.empty()) return;
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

}  // extern "C"
