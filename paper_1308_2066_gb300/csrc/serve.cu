// serve.cu -- the real-time pricing scenario (Section I and IV: contract
// terms priced while an underwriter is on the phone) as a continuously
// batching server over a resident YET and the context's resident ELTs.
//
// A scheduler thread owns a CUDA stream.  Each iteration it
//   1. admits queued requests in arrival order while a request slot and
//      arena memory for the request's table and YLT are free (admission by
//      memory), building each admitted request's direct-access table;
//   2. hands out events_per_launch to the running requests in arrival
//      order (the oldest runs whole, the others share the budget), or
//      (least_work_first) in order of least remaining work less the time
//      each has already waited (so a long request is not overtaken for
//      ever by short ones that keep arriving); each takes what it needs,
//      the last one a partial slice.  The slices of small
//      requests run in one persistent launch of the multi-layer kernel (one
//      launch per table width); a request of at least kLargeSlice events
//      runs its slices on the single-layer register-rows kernel, which is
//      faster per event.  The kernel is chosen per request, so a request's
//      result does not depend on the requests around it;
//   3. selects PML/TVaR for the requests whose last slice was in the launch;
//   4. waits (bounded) for the previous iteration and posts its results.
// One iteration is always queued ahead of the one being waited for, so the
// GPU is not left idle while the host reacts.
//
// With cfg.folded set, each admitted request gets a folded table instead
// (its FP64 occurrence loss per catalog event, as are_prepare_folded builds
// it) and its slices run on the folded trial kernel: one lookup per
// occurrence and exact trial sums -- the folded-table variant of the method.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <thread>

#include "are_internal.cuh"

namespace are {

namespace {

using Clock = std::chrono::steady_clock;
constexpr int kMaxSlots = 256;
constexpr int kWidths3[3] = {8, 16, 32};
constexpr size_t kAlign = 256;
constexpr int64_t kWaitLimitUs = 120LL * 1000 * 1000;   // one iteration may not take longer
constexpr double kLargeSlice = 32e6;         // events: a request this large runs on its own kernel
constexpr double kEventsPerUs = 2.4e5;        // occurrences per microsecond (a table row each), for the aging

size_t up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

double us_between(Clock::time_point a, Clock::time_point b)
{
    return std::chrono::duration<double, std::micro>(b - a).count();
}

// First-fit allocator over one device allocation.
struct Arena {
    char *base = nullptr;
    size_t size = 0;
    std::map<size_t, size_t> free_;   // offset -> bytes
    void reset(char *b, size_t n)
    {
        base = b;
        size = n;
        free_.clear();
        if (n) free_[0] = n;
    }
    bool take(size_t n, size_t &off)
    {
        n = up(n);
        for (auto it = free_.begin(); it != free_.end(); ++it)
            if (it->second >= n) {
                off = it->first;
                const size_t rest = it->second - n;
                free_.erase(it);
                if (rest) free_[off + n] = rest;
                return true;
            }
        return false;
    }
    void give(size_t off, size_t n)
    {
        n = up(n);
        auto it = free_.emplace(off, n).first;
        auto next = std::next(it);
        if (next != free_.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_.erase(it);
            }
        }
    }
};

struct Request {
    int64_t ticket = 0;
    std::vector<int32_t> elts;
    are_layer_terms terms{};
    int64_t n_trials = 0;
    int64_t entries = 0;            // ELT entries of the request's layer
    int n_rp = 0, n_tv = 0;
    int64_t ranks[kMaxTargets] = {};
    Clock::time_point t_submit;
};

struct Slot {
    bool busy = false, cancelled = false, finishing = false;
    Request req;
    int jp = 0;
    size_t tab_off = 0, tab_bytes = 0, ylt_off = 0, ylt_bytes = 0;
    LayerF32 rec{};
    int64_t launched = 0;           // trials handed to launches so far
    bool large = false;             // its slices run on the single-layer register-rows kernel
    int pw = 0;                     // large: words per packed row (0: the dense rows)
    size_t dense_bytes = 0;         // the dense table (0 for packed rows, which fill the block)
    uint64_t finish_iter = 0;       // iteration whose completion posts the result
    cudaEvent_t done_ev = nullptr;  // recorded after the result's copy: posts it as soon as it fires
    SelectScratch sel;
    double *h_res = nullptr;        // pinned, 2 * kMaxTargets
    Clock::time_point t_admit;
};

struct Posted {
    bool ready = false;
    are_result res{};
};

}  // namespace

struct Server {
    are_ctx *ctx = nullptr;
    int32_t yet = 0;
    are_server_cfg cfg{};
    const Yet *y = nullptr;
    double mean_events = 0;
    std::thread th;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request> pending;
    std::map<int64_t, Posted> results;
    std::map<int64_t, int> running;  // ticket -> slot
    int64_t next_ticket = 1;
    bool stop = false;
    are_status failed = ARE_OK;
    std::string fail_msg;
    std::vector<Slot> slots;
    Arena arena;
    char *d_arena = nullptr;
    cudaStream_t stream = nullptr;
    // double-buffered work lists of the iterations
    LayerF32 *h_layers[2] = {nullptr, nullptr};
    void *d_work[2] = {nullptr, nullptr};
    size_t work_bytes = 0;
    cudaEvent_t iter_done[2] = {nullptr, nullptr};
    uint64_t iter = 0;
};

namespace {

void add_launches(Server &S, int n)
{
    std::lock_guard<std::recursive_mutex> lk(S.ctx->mu);
    S.ctx->launches += (uint64_t)n;
}

void post(Server &S, const Request &r, are_status st, const double *res, Clock::time_point t_admit,
          bool admitted)
{
    Posted p;
    p.ready = true;
    p.res.status = st;
    p.res.n_rp = r.n_rp;
    p.res.n_tv = r.n_tv;
    p.res.n_trials = r.n_trials;
    if (res) {
        for (int i = 0; i < r.n_rp; ++i) p.res.pml[i] = res[2 * i];
        for (int i = 0; i < r.n_tv; ++i) p.res.tvar[i] = res[2 * (r.n_rp + i) + 1];
    }
    const Clock::time_point now = Clock::now();
    p.res.total_us = us_between(r.t_submit, now);
    p.res.queue_us = admitted ? us_between(r.t_submit, t_admit) : p.res.total_us;
    p.res.run_us = admitted ? us_between(t_admit, now) : 0.0;
    S.results[r.ticket] = p;
}

// A folded table in an arena block: [hmax | 248 B][bits][F].
size_t folded_block_bytes(int32_t catalog)
{
    return 256 + up((size_t)folded_words(catalog) * 4) + (size_t)catalog * 16;
}
unsigned long long *folded_hmax(char *b) { return reinterpret_cast<unsigned long long *>(b); }
uint32_t *folded_bits(char *b) { return reinterpret_cast<uint32_t *>(b + 256); }
ulonglong2 *folded_F(char *b, int32_t catalog)
{
    return reinterpret_cast<ulonglong2 *>(b + 256 + up((size_t)folded_words(catalog) * 4));
}

// A large request's packed rows in its arena block: [rows | counter (256 B) |
// overflow].
uint32_t *packed_rows(Server &S, const Slot &sl)
{
    return reinterpret_cast<uint32_t *>(S.d_arena + sl.tab_off + up(sl.dense_bytes));
}
unsigned long long *packed_used(Server &S, const Slot &sl)
{
    return reinterpret_cast<unsigned long long *>(
        reinterpret_cast<char *>(packed_rows(S, sl)) + up((size_t)S.y->catalog * sl.pw * sizeof(float)));
}
float *packed_ovf(Server &S, const Slot &sl)
{
    return reinterpret_cast<float *>(reinterpret_cast<char *>(packed_used(S, sl)) + 256);
}

// Table of an admitted request, built on the server stream in its arena block.
void build_request_table(Server &S, Slot &sl)
{
    ScatterArgs a{};
    {
        std::lock_guard<std::recursive_mutex> lk(S.ctx->mu);
        a.n_elts = (int32_t)sl.req.elts.size();
        a.jp = sl.jp;
        for (size_t j = 0; j < sl.req.elts.size(); ++j) {
            const Elt &e = S.ctx->elts.at(sl.req.elts[j]);
            a.ids[j] = e.d_ids;
            a.loss[j] = e.d_loss;
            a.n[j] = e.n;
            a.fx[j] = e.terms.fx;
            a.ded[j] = e.terms.deductible;
            a.lim[j] = e.terms.limit;
            a.share[j] = e.terms.share;
        }
    }
    if (S.cfg.folded) {
        char *b = S.d_arena + sl.tab_off;
        add_launches(S, launch_fold(a, sl.req.terms.occ_ret, sl.req.terms.occ_lim, S.y->catalog,
                                    folded_F(b, S.y->catalog), folded_bits(b), folded_hmax(b),
                                    S.ctx->num_sms, S.stream));
        return;
    }
    if (sl.pw) {   // packed rows straight from the ELT entries
        add_launches(S, launch_pack32_direct(a, S.y->catalog, sl.pw, packed_rows(S, sl), packed_ovf(S, sl),
                                             packed_used(S, sl), S.stream));
        return;
    }
    char *b = S.d_arena + sl.tab_off;
    ARE_CUDA_TRY(cudaMemsetAsync(b, 0, sl.dense_bytes, S.stream));
    add_launches(S, launch_scatter_table(b, true, a, S.stream));
}

void fill_record(Server &S, Slot &sl)
{
    LayerF32 &o = sl.rec;
    std::memset(&o, 0, sizeof o);
    o.table = reinterpret_cast<const float *>(S.d_arena + sl.tab_off);
    o.ylt = reinterpret_cast<double *>(S.d_arena + sl.ylt_off);
    o.jp = sl.jp;
    o.occ_r = (float)sl.req.terms.occ_ret;
    o.occ_l = (float)sl.req.terms.occ_lim;
    o.agg_r = sl.req.terms.agg_ret;
    o.agg_l = sl.req.terms.agg_lim;
}

// A request's terms with -0.0 read as +0.0 (as are_define_layer does): the
// kernels compare non-negative doubles by their bit patterns.
are_layer_terms positive_zeros(are_layer_terms t)
{
    for (double *x : {&t.occ_ret, &t.occ_lim, &t.agg_ret, &t.agg_lim})
        if (*x == 0.0) *x = 0.0;
    return t;
}

// Posts slot sl's result (or drops it when cancelled) and frees the slot.
// Caller holds S.mu.
void release_slot(Server &S, Slot &sl)
{
    if (sl.cancelled) {
        S.results.erase(sl.req.ticket);
    } else {
        post(S, sl.req, ARE_OK, sl.h_res, sl.t_admit, true);
    }
    S.running.erase(sl.req.ticket);
    S.arena.give(sl.tab_off, sl.tab_bytes);
    S.arena.give(sl.ylt_off, sl.ylt_bytes);
    sl.busy = sl.cancelled = sl.finishing = false;
    sl.launched = 0;
}

// Posts the results of every slot whose last iteration has completed.
void retire(Server &S, uint64_t completed_iter)
{
    std::lock_guard<std::mutex> lk(S.mu);
    for (int i = 0; i < (int)S.slots.size(); ++i) {
        Slot &sl = S.slots[i];
        if (!sl.busy) continue;
        const bool done = sl.finishing && sl.finish_iter <= completed_iter;
        const bool dropped = sl.cancelled && (!sl.finishing || done) && sl.finish_iter <= completed_iter;
        if (!done && !dropped) continue;
        release_slot(S, sl);
    }
    S.cv_done.notify_all();
    S.cv_work.notify_all();
}

// Posts the results whose own work has finished, before the rest of their
// iteration has: a request's latency is its own work and what ran before it.
void retire_finished(Server &S)
{
    std::lock_guard<std::mutex> lk(S.mu);
    bool any = false;
    for (Slot &sl : S.slots) {
        if (!sl.busy || !sl.finishing || sl.cancelled) continue;
        const cudaError_t e = cudaEventQuery(sl.done_ev);
        if (e == cudaErrorNotReady) continue;
        if (e != cudaSuccess) throw Error{ARE_ECUDA, std::string("server: ") + cudaGetErrorString(e)};
        release_slot(S, sl);
        any = true;
    }
    if (any) {
        S.cv_done.notify_all();
        S.cv_work.notify_all();
    }
}

// Waits for an event without blocking forever (the GPU is shared), posting
// the results that finish meanwhile.
bool bounded_wait(Server &S, cudaEvent_t ev)
{
    const Clock::time_point t0 = Clock::now();
    for (;;) {
        const cudaError_t e = cudaEventQuery(ev);
        if (e == cudaSuccess) return true;
        if (e != cudaErrorNotReady) throw Error{ARE_ECUDA, std::string("server: ") + cudaGetErrorString(e)};
        retire_finished(S);
        if (us_between(t0, Clock::now()) > kWaitLimitUs) return false;
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

void fail_all(Server &S, are_status st, const std::string &msg)
{
    std::lock_guard<std::mutex> lk(S.mu);
    S.failed = st;
    S.fail_msg = msg;
    for (Slot &sl : S.slots)
        if (sl.busy && !sl.cancelled) post(S, sl.req, st, nullptr, sl.t_admit, true);
    for (const Request &r : S.pending) post(S, r, st, nullptr, r.t_submit, false);
    S.pending.clear();
    S.running.clear();
    S.cv_done.notify_all();
}

void scheduler(Server *SP)
{
    Server &S = *SP;
    const int tpi = S.cfg.trials_per_item > 0 ? S.cfg.trials_per_item : 8;
    // events per iteration (a folded table's occurrence costs far less)
    const int64_t budget = S.cfg.events_per_launch > 0 ? S.cfg.events_per_launch
                                                       : S.cfg.folded ? 1000000000 : 200000000;
    try {
        ARE_CUDA_TRY(cudaSetDevice(S.ctx->device));
        for (;;) {
            std::vector<int> admitted;
            {
                std::unique_lock<std::mutex> lk(S.mu);
                bool any_busy = false;
                for (const Slot &sl : S.slots) any_busy |= sl.busy;
                if (!any_busy && S.pending.empty()) {
                    if (S.stop) break;
                    S.cv_work.wait_for(lk, std::chrono::milliseconds(2));
                    continue;
                }
                // admission in arrival order, while a slot and arena memory are free
                while (!S.pending.empty()) {
                    if (S.cfg.one_at_a_time && any_busy) break;
                    int free_slot = -1;
                    for (int i = 0; i < (int)S.slots.size(); ++i)
                        if (!S.slots[i].busy) {
                            free_slot = i;
                            break;
                        }
                    if (free_slot < 0) break;
                    Request &r = S.pending.front();
                    Slot &sl = S.slots[free_slot];
                    sl.jp = table_jp((int)r.elts.size(), true);
                    sl.large = (double)r.n_trials * S.mean_events >= kLargeSlice;
                    // a large request's single-layer kernel reads packed rows
                    // where the layer's entries per catalog event are few
                    sl.pw = sl.large && !S.cfg.folded
                                ? packed_row_words((int)r.elts.size(),
                                                   (double)r.entries / (double)S.y->catalog, true)
                                : 0;
                    sl.dense_bytes = sl.pw ? 0 : (size_t)S.y->catalog * sl.jp * sizeof(float);
                    sl.tab_bytes = S.cfg.folded ? folded_block_bytes(S.y->catalog)
                                   : sl.pw ? up((size_t)S.y->catalog * sl.pw * sizeof(float)) + 256 +
                                                 up(sizeof(float) * (size_t)r.entries + 8)
                                           : sl.dense_bytes;
                    sl.ylt_bytes = sizeof(double) * (size_t)r.n_trials;
                    size_t a = 0, b = 0;
                    if (!S.arena.take(sl.tab_bytes, a)) break;
                    if (!S.arena.take(sl.ylt_bytes, b)) {
                        S.arena.give(a, sl.tab_bytes);
                        break;
                    }
                    sl.tab_off = a;
                    sl.ylt_off = b;
                    sl.req = std::move(r);
                    S.pending.pop_front();
                    sl.busy = true;
                    sl.cancelled = sl.finishing = false;
                    sl.launched = 0;
                    sl.t_admit = Clock::now();
                    S.running[sl.req.ticket] = free_slot;
                    admitted.push_back(free_slot);
                    any_busy = true;
                }
            }
            for (int i : admitted) {
                build_request_table(S, S.slots[i]);
                fill_record(S, S.slots[i]);
            }

            // Slices of this iteration: running requests in arrival order
            // (or least remaining work first), each taking what is left of
            // the event budget.  Arrival order keeps a request from being
            // stretched by later ones -- with request sizes bounded that
            // gives the lowest tail latency; least work first lets short
            // requests overtake long ones.  Either way a launch touches only
            // a few requests' tables, which keeps them resident in L2.
            const int buf = (int)(S.iter & 1);
            std::vector<int> part[3], big, fold;
            std::vector<int64_t> slice;
            bool big_first = false;   // the oldest request is a large one: its launch goes first
            {
                std::lock_guard<std::mutex> lk(S.mu);
                std::vector<std::pair<double, int>> order;
                const Clock::time_point now = Clock::now();
                for (int i = 0; i < (int)S.slots.size(); ++i) {
                    const Slot &sl = S.slots[i];
                    if (!sl.busy || sl.cancelled || sl.launched >= sl.req.n_trials) continue;
                    // arrival order: the time since submission, longest first;
                    // least work first: remaining GPU time (estimated: a row
                    // gather per occurrence) less the time since submission
                    const double waited = us_between(sl.req.t_submit, now);
                    const double work_us = (double)(sl.req.n_trials - sl.launched) * S.mean_events / kEventsPerUs;
                    order.emplace_back(S.cfg.least_work_first ? work_us - waited : -waited, i);
                }
                std::sort(order.begin(), order.end());
                slice.assign(S.slots.size(), 0);
                double left_budget = (double)budget / std::max(1.0, S.mean_events);  // in trials
                for (const auto &o : order) {
                    Slot &sl = S.slots[o.second];
                    const int64_t left = sl.req.n_trials - sl.launched;
                    int64_t take = left;
                    // in arrival order the oldest request runs whole: nothing
                    // may overtake it, so cutting it into slices would only
                    // add launches; the requests behind it share the budget
                    const bool head = !S.cfg.least_work_first && &o == &order.front();
                    if (!S.cfg.one_at_a_time && !head) {
                        if (left_budget < tpi) break;
                        take = std::min<int64_t>(left, (int64_t)left_budget / tpi * tpi);
                        if (take < left && take < tpi) take = std::min<int64_t>(left, tpi);
                    }
                    slice[o.second] = take;
                    left_budget -= (double)take;
                    if (head) big_first = sl.large && !S.cfg.folded;
                    if (S.cfg.folded)
                        fold.push_back(o.second);
                    else if (sl.large)
                        big.push_back(o.second);
                    else
                        part[sl.jp == 8 ? 0 : sl.jp == 16 ? 1 : 2].push_back(o.second);
                }
            }
            if (S.cfg.stall_us > 0) std::this_thread::sleep_for(std::chrono::microseconds(S.cfg.stall_us));
            // work list: records by table width, then three counters
            size_t offs[3], off = 0;
            for (int g = 0; g < 3; ++g) {
                offs[g] = off;
                off += up(sizeof(LayerF32) * part[g].size());
            }
            LayerF32 *h = S.h_layers[buf];
            unsigned char *d = static_cast<unsigned char *>(S.d_work[buf]);
            for (int g = 0; g < 3; ++g) {
                int64_t next = 0;
                for (size_t k = 0; k < part[g].size(); ++k) {
                    Slot &sl = S.slots[part[g][k]];
                    LayerF32 r = sl.rec;
                    r.t0 = sl.launched;
                    r.nt = slice[part[g][k]];
                    r.item_begin = next;
                    next += (r.nt + tpi - 1) / tpi;
                    std::memcpy(reinterpret_cast<unsigned char *>(h) + offs[g] + k * sizeof(LayerF32),
                                &r, sizeof r);
                }
            }
            if (off)
                ARE_CUDA_TRY(cudaMemcpyAsync(d, h, off, cudaMemcpyHostToDevice, S.stream));
            int launches = 0;
            // A request whose last slice is in this launch has its risk
            // measures selected and copied right after its own kernels, then
            // its own completion event: its result is posted when that
            // fires, not when the whole iteration has.
            auto finish_if_last = [&](int i) {
                std::lock_guard<std::mutex> lk(S.mu);
                Slot &sl = S.slots[i];
                sl.launched += slice[i];
                if (sl.launched < sl.req.n_trials) return;
                launches += launch_select(reinterpret_cast<const double *>(S.d_arena + sl.ylt_off),
                                          sl.req.n_trials, sl.req.ranks, sl.req.n_rp + sl.req.n_tv, sl.sel,
                                          S.ctx->num_sms, S.stream);
                ARE_CUDA_TRY(cudaMemcpyAsync(sl.h_res, sl.sel.result, sizeof(double) * 2 * kMaxTargets,
                                             cudaMemcpyDeviceToHost, S.stream));
                ARE_CUDA_TRY(cudaEventRecord(sl.done_ev, S.stream));
                sl.finishing = true;
                sl.finish_iter = S.iter;
            };
            // small requests, many per persistent launch, then the folded tables
            auto launch_small = [&] {
                for (int g = 0; g < 3; ++g) {
                    if (part[g].empty()) continue;
                    ItemWork w;
                    std::memset(&w, 0, sizeof w);
                    w.ids = S.y->d_ids;
                    w.off = S.y->d_off;
                    w.k = S.y->k;
                    w.trial_begin = 0;
                    w.n_trials = S.y->n_trials;
                    w.trials_per_item = tpi;
                    w.layers = reinterpret_cast<const LayerF32 *>(d + offs[g]);
                    w.n_layers = (int32_t)part[g].size();
                    int64_t items = 0;
                    for (int i : part[g]) items += (slice[i] + tpi - 1) / tpi;
                    w.n_items = items;
                    w.counter = reinterpret_cast<unsigned long long *>(d + off) + g;
                    ARE_CUDA_TRY(cudaMemsetAsync(w.counter, 0, sizeof(unsigned long long), S.stream));
                    ItemConfig cfg;
                    cfg.trials_per_item = tpi;
                    cfg.rows_in_flight = 2;
                    launches += launch_items(w, kWidths3[g], cfg, S.cfg.precision, S.ctx->num_sms, S.stream);
                    for (int i : part[g]) finish_if_last(i);
                }
                // folded tables: one trial-pass launch per request slice
                for (int i : fold) {
                    const Slot &sl = S.slots[i];
                    char *b = S.d_arena + sl.tab_off;
                    FoldArgs fa{};
                    fa.ids = S.y->d_ids;
                    fa.off = S.y->d_off;
                    fa.k = S.y->k;
                    fa.trial_begin = sl.launched;
                    fa.n_trials = slice[i];
                    fa.n_events = S.y->n_events;
                    fa.F = folded_F(b, S.y->catalog);
                    fa.bits = folded_bits(b);
                    fa.words = folded_words(S.y->catalog);
                    fa.hmax = folded_hmax(b);
                    fa.agg_r = sl.req.terms.agg_ret;
                    fa.agg_l = sl.req.terms.agg_lim;
                    fa.ylt = reinterpret_cast<double *>(S.d_arena + sl.ylt_off) + sl.launched;
                    launches += launch_folded(fa, S.ctx->num_sms, S.stream);
                    finish_if_last(i);
                }
            };
            auto launch_large = [&] {
                // large slices, one single-layer register-rows launch each
                for (int i : big) {
                    const Slot &sl = S.slots[i];
                    SimArgs sa;
                    std::memset(&sa, 0, sizeof sa);
                    sa.ids = S.y->d_ids;
                    sa.off = S.y->d_off;
                    sa.k = S.y->k;
                    sa.trial_begin = sl.launched;
                    sa.n_trials = slice[i];
                    sa.table = sl.rec.table;
                    sa.agg_r = sl.rec.agg_r;
                    sa.agg_l = sl.rec.agg_l;
                    sa.ylt = sl.rec.ylt + sl.launched;
                    sa.kernel = 2;
                    sa.epl = 0;   // the kernel's default batch for the row width
                    if (sl.pw) {   // over the packed rows
                        sa.table = packed_rows(S, sl);
                        sa.table2 = packed_ovf(S, sl);
                        sa.kernel = 5;
                    }
                    TermsF32 tm;
                    tm.occ_r = sl.rec.occ_r;
                    tm.occ_l = sl.rec.occ_l;
                    launches += launch_simulate(sa, S.cfg.precision, sl.pw ? sl.pw : sl.jp, &tm, nullptr,
                                                S.ctx->num_sms, S.stream);
                    finish_if_last(i);
                }
            };
            // the oldest request's kind of work first
            if (big_first) {
                launch_large();
                launch_small();
            } else {
                launch_small();
                launch_large();
            }
            {
                std::lock_guard<std::mutex> lk(S.mu);
                // cancelled slots with nothing in flight retire with this iteration
                for (Slot &sl : S.slots)
                    if (sl.busy && sl.cancelled && !sl.finishing) sl.finish_iter = S.iter;
            }
            add_launches(S, launches);
            ARE_CUDA_TRY(cudaEventRecord(S.iter_done[buf], S.stream));
            // wait for the previous iteration (this one stays queued behind it)
            if (S.iter > 0) {
                if (!bounded_wait(S, S.iter_done[buf ^ 1]))
                    throw Error{ARE_ETIMEOUT, "server: a launch did not finish within its time limit"};
                retire(S, S.iter - 1);
            }
            ++S.iter;
            // nothing new to launch: drain this iteration too
            bool more = false;
            {
                std::lock_guard<std::mutex> lk(S.mu);
                for (const Slot &sl : S.slots)
                    more |= sl.busy && !sl.cancelled && sl.launched < sl.req.n_trials;
                more |= !S.pending.empty();
            }
            if (!more) {
                if (!bounded_wait(S, S.iter_done[buf]))
                    throw Error{ARE_ETIMEOUT, "server: a launch did not finish within its time limit"};
                retire(S, S.iter - 1);
            }
        }
    } catch (const Error &e) {
        fail_all(S, e.code, e.msg);
    } catch (...) {
        fail_all(S, ARE_ECUDA, "server: unexpected failure");
    }
}

}  // namespace

void server_free(Server *S)
{
    if (!S) return;
    if (S->stream) cudaStreamSynchronize(S->stream);
    for (Slot &sl : S->slots) {
        select_free(sl.sel);
        if (sl.h_res) cudaFreeHost(sl.h_res);
        if (sl.done_ev) cudaEventDestroy(sl.done_ev);
    }
    for (int b = 0; b < 2; ++b) {
        if (S->h_layers[b]) cudaFreeHost(S->h_layers[b]);
        if (S->d_work[b]) ctx_free(S->ctx, S->d_work[b], S->work_bytes);
        if (S->iter_done[b]) cudaEventDestroy(S->iter_done[b]);
    }
    if (S->d_arena) ctx_free(S->ctx, S->d_arena, S->arena.size);
    if (S->stream) cudaStreamDestroy(S->stream);
    delete S;
}

void server_destroy(are_ctx *ctx)
{
    Server *S = ctx->server;
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        for (const Request &r : S->pending) S->results.erase(r.ticket);
        S->pending.clear();
    }
    S->cv_work.notify_all();
    if (S->th.joinable()) S->th.join();
    ctx->server = nullptr;
    server_free(S);
}

}  // namespace are

using namespace are;

namespace {

template <typename F>
are_status server_call(are_ctx *ctx, F &&fn)
{
    if (!ctx) return ARE_EINVAL;
    try {
        fn();
        set_error(ctx, "");
        return ARE_OK;
    } catch (const Error &e) {
        set_error(ctx, e.msg);
        return e.code;
    } catch (const std::bad_alloc &) {
        set_error(ctx, "host allocation failed");
        return ARE_ENOMEM;
    }
}

}  // namespace

extern "C" {

are_status are_server_start(are_ctx *ctx, int32_t yet, const are_server_cfg *cfg)
{
    return server_call(ctx, [&] {
        std::lock_guard<std::recursive_mutex> lk(ctx->mu);
        ARE_CHECK(cfg, ARE_EINVAL, "cfg is NULL");
        ARE_CHECK(!ctx->server, ARE_EBUSY, "a server is already running on this context");
        auto it = ctx->yets.find(yet);
        ARE_CHECK(it != ctx->yets.end(), ARE_ENOTFOUND, "unknown YET handle " + std::to_string(yet));
        ARE_CHECK(cfg->max_inflight >= 1 && cfg->max_inflight <= kMaxSlots, ARE_EINVAL,
                  "max_inflight must lie in 1..256");
        ARE_CHECK(cfg->max_pending >= 1, ARE_EINVAL, "max_pending must be >= 1");
        ARE_CHECK(cfg->arena_bytes >= 4096, ARE_EINVAL, "arena_bytes too small");
        ARE_CHECK(cfg->folded || cfg->precision == ARE_FP32_KAHAN || cfg->precision == ARE_FP32_FP64AGG,
                  ARE_EINVAL, "the server runs the FP32 table paths (or folded tables)");
        ARE_CHECK(cfg->trials_per_item >= 0 && cfg->events_per_launch >= 0 && cfg->stall_us >= 0,
                  ARE_EINVAL, "negative server setting");
        ARE_CUDA_TRY(cudaSetDevice(ctx->device));
        Server *S = new Server();
        S->ctx = ctx;
        S->yet = yet;
        S->cfg = *cfg;
        S->y = &it->second;
        S->mean_events = S->y->n_trials ? (double)S->y->n_events / (double)S->y->n_trials : 0.0;
        try {
            ARE_CUDA_TRY(cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking));
            S->d_arena = static_cast<char *>(ctx_alloc(ctx, cfg->arena_bytes));
            S->arena.reset(S->d_arena, cfg->arena_bytes);
            S->slots.resize(cfg->max_inflight);
            for (Slot &sl : S->slots) {
                select_alloc(sl.sel, ctx->num_sms);
                ARE_CUDA_TRY(cudaMallocHost(&sl.h_res, sizeof(double) * 2 * kMaxTargets));
                ARE_CUDA_TRY(cudaEventCreateWithFlags(&sl.done_ev, cudaEventDisableTiming));
            }
            S->work_bytes = 3 * up(sizeof(LayerF32) * cfg->max_inflight) + 3 * sizeof(unsigned long long);
            for (int b = 0; b < 2; ++b) {
                ARE_CUDA_TRY(cudaMallocHost(&S->h_layers[b], S->work_bytes));
                S->d_work[b] = ctx_alloc(ctx, S->work_bytes);
                ARE_CUDA_TRY(cudaEventCreateWithFlags(&S->iter_done[b], cudaEventDisableTiming));
            }
        } catch (...) {
            server_free(S);
            throw;
        }
        ctx->server = S;
        S->th = std::thread(scheduler, S);
    });
}

are_status are_submit(are_ctx *ctx, const are_request *req, int64_t *ticket)
{
    return server_call(ctx, [&] {
        ARE_CHECK(req && ticket, ARE_EINVAL, "NULL argument");
        Request r;
        {
            std::lock_guard<std::recursive_mutex> lk(ctx->mu);
            Server *S = ctx->server;
            ARE_CHECK(S, ARE_EINVAL, "no server is running");
            ARE_CHECK(req->n_elts >= 1 && req->n_elts <= kMaxElts && req->elt_handles, ARE_EINVAL,
                      "a request holds 1.." + std::to_string(kMaxElts) + " ELTs");
            ARE_CHECK(req->n_trials >= 1 && req->n_trials <= S->y->n_trials, ARE_EINVAL,
                      "n_trials must lie in 1..trials of the YET");
            ARE_CHECK(req->n_rp >= 0 && req->n_tv >= 0 && req->n_rp + req->n_tv >= 1 &&
                          req->n_rp + req->n_tv <= kMaxTargets,
                      ARE_EINVAL, "a request asks for 1..8 return periods and TVaR levels");
            ARE_CHECK(req->n_rp == 0 || req->return_periods, ARE_EINVAL, "return_periods is NULL");
            ARE_CHECK(req->n_tv == 0 || req->tvar_levels, ARE_EINVAL, "tvar_levels is NULL");
            const are_layer_terms &t = req->terms;
            ARE_CHECK(std::isfinite(t.occ_ret) && t.occ_ret >= 0 && std::isfinite(t.agg_ret) &&
                          t.agg_ret >= 0 && !std::isnan(t.occ_lim) && t.occ_lim >= 0 &&
                          !std::isnan(t.agg_lim) && t.agg_lim >= 0,
                      ARE_EINVAL, "bad layer terms");
            for (int32_t j = 0; j < req->n_elts; ++j) {
                auto e = ctx->elts.find(req->elt_handles[j]);
                ARE_CHECK(e != ctx->elts.end(), ARE_ENOTFOUND,
                          "unknown ELT handle " + std::to_string(req->elt_handles[j]));
                ARE_CHECK(e->second.max_id < S->y->catalog, ARE_EINVAL, "ELT id outside the YET's catalog");
                ARE_CHECK(std::find(r.elts.begin(), r.elts.end(), req->elt_handles[j]) == r.elts.end(),
                          ARE_EINVAL, "ELT appears twice in the request");
                r.elts.push_back(req->elt_handles[j]);
                r.entries += e->second.n;
            }
            for (int32_t i = 0; i < req->n_rp; ++i) {
                r.ranks[i] = rank_for_return_period(req->n_trials, req->return_periods[i]);
                ARE_CHECK(r.ranks[i] >= 1, ARE_EINVAL, "return period must be finite and >= 1");
            }
            for (int32_t i = 0; i < req->n_tv; ++i) {
                r.ranks[req->n_rp + i] = rank_for_level(req->n_trials, req->tvar_levels[i]);
                ARE_CHECK(r.ranks[req->n_rp + i] >= 1, ARE_EINVAL, "TVaR level must lie in (0, 1)");
            }
        }
        r.terms = positive_zeros(req->terms);
        r.n_trials = req->n_trials;
        r.n_rp = req->n_rp;
        r.n_tv = req->n_tv;
        r.t_submit = Clock::now();
        Server *S = ctx->server;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            ARE_CHECK(S->failed == ARE_OK, S->failed, S->fail_msg);
            ARE_CHECK(!S->stop, ARE_EINVAL, "the server is stopping");
            ARE_CHECK((int)S->pending.size() < S->cfg.max_pending, ARE_EBUSY, "the request queue is full");
            r.ticket = S->next_ticket++;
            *ticket = r.ticket;
            S->results[r.ticket] = Posted{};
            S->pending.push_back(std::move(r));
        }
        S->cv_work.notify_all();
    });
}

are_status are_wait(are_ctx *ctx, int64_t ticket, int64_t timeout_us, are_result *out)
{
    return server_call(ctx, [&] {
        ARE_CHECK(out, ARE_EINVAL, "out is NULL");
        Server *S = ctx->server;
        ARE_CHECK(S, ARE_EINVAL, "no server is running");
        std::unique_lock<std::mutex> lk(S->mu);
        auto ready = [&] {
            auto it = S->results.find(ticket);
            return it == S->results.end() || it->second.ready;
        };
        if (timeout_us < 0)
            S->cv_done.wait(lk, ready);
        else if (!S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready))
            throw Error{ARE_ETIMEOUT, "result not ready in time"};
        auto it = S->results.find(ticket);
        ARE_CHECK(it != S->results.end(), ARE_ENOTFOUND,
                  "unknown, already taken or cancelled ticket " + std::to_string(ticket));
        *out = it->second.res;
        S->results.erase(it);
    });
}

are_status are_cancel(are_ctx *ctx, int64_t ticket)
{
    return server_call(ctx, [&] {
        Server *S = ctx->server;
        ARE_CHECK(S, ARE_EINVAL, "no server is running");
        std::lock_guard<std::mutex> lk(S->mu);
        auto rit = S->results.find(ticket);
        ARE_CHECK(rit != S->results.end() && !rit->second.ready, ARE_ENOTFOUND,
                  "no queued or running request with ticket " + std::to_string(ticket));
        for (auto it = S->pending.begin(); it != S->pending.end(); ++it)
            if (it->ticket == ticket) {
                S->pending.erase(it);
                S->results.erase(ticket);
                S->cv_done.notify_all();
                return;
            }
        auto sit = S->running.find(ticket);
        ARE_CHECK(sit != S->running.end(), ARE_ENOTFOUND, "request is not queued or running");
        S->slots[sit->second].cancelled = true;
        S->results.erase(ticket);
        S->cv_done.notify_all();
        S->cv_work.notify_all();
    });
}

are_status are_server_stop(are_ctx *ctx)
{
    return server_call(ctx, [&] {
        ARE_CHECK(ctx->server, ARE_EINVAL, "no server is running");
        server_destroy(ctx);
    });
}

}  // extern "C"
