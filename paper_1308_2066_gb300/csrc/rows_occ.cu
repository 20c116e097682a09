// rows_occ.cu -- the per-occurrence outputs of the analysis stage (Basic
// Algorithm, Section II-B, step 4 before its final sum) over the rows the
// register-rows kernels read: for every occurrence its marginal m_d =
// A_d - A_{d-1} (A_d the aggregate-clamped running total, A_0 = 0), for
// every trial its largest occurrence loss and its loss A_k.
//
// The occurrence losses come from the layer's body (rows.cuh: packed FP64
// rows, the oracle's bit for bit; packed or dense FP32 rows), one event per
// lane per group of 32.  Within a trial the running total S_d is an exact
// fixed-point sum (fixed.cuh): a warp-shuffle inclusive scan of the group's
// 32 occurrence losses, in event order, on top of the total before it (a
// group without a loss only writes zero marginals).  The
// aggregate terms are applied to S_d in the same fixed point, so every A_d,
// every marginal and the trial loss are exact and rounded to double once;
// marginals are never negative.  Marginals are written coalesced, one
// 8-byte value per lane.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "are_internal.cuh"
#include "rows.cuh"

namespace are {
namespace {

using fixed::Acc;
constexpr unsigned kAll = 0xffffffffu;

// A 160-bit threshold of the aggregate terms: its value * 2^scale, or
// `inf` where that does not fit (a retention no total reaches, no limit).
struct Fix160 {
    unsigned long long lo = 0, hi = 0;
    uint32_t top = 0;
    int inf = 0;
};

struct OccArgs {
    double *marg;            // marginals, indexed by event - marg_base
    double *occ_max;         // per trial, or nullptr
    int64_t marg_base;
    int scale;
    Fix160 agg_r, agg_l;
};

__device__ __forceinline__ bool ge(const Acc &a, unsigned long long lo, unsigned long long hi, uint32_t top)
{
    if (a.top != top) return a.top > top;
    if (a.hi != hi) return a.hi > hi;
    return a.lo >= lo;
}

__device__ __forceinline__ Acc sub(const Acc &a, unsigned long long lo, unsigned long long hi, uint32_t top)
{
    Acc r;
    asm("sub.cc.u64 %0, %3, %6;\n\t"
        "subc.cc.u64 %1, %4, %7;\n\t"
        "subc.u32 %2, %5, %8;"
        : "=l"(r.lo), "=l"(r.hi), "=r"(r.top)
        : "l"(a.lo), "l"(a.hi), "r"(a.top), "l"(lo), "l"(hi), "r"(top));
    return r;
}

__device__ __forceinline__ Acc shfl(const Acc &a, int src)
{
    Acc r;
    r.lo = __shfl_sync(kAll, a.lo, src);
    r.hi = __shfl_sync(kAll, a.hi, src);
    r.top = __shfl_sync(kAll, a.top, src);
    return r;
}

__device__ __forceinline__ Acc shfl_up(const Acc &a, int d)
{
    Acc r;
    r.lo = __shfl_up_sync(kAll, a.lo, d);
    r.hi = __shfl_up_sync(kAll, a.hi, d);
    r.top = __shfl_up_sync(kAll, a.top, d);
    return r;
}

// Step 4's aggregate terms on an exact total: min(max(S - AggR, 0), AggL).
__device__ __forceinline__ Acc clamp_agg(const Acc &s, const Fix160 &r, const Fix160 &l)
{
    if (r.inf || !ge(s, r.lo, r.hi, r.top)) return Acc{};
    Acc a = sub(s, r.lo, r.hi, r.top);
    if (!l.inf && ge(a, l.lo, l.hi, l.top)) {
        a.lo = l.lo;
        a.hi = l.hi;
        a.top = l.top;
    }
    return a;
}

// a * 2^-s rounded once to the nearest double (ties to even), built on the
// integer pipes: the FP64 pipe, which GB300 issues at a small fraction of
// its integer rate, is left to the occurrence losses.  Results below the
// normal range (never at the scales of real losses) take fixed::to_double.
__device__ __forceinline__ double to_double_int(const Acc &a, int s)
{
    int L;   // bit length
    if (a.top) L = 160 - __clz((int)a.top);
    else if (a.hi) L = 128 - __clzll((long long)a.hi);
    else if (a.lo) L = 64 - __clzll((long long)a.lo);
    else return 0.0;
    const int e = L - 1 - s;   // the result's binary exponent
    if (e < -1022) return fixed::to_double(a, s);
    unsigned long long w, sticky = 0;   // the top 64 bits, top bit set
    if (L <= 64) {
        w = a.lo << (64 - L);
    } else {
        const int r = L - 64;  // 1 .. 96
        if (r < 64) {
            w = (a.lo >> r) | (a.hi << (64 - r));
            sticky = a.lo & ((1ull << r) - 1);
        } else if (r == 64) {
            w = a.hi;
            sticky = a.lo;
        } else {
            const int q = r - 64;
            w = (a.hi >> q) | ((unsigned long long)a.top << (64 - q));
            sticky = a.lo | (a.hi & ((1ull << q) - 1));
        }
    }
    unsigned long long m = w >> 11;                       // 53 bits
    const unsigned long long rest = w & 0x7ffull;         // the 11 bits below them
    const bool up = rest > 0x400ull || (rest == 0x400ull && (sticky != 0 || (m & 1ull)));
    int ex = e;
    if (up && ++m == (1ull << 53)) {
        m >>= 1;
        ++ex;
    }
    return __longlong_as_double((long long)(((unsigned long long)(ex + 1023) << 52) | (m & ((1ull << 52) - 1))));
}

__device__ __forceinline__ double as_double(float x) { return rows::widen(x); }
__device__ __forceinline__ double as_double(double x) { return x; }

template <typename Body, int U, bool FIXED>
__global__ void __launch_bounds__(256, 2)
    k_rows_occ(const rows::Trials a, const Body body, const OccArgs oa, const int64_t n_trials)
{
    constexpr int R = Body::R, RPW = Body::RPW;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t t0 = warp * n_trials / nw, t1 = (warp + 1) * n_trials / nw;
    if (t0 >= t1) return;
    // the lane holding the occurrence loss of event `lane` of a group
    const int holder = (lane % RPW) * R + lane / RPW;
    rows::Cursor<U, FIXED> cur(a, t0, t1, lane);
    Acc s, ap;              // the running total before the group, A of the event before it
    double omax = 0.0;      // this lane's largest occurrence loss of the trial
    while (cur.more()) {
        const int64_t first = cur.pos;   // the batch's first event
        int32_t id[U];
        int cnt;
        int64_t tc;
        bool last;
        cur.take(id, cnt, tc, last);
        if (cnt > 0) {
            typename Body::Occ o[U];
            body.occ(id, cnt == 32 * U, lane, o);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const double x = __shfl_sync(kAll, as_double(o[u]), holder);   // event u * 32 + lane
                const bool valid = u * 32 + lane < cnt;
                double *const out = oa.marg + (first + u * 32 + lane - oa.marg_base);
                const bool pos = valid && __double_as_longlong(x) != 0;
                if (!__any_sync(kAll, pos)) {   // no loss in the group: A stays, every marginal is 0
                    if (valid) __stcs(out, 0.0);
                    continue;
                }
                if (pos && __double_as_longlong(x) > __double_as_longlong(omax)) omax = x;
                // inclusive scan over the group's events in 128 bits (32
                // values below 2^123 each), then the total before it
                unsigned long long lo = 0, hi = 0;
                if (pos) fixed::to_fixed(x, oa.scale, lo, hi);
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const unsigned long long wl = __shfl_up_sync(kAll, lo, d);
                    const unsigned long long wh = __shfl_up_sync(kAll, hi, d);
                    if (lane >= d)
                        asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, %3;" : "+l"(lo), "+l"(hi) : "l"(wl), "l"(wh));
                }
                Acc v = s;
                v.add(lo, hi, 0u);
                const Acc ad = clamp_agg(v, oa.agg_r, oa.agg_l);
                Acc before = shfl_up(ad, 1);
                if (lane == 0) before = ap;
                if (valid) __stcs(out, to_double_int(sub(ad, before.lo, before.hi, before.top), oa.scale));
                s = shfl(v, 31);
                ap = shfl(ad, 31);
            }
        }
        if (last) {   // the trial's loss A_k and its largest occurrence loss
#pragma unroll
            for (int d = 16; d; d >>= 1) {
                const double w = __shfl_xor_sync(kAll, omax, d);
                if (__double_as_longlong(w) > __double_as_longlong(omax)) omax = w;
            }
            if (lane == 0) {
                if (a.ylt) a.ylt[tc] = to_double_int(ap, oa.scale);
                if (oa.occ_max) oa.occ_max[tc] = omax;
            }
            s = Acc{};
            ap = Acc{};
            omax = 0.0;
        }
    }
}

template <typename Body, int U>
void launch_t(const SimArgs &a, const Body &body, const OccArgs &oa, int num_sms, cudaStream_t s)
{
    rows::Trials t;
    t.ids = a.ids;
    t.off = a.off;
    t.k = a.k;
    t.trial_begin = a.trial_begin;
    t.ylt = a.ylt;
    t.agg_r = a.agg_r;
    t.agg_l = a.agg_l;
    auto kern = a.off ? k_rows_occ<Body, U, false> : k_rows_occ<Body, U, true>;
    const int per_sm = fit_blocks(reinterpret_cast<const void *>(kern), 256, 0);
    int64_t blocks = (a.n_trials + 7) / 8;
    const int64_t cap = (int64_t)num_sms * per_sm;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, 256, 0, s>>>(t, body, oa, a.n_trials);
    ARE_CUDA_TRY(cudaGetLastError());
}

// v * 2^s as a 160-bit integer (rounded to nearest), or inf where it does
// not fit in 160 bits.
Fix160 to_fix160(double v, int s)
{
    Fix160 f;
    if (!(v < INFINITY)) {
        f.inf = 1;
        return f;
    }
    if (v <= 0.0) return f;
    int ex = 0;
    const double m = std::frexp(v, &ex);                  // v = m * 2^ex, 0.5 <= m < 1
    unsigned long long mant = (unsigned long long)std::ldexp(m, 53);   // exact: 53 bits
    int sh = ex - 53 + s;                                 // v * 2^s = mant * 2^sh
    if (sh >= 160 - 53) {
        f.inf = 1;
        return f;
    }
    if (sh < 0) {
        if (sh < -63) return f;                          // below 2^-s * 2^-10: 0
        const unsigned long long half = 1ull << (-sh - 1);
        mant = (mant + half) >> (-sh);
        sh = 0;
    }
    // mant * 2^sh with sh < 107 into lo/hi/top
    unsigned __int128 w = (unsigned __int128)mant;
    if (sh < 64) {
        const unsigned __int128 x = w << sh;                 // below 2^117
        f.lo = (unsigned long long)x;
        f.hi = (unsigned long long)(x >> 64);
        f.top = 0;
    } else {
        const unsigned __int128 x = w << (sh - 64);          // the value / 2^64, below 2^96
        f.lo = 0;
        f.hi = (unsigned long long)x;
        f.top = (uint32_t)(x >> 64);
    }
    return f;
}

}  // namespace

// a: the analysis arguments (ids, offsets, trial range, ylt, aggregate
// terms; table/table2 the rows and overflow of the chosen form); form: 0
// packed FP64 rows of row_words words, 1 packed FP32 rows of row_words
// words, 2 dense FP32 rows of row_words (8 or 16) floats.
int launch_rows_occ(const SimArgs &a, int form, int row_words, const TermsF32 &t32, const TermsF64 &t64, int scale,
                    int num_sms, cudaStream_t s)
{
    if (a.n_trials <= 0) return 0;
    OccArgs oa;
    oa.marg = a.marg;
    oa.occ_max = a.occ_max;
    oa.marg_base = a.marg_base;
    oa.scale = scale - 3;   // a loss below 2^123: a group of 32 sums in 128 bits
    scale = oa.scale;
    oa.agg_r = to_fix160(a.agg_r, scale);
    oa.agg_l = to_fix160(a.agg_l, scale);
    if (form == 0) {
        if (row_words == 4 || row_words == 8) {
            auto go = [&](auto body) {
                body.rows = static_cast<const unsigned long long *>(a.table);
                body.ovf = static_cast<const double *>(a.table2);
                body.scale = scale;
                body.occ_r = t64.occ_r;
                body.occ_l = t64.occ_l;
                launch_t<decltype(body), 1>(a, body, oa, num_sms, s);
            };
            if (row_words == 4) go(rows::BodyP64<4, 1>{});
            else go(rows::BodyP64<8, 1>{});
            return 1;
        }
    } else if (form == 1) {
        if (row_words == 8 || row_words == 16) {
            auto go = [&](auto body) {
                body.rows = static_cast<const float *>(a.table);
                body.ovf = static_cast<const float *>(a.table2);
                body.occ_r = t32.occ_r;
                body.occ_l = t32.occ_l;
                launch_t<decltype(body), 1>(a, body, oa, num_sms, s);
            };
            if (row_words == 8) go(rows::BodyPackedF32<8, 1, ARE_FP32_KAHAN>{});
            else go(rows::BodyPackedF32<16, 1, ARE_FP32_KAHAN>{});
            return 1;
        }
    } else if (form == 2) {
        if (row_words == 8 || row_words == 16) {   // (a layer of more than 16 ELTs has packed rows)
            auto go = [&](auto body) {
                body.table = static_cast<const float *>(a.table);
                body.occ_r = t32.occ_r;
                body.occ_l = t32.occ_l;
                launch_t<decltype(body), 1>(a, body, oa, num_sms, s);
            };
            if (row_words == 8) go(rows::BodyF32<8, 1, ARE_FP32_KAHAN>{});
            else go(rows::BodyF32<16, 1, ARE_FP32_KAHAN>{});
            return 1;
        }
    }
    throw Error{ARE_EINVAL, "no per-occurrence kernel for rows of form " + std::to_string(form) + " and " +
                                std::to_string(row_words) + " words"};
}

}  // namespace are
