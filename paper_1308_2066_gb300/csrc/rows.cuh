// rows.cuh -- the analysis stage (Basic Algorithm, Section II-B) over an FP32
// layer table with every table row held in registers: the core of the
// single-layer FP32 kernel (simulate.cu) and of the persistent multi-layer
// kernel (sim_items.cu).
//
// The layer table holds, for each catalog event and each ELT of the layer,
// the event's financial term f_j(x) = share * min(max(fx * x - D, 0), Lim)
// (step 2 before its sum over ELTs), formed in FP64 when the table is built
// and rounded once to FP32; a row is jp = 8, 16 or 32 floats.
//
// Mapping (GB300).  A warp takes a contiguous range of trials and walks each
// trial's events in batches of 32 * U events (a batch never spans two
// trials).  Each group of 32 events is loaded with one coalesced read of
// their ids; the rows are then read by R = jp / 8 lanes each, one 32-byte
// (256-bit) load per lane, so a warp load instruction fetches 32 / R whole
// rows and every lane holds R * U row pieces in flight.  Each lane adds its
// pieces' 8 terms (packed FP32x2 adds); a reduce-scatter across the R lanes
// of a row (R - 1 shuffles) completes the sum over ELTs and leaves every lane
// with one whole event per group, whose occurrence terms (step 3) and
// running sum (step 4) it does alone.  Ids are read one batch ahead.
//
// A trial's total is the warp's merge of its lanes' running sums.  The
// totals of 32 consecutive trials are kept one per lane and finished
// together: the aggregate terms in FP64 for 32 trials per instruction, and
// one coalesced write of 32 trial losses.  (GB300 issues FP64 arithmetic at
// a small fraction of its FP32 rate; one instruction per trial would cost
// about as much as all the occurrence arithmetic of the trial.)
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "are_internal.cuh"

namespace are {
namespace rows {

constexpr unsigned kFull = 0xffffffffu;

struct F8 {
    float v[8];
};

// 32 bytes of a table row in one 256-bit load through the read-only path.
__device__ __forceinline__ F8 load8(const float *p)
{
    F8 r;
    asm volatile("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=f"(r.v[0]), "=f"(r.v[1]), "=f"(r.v[2]), "=f"(r.v[3]), "=f"(r.v[4]),
                   "=f"(r.v[5]), "=f"(r.v[6]), "=f"(r.v[7])
                 : "l"(p));
    return r;
}

__device__ __forceinline__ F8 zero8()
{
    F8 r;
#pragma unroll
    for (int i = 0; i < 8; ++i) r.v[i] = 0.f;
    return r;
}

// Two FP32 additions in one packed instruction (sm_100 and later).
__device__ __forceinline__ float2 add2(float2 a, float2 b)
{
    unsigned long long ra, rb, rd;
    asm("mov.b64 %0, {%1, %2};" : "=l"(ra) : "f"(a.x), "f"(a.y));
    asm("mov.b64 %0, {%1, %2};" : "=l"(rb) : "f"(b.x), "f"(b.y));
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
    float2 d;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(d.x), "=f"(d.y) : "l"(rd));
    return d;
}

// Sum of a row piece's 8 terms.
__device__ __forceinline__ float sum8(const F8 &x)
{
    const float2 a = add2(make_float2(x.v[0], x.v[1]), make_float2(x.v[2], x.v[3]));
    const float2 b = add2(make_float2(x.v[4], x.v[5]), make_float2(x.v[6], x.v[7]));
    const float2 c = add2(a, b);
    return __fadd_rn(c.x, c.y);
}

// Exact float -> double for finite x >= 0 on the integer pipes; subnormal
// inputs take the FP64 conversion in a warp-uniform branch.
__device__ __forceinline__ double widen(float x)
{
    const uint32_t u = __float_as_uint(x);
    double d = __longlong_as_double(
        u ? (long long)(((unsigned long long)u << 29) + (896ull << 52)) : 0ll);
    const bool sub = u != 0 && u < 0x00800000u;
    if (__any_sync(kFull, sub)) {
        double c;
        asm volatile("cvt.f64.f32 %0, %1;" : "=d"(c) : "f"(x));
        if (sub) d = c;
    }
    return d;
}

__device__ __forceinline__ double clamp_d(double v, double r, double l)
{
    double a = __dsub_rn(v, r);
    a = a > 0.0 ? a : 0.0;
    return a < l ? a : l;
}

// Running sum of a lane's occurrence losses in FP32 with Kahan's
// compensation; the value is s - c.  A trial's total merges the lanes' pairs
// with exact two-sum steps, so the compensation survives the merge.
struct SumKahan {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float o)
    {
        const float y = __fsub_rn(o, c);
        const float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
    __device__ __forceinline__ void warp_merge()
    {
#pragma unroll
        for (int m = 16; m > 0; m >>= 1) {
            const float s2 = __shfl_xor_sync(kFull, s, m);
            const float c2 = __shfl_xor_sync(kFull, c, m);
            const float t = __fadd_rn(s, s2);
            const float bp = __fsub_rn(t, s);
            const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(s2, bp));
            c = __fsub_rn(__fadd_rn(c, c2), err);   // s + s2 = t + err exactly
            s = t;
        }
    }
    __device__ __forceinline__ double value() const { return __dsub_rn((double)s, (double)c); }
};

// Running sum in FP64: an FP64 add is issued only when some lane of the warp
// adds a non-zero loss (adding an exact zero changes nothing).
struct SumF64 {
    double s = 0.0;
    __device__ __forceinline__ void add(float o)
    {
        const bool need = o != 0.f;
        if (__any_sync(kFull, need)) {
            double r;
            asm volatile("add.rn.f64 %0, %1, %2;" : "=d"(r) : "d"(s), "d"(widen(o)));
            if (need) s = r;
        }
    }
    __device__ __forceinline__ void warp_merge()
    {
#pragma unroll
        for (int m = 16; m > 0; m >>= 1) s = __dadd_rn(s, __shfl_xor_sync(kFull, s, m));
    }
    __device__ __forceinline__ double value() const { return s; }
};

template <int ACC>
using SumOf = typename std::conditional<ACC == ARE_FP32_KAHAN, SumKahan, SumF64>::type;

// What one range of trials reads and writes.
struct Trials {
    const int32_t *ids;      // YET event ids
    const int64_t *off;      // ragged offsets (indexed by YET trial) or nullptr
    int32_t k;               // fixed events per trial
    int64_t trial_begin;     // YET trial of index 0
    const float *table;      // [catalog][JP] terms
    double *ylt;             // trial losses, indexed like the trials
    float occ_r, occ_l;
    double agg_r, agg_l;
};

// Analyses trials [t0, t1) (indices relative to trial_begin) and writes
// their losses.  All 32 lanes of the warp call it with the same range.
template <int JP, int U, int ACC, bool FIXED>
__device__ __forceinline__ void run_trials(const Trials &a, int64_t t0, int64_t t1, int lane)
{
    constexpr int R = JP / 8;       // lanes per row
    constexpr int RPW = 32 / R;     // rows per warp load
    constexpr int B = 32 * U;       // events per batch
    static_assert(JP == 8 || JP == 16 || JP == 32, "table width");
    const int row = lane / R, col = lane % R;
    if (t0 >= t1) return;

    // Trial bounds.  Ragged YETs: lane i holds the offsets of trial w + i of
    // a window of 32 trials, read once per window.
    int64_t wt = t0 - 64, wb = 0, we = 0;
    auto bounds = [&](int64_t t, int64_t &b, int64_t &e) {
        if (FIXED) {
            b = (a.trial_begin + t) * (int64_t)a.k;
            e = b + a.k;
            return;
        }
        if (t - wt >= 32) {
            wt = t;
            const bool in = t + lane < t1;
            wb = in ? __ldg(a.off + a.trial_begin + t + lane) : 0;
            we = in ? __ldg(a.off + a.trial_begin + t + lane + 1) : 0;
        }
        const int i = (int)(t - wt);
        b = __shfl_sync(kFull, wb, i);
        e = __shfl_sync(kFull, we, i);
    };
    // ids of a batch: group u's event u * 32 + lane (-1 past the trial)
    auto load_ids = [&](int32_t(&d)[U], int64_t p, int64_t e) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t ev = p + u * 32 + lane;
            d[u] = ev < e ? __ldcs(a.ids + ev) : -1;
        }
    };

    SumOf<ACC> acc;
    SumOf<ACC> kept;    // lane i: the total of trial (first of its 32) + i
    int64_t t = t0, pos = 0, end = 0;
    bounds(t, pos, end);
    int32_t nid[U];
    load_ids(nid, pos, end);
    while (t < t1) {
        const int64_t tc = t;
        const int64_t left = end - pos;
        const int cnt = left < B ? (int)left : B;   // <= 0: a trial without events
        int32_t id[U];
#pragma unroll
        for (int u = 0; u < U; ++u) id[u] = nid[u];
        pos += B;
        const bool last = pos >= end;
        if (last) {
            ++t;
            if (t < t1) bounds(t, pos, end);
        }
        if (t < t1) load_ids(nid, pos, end);

        if (cnt > 0) {
            // step 1: every ELT's entry of each event, one row read per event
            F8 v[U][R];
            if (cnt == B) {
#pragma unroll
                for (int u = 0; u < U; ++u)
#pragma unroll
                    for (int q = 0; q < R; ++q) {
                        const int32_t e = __shfl_sync(kFull, id[u], q * RPW + row);
                        v[u][q] = load8(a.table + (size_t)(uint32_t)e * JP + col * 8);
                    }
            } else {
#pragma unroll
                for (int u = 0; u < U; ++u)
#pragma unroll
                    for (int q = 0; q < R; ++q) {
                        const int32_t e = __shfl_sync(kFull, id[u], q * RPW + row);
                        v[u][q] = e >= 0 ? load8(a.table + (size_t)(uint32_t)e * JP + col * 8) : zero8();
                    }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                // step 2: the sum over ELTs -- this lane's pieces, then a
                // reduce-scatter over the row's lanes (lane col keeps the
                // event of load q = col; the others of a partial batch hold 0)
                float p[R];
#pragma unroll
                for (int q = 0; q < R; ++q) p[q] = sum8(v[u][q]);
#pragma unroll
                for (int h = R / 2; h >= 1; h >>= 1) {
                    const bool hi = (col & h) != 0;
#pragma unroll
                    for (int m = 0; m < h; ++m) {
                        const float keep = hi ? p[m + h] : p[m];
                        const float send = hi ? p[m] : p[m + h];
                        p[m] = __fadd_rn(keep, __shfl_xor_sync(kFull, send, h));
                    }
                }
                // step 3 (occurrence terms), then the running sum of step 4
                acc.add(fminf(fmaxf(__fsub_rn(p[0], a.occ_r), 0.f), a.occ_l));
            }
        }
        if (last) {
            acc.warp_merge();
            const int slot = (int)((tc - t0) & 31);
            if (lane == slot) kept = acc;
            acc = SumOf<ACC>{};
            if (slot == 31 || t >= t1) {
                // step 4's aggregate terms for up to 32 trials at once: the
                // trial loss is A_k = min(max(S_k - AggR, 0), AggL)
                if (lane <= slot) a.ylt[tc - slot + lane] = clamp_d(kept.value(), a.agg_r, a.agg_l);
            }
        }
    }
}

}  // namespace rows
}  // namespace are
