// rows.cuh -- the analysis stage (Basic Algorithm, Section II-B) with every
// table row held in registers: the core of the single-layer register-rows
// kernels (simulate.cu for FP32 tables, rows64.cu for the FP64 path) and of
// the persistent multi-layer kernel (sim_items.cu).
//
// A layer table holds, for each catalog event and each ELT of the layer, the
// event's financial term f_j(x) = share * min(max(fx * x - D, 0), Lim) (step
// 2 before its sum over ELTs), formed in FP64 when the table is built; an
// FP32 table holds it rounded once to FP32 in rows of JP = 8, 16 or 32
// floats; a packed table holds each event's non-zero terms (FP32 or FP64)
// behind the mask of their columns, in rows of 32 or 64 bytes.
//
// Mapping (GB300).  A warp takes a contiguous range of trials and walks each
// trial's events in batches of 32 * U events (a batch never spans two
// trials).  Each group of 32 events is loaded with one coalesced read of
// their ids; the rows are then read by R = JP / 8 lanes each, one 32-byte
// (256-bit) load per lane, so a warp load instruction fetches 32 / R whole
// rows and every lane holds R * U row pieces in flight.  A reduce-scatter
// across the R lanes of a row (R - 1 shuffles) leaves every lane with one
// whole event per group, whose occurrence terms (step 3) and running sum
// (step 4) it does alone.  Ids are read one batch ahead.  (Packed rows are
// read the same way: 32-byte rows by one lane each, 64-byte rows by two.)
//
//   BodyF32  sums the FP32 terms (packed FP32x2 adds), clamps the event loss
//            with the occurrence terms and keeps a Kahan-compensated or an
//            FP64 running sum per lane.
//   BodyPackedF32  the same over packed FP32 rows (32- or 64-byte rows of
//            the non-zero terms behind their column mask).
//   BodyP64  reads the packed FP64 table (a row: the mask of the non-zero
//            terms, then those terms in column order), adds the terms in
//            column order (the first taken as is, an FP64 add only where an
//            event has two or more), so each event loss and occurrence loss
//            is the oracle's bit for bit; the running sum is exact: 160-bit
//            fixed-point integers, rounded to double once per trial
//            (fixed.cuh).
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
#include "fixed.cuh"

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

__device__ __forceinline__ uint64_t bits(double x) { return (uint64_t)__double_as_longlong(x); }
__device__ __forceinline__ double dbl(uint64_t b) { return __longlong_as_double((long long)b); }

// FP64 add/sub that the compiler may not hoist out of warp-uniform branches.
__device__ __forceinline__ double vadd(double a, double b)
{
    double r;
    asm volatile("add.rn.f64 %0, %1, %2;" : "=d"(r) : "d"(a), "d"(b));
    return r;
}
__device__ __forceinline__ double vsub(double a, double b)
{
    double r;
    asm volatile("sub.rn.f64 %0, %1, %2;" : "=d"(r) : "d"(a), "d"(b));
    return r;
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
};

// Running sum in FP64: an FP64 add is issued only when some lane of the warp
// adds a non-zero loss (adding an exact zero changes nothing).
struct SumF64 {
    double s = 0.0;
    __device__ __forceinline__ void add(float o)
    {
        const bool need = o != 0.f;
        if (__any_sync(kFull, need)) {
            const double r = vadd(s, widen(o));
            if (need) s = r;
        }
    }
    __device__ __forceinline__ void warp_merge()
    {
#pragma unroll
        for (int m = 16; m > 0; m >>= 1) s = __dadd_rn(s, __shfl_xor_sync(kFull, s, m));
    }
};

// The running sum of the FP64 path: exact, in fixed point.
struct SumFixed {
    fixed::Acc a;
    __device__ __forceinline__ void warp_merge() { fixed::warp_sum(a); }
};

// What one range of trials reads and writes, whatever the precision.
struct Trials {
    const int32_t *ids;      // YET event ids
    const int64_t *off;      // ragged offsets (indexed by YET trial) or nullptr
    int32_t k;               // fixed events per trial
    int64_t trial_begin;     // YET trial of index 0
    double *ylt;             // trial losses, indexed like the trials
    double agg_r, agg_l;
};

// Reads U groups of 32 events' row pieces: lane (row, col) takes piece col
// of the rows q * RPW + row of each group (R = JP / 8 lanes per row).
template <int JP, int U>
__device__ __forceinline__ void load_rows(const float *__restrict__ tab, const int32_t (&id)[U],
                                          bool full, int lane, F8 (&v)[U][JP / 8])
{
    constexpr int R = JP / 8, RPW = 32 / R;
    const int row = lane / R, col = lane % R;
    if (full) {
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int32_t e = __shfl_sync(kFull, id[u], q * RPW + row);
                v[u][q] = load8(tab + (size_t)(uint32_t)e * JP + col * 8);
            }
    } else {
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int32_t e = __shfl_sync(kFull, id[u], q * RPW + row);
                v[u][q] = e >= 0 ? load8(tab + (size_t)(uint32_t)e * JP + col * 8) : zero8();
            }
    }
}

// FP32 table: the event losses are sums of FP32 terms.
template <int JP, int U, int ACC>
struct BodyF32 {
    static_assert(JP == 8 || JP == 16 || JP == 32, "table width");
    using Sum = typename std::conditional<ACC == ARE_FP32_KAHAN, SumKahan, SumF64>::type;
    const float *table;      // [catalog][JP] terms
    float occ_r, occ_l;

    static constexpr int R = JP / 8, RPW = 32 / R;
    using Occ = float;

    __device__ __forceinline__ void batch(const int32_t (&id)[U], bool full, int lane, Sum &acc) const
    {
        float o[U];
        occ(id, full, lane, o);
#pragma unroll
        for (int u = 0; u < U; ++u) acc.add(o[u]);   // the running sum of step 4
    }
    // Steps 1-3 for a batch: lane (row, col) ends with the occurrence loss of
    // event col * RPW + row of each group (0 past the trial).
    __device__ __forceinline__ void occ(const int32_t (&id)[U], bool full, int lane, float (&o)[U]) const
    {
        const int col = lane % R;
        F8 v[U][R];
        load_rows<JP, U>(table, id, full, lane, v);   // step 1: every ELT's entry, one row read
#pragma unroll
        for (int u = 0; u < U; ++u) {
            // step 2: the sum over ELTs -- this lane's pieces, then a
            // reduce-scatter over the row's lanes (lane col keeps the event
            // of load q = col; the others of a partial batch hold 0)
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
            o[u] = fminf(fmaxf(__fsub_rn(p[0], occ_r), 0.f), occ_l);   // step 3 (occurrence terms)
        }
    }
    __device__ __forceinline__ double total(const Sum &t) const
    {
        if constexpr (ACC == ARE_FP32_KAHAN) return __dsub_rn((double)t.s, (double)t.c);
        else return t.s;
    }
};

// Packed FP32 table (repack.cu, launch_pack32_direct): row e is PW = 8 or
// 16 words (32 or 64 bytes) -- word 0 the mask of the ELT columns whose term
// is not 0, then up to PW - 1 of those terms in column order.  A row of more terms
// keeps the first PW - 2 inline and in word PW - 1 the offset of the rest
// (in column order) in the overflow array.  The rows are read and summed as
// BodyF32's, the mask word taken out of the sum; the events with an
// overflow (rare: where some lane has one) redo their sum from the row's
// inline terms and the overflow.
template <int PW, int U, int ACC>
struct BodyPackedF32 {
    using Sum = typename std::conditional<ACC == ARE_FP32_KAHAN, SumKahan, SumF64>::type;
    static constexpr int R = PW / 8, RPW = 32 / R, SLOTS = PW - 1;
    using Occ = float;
    const float *rows;       // [catalog][PW]
    const float *ovf;        // the terms past the inline ones of the longer rows
    float occ_r, occ_l;

    __device__ __forceinline__ void batch(const int32_t (&id)[U], bool full, int lane, Sum &acc) const
    {
        float o[U];
        occ(id, full, lane, o);
#pragma unroll
        for (int u = 0; u < U; ++u) acc.add(o[u]);   // the running sum of step 4
    }
    // Steps 1-3 for a batch: lane (row, col) ends with the occurrence loss of
    // event col * RPW + row of each group (0 past the trial).
    __device__ __forceinline__ void occ(const int32_t (&id)[U], bool full, int lane, float (&o)[U]) const
    {
        const int row = lane / R, col = lane % R;
        F8 v[U][R];
        load_rows<PW, U>(rows, id, full, lane, v);   // step 1: each event's whole row
        // the masks are in the pieces of the rows' first lanes
        bool over = false;
        if (col == 0) {
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    over |= __popc(__float_as_uint(v[u][q].v[0])) > SLOTS;
                    v[u][q].v[0] = 0.f;
                }
        }
        float g[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            // step 2: the sum over ELTs -- this lane's pieces, then (two
            // lanes per row) a reduce-scatter over the row's lanes
            if constexpr (R == 1) {
                g[u] = sum8(v[u][0]);
            } else {
                float p[R];
#pragma unroll
                for (int q = 0; q < R; ++q) p[q] = sum8(v[u][q]);
                const bool hi = (col & 1) != 0;
                const float keep = hi ? p[1] : p[0];
                const float send = hi ? p[0] : p[1];
                g[u] = __fadd_rn(keep, __shfl_xor_sync(kFull, send, 1));
            }
        }
        if (__any_sync(kFull, over)) {   // rare: a row with an overflow
            const uint32_t *w = reinterpret_cast<const uint32_t *>(rows);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int32_t ev = __shfl_sync(kFull, id[u], col * RPW + row);   // the lane's event
                const uint32_t *r = w + (size_t)(uint32_t)(ev >= 0 ? ev : 0) * PW;
                const int cnt = ev >= 0 ? __popc(__ldg(r)) : 0;
                if (cnt > SLOTS) {
                    float t = 0.f;
                    for (int i = 1; i < SLOTS; ++i) t = __fadd_rn(t, __uint_as_float(__ldg(r + i)));
                    const float *o = ovf + __ldg(r + SLOTS);
                    for (int i = 0; i < cnt - (SLOTS - 1); ++i) t = __fadd_rn(t, __ldg(o + i));
                    g[u] = t;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)   // step 3 (occurrence terms)
            o[u] = fminf(fmaxf(__fsub_rn(g[u], occ_r), 0.f), occ_l);
    }
    __device__ __forceinline__ double total(const Sum &t) const
    {
        if constexpr (ACC == ARE_FP32_KAHAN) return __dsub_rn((double)t.s, (double)t.c);
        else return t.s;
    }
};

// 32 bytes of a packed FP64 row as four 64-bit words.
struct W4 {
    unsigned long long w[4];
};
__device__ __forceinline__ W4 load4w(const unsigned long long *p)
{
    W4 r;
    asm volatile("ld.global.nc.v4.b64 {%0, %1, %2, %3}, [%4];"
                 : "=l"(r.w[0]), "=l"(r.w[1]), "=l"(r.w[2]), "=l"(r.w[3])
                 : "l"(p));
    return r;
}

// FP64 path over the packed FP64 table (repack.cu, launch_pack64_direct):
// row e is RW = 4 or 8 words (32 or 64 bytes) -- word 0 holds the mask of
// the ELT columns whose term is not 0 (low 32 bits) and an overflow offset
// (high 32 bits), words 1 .. RW - 1 the non-zero terms in column order.  A
// row with more non-zero terms than that keeps the first RW - 1 inline and
// all of them at the overflow offset.  The terms are added in column order
// (the first taken as is, an FP64 add only where some event has two or
// more), so every event loss and occurrence loss is the oracle's bit for
// bit; the running sum is exact (fixed point, fixed.cuh).
template <int RW, int U>
struct BodyP64 {
    using Sum = SumFixed;
    static constexpr int R = RW / 4, RPW = 32 / R, CAP = RW - 1;
    using Occ = double;
    const unsigned long long *rows;   // [catalog][RW]
    const double *ovf;                // overflow terms
    int32_t scale;                    // fixed-point scale s: every occurrence loss * 2^s < 2^126
    double occ_r, occ_l;

    __device__ __forceinline__ void batch(const int32_t (&id)[U], bool full, int lane, Sum &acc) const
    {
        double o[U];
        occ(id, full, lane, o);
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (bits(o[u]) != 0) {   // step 4's running sum, exact
                unsigned long long lo, hi;
                fixed::to_fixed(o[u], scale, lo, hi);
                acc.a.add(lo, hi, 0u);
            }
    }
    // Steps 1-3 for a batch: lane (row, col) ends with the occurrence loss of
    // event col * RPW + row of each group (0 past the trial), the oracle's
    // bit for bit.
    __device__ __forceinline__ void occ(const int32_t (&id)[U], bool full, int lane, double (&out)[U]) const
    {
        const int row = lane / R, col = lane % R;
        // step 1: each event's whole row -- lane (row, col) reads piece col
        // of the rows q * RPW + row
        W4 v[U][R];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int32_t e = __shfl_sync(kFull, id[u], q * RPW + row);
                if (full || e >= 0) {
                    v[u][q] = load4w(rows + (size_t)(uint32_t)e * RW + col * 4);
                } else {
#pragma unroll
                    for (int i = 0; i < 4; ++i) v[u][q].w[i] = 0ull;
                }
            }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            // the lane's event is load q = col: its header and first two
            // terms come from the row's lane col 0, one round per q
            unsigned long long h = v[u][0].w[0], x0 = v[u][0].w[1], x1 = v[u][0].w[2];
#pragma unroll
            for (int q = 1; q < R; ++q) {
                const unsigned long long a = __shfl_sync(kFull, v[u][q].w[0], row * R);
                const unsigned long long b = __shfl_sync(kFull, v[u][q].w[1], row * R);
                const unsigned long long c = __shfl_sync(kFull, v[u][q].w[2], row * R);
                if (col == q) {
                    h = a;
                    x0 = b;
                    x1 = c;
                }
            }
            const int32_t ev = __shfl_sync(kFull, id[u], col * RPW + row);
            const uint32_t mask = (uint32_t)h;
            const int cnt = __popc(mask);
            // step 2: the sum over ELTs in column order
            double g = dbl(x0);                    // 0 when the row has no term
            if (__any_sync(kFull, cnt >= 2)) {
                if (cnt >= 2) g = vadd(g, dbl(x1));
            }
            if (__any_sync(kFull, cnt >= 3)) {     // rare: the rest from the row or its overflow
                const unsigned long long *r = rows + (size_t)(uint32_t)ev * RW;
                const double *o = ovf + (uint32_t)(h >> 32);
                for (int i = 2; __any_sync(kFull, i < cnt); ++i) {
                    if (i < cnt) {
                        const double x = (cnt <= CAP || i < CAP) ? dbl(__ldg(r + 1 + i)) : __ldg(o + i);
                        g = vadd(g, x);
                    }
                }
            }
            // step 3 on bit patterns: min(max(g - OccR, 0), OccL), the
            // subtraction only where some lane has g > OccR
            const bool need = bits(g) > bits(occ_r);
            double o = 0.0;
            if (__any_sync(kFull, need)) {
                const double d = vsub(g, occ_r);
                if (need) o = dbl(bits(d) < bits(occ_l) ? bits(d) : bits(occ_l));
            }
            out[u] = o;
        }
    }
    __device__ __forceinline__ double total(const Sum &t) const { return fixed::to_double(t.a, scale); }
};

// The batches of a warp's trials [t0, t1): a cursor over the trials' events
// in batches of 32 * U (a batch never spans two trials), with the ids of the
// next batch read one batch ahead.  Ragged YETs: lane i holds the offsets of
// trial w + i of a window of 32 trials, read once per window.
template <int U, bool FIXED>
struct Cursor {
    static constexpr int B = 32 * U;
    const Trials &a;
    const int64_t t0, t1;
    const int lane;
    int64_t t, pos = 0, end = 0;
    int64_t wt, wb = 0, we = 0;
    int32_t nid[U];

    __device__ __forceinline__ Cursor(const Trials &a_, int64_t t0_, int64_t t1_, int lane_)
        : a(a_), t0(t0_), t1(t1_), lane(lane_), t(t0_), wt(t0_ - 64)
    {
        bounds();
        load_ids();
    }
    __device__ __forceinline__ void bounds()
    {
        if (FIXED) {
            pos = (a.trial_begin + t) * (int64_t)a.k;
            end = pos + a.k;
            return;
        }
        if (t - wt >= 32) {
            wt = t;
            const bool in = t + lane < t1;
            wb = in ? __ldg(a.off + a.trial_begin + t + lane) : 0;
            we = in ? __ldg(a.off + a.trial_begin + t + lane + 1) : 0;
        }
        const int i = (int)(t - wt);
        pos = __shfl_sync(kFull, wb, i);
        end = __shfl_sync(kFull, we, i);
    }
    // ids of the next batch: group u's event u * 32 + lane (-1 past the trial)
    __device__ __forceinline__ void load_ids()
    {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t ev = pos + u * 32 + lane;
            nid[u] = ev < end ? __ldcs(a.ids + ev) : -1;
        }
    }
    __device__ __forceinline__ bool more() const { return t < t1; }
    // Hands out the next batch: its ids, event count (<= 0: a trial without
    // events), trial and whether it ends the trial.
    __device__ __forceinline__ void take(int32_t (&id)[U], int &cnt, int64_t &tc, bool &last)
    {
        tc = t;
        const int64_t left = end - pos;
        cnt = left < B ? (int)left : B;
#pragma unroll
        for (int u = 0; u < U; ++u) id[u] = nid[u];
        pos += B;
        last = pos >= end;
        if (last) {
            ++t;
            if (t < t1) bounds();
        }
        if (t < t1) load_ids();
    }
};

// A trial's end: the warp merges its lanes' sums; the totals of 32
// consecutive trials are kept one per lane and finished together with
// step 4's aggregate terms, A_k = min(max(S_k - AggR, 0), AggL), and one
// coalesced write.
template <typename Body>
__device__ __forceinline__ void end_trial(const Trials &a, const Body &body, typename Body::Sum &acc,
                                          typename Body::Sum &kept, int64_t tc, int64_t t0, bool done,
                                          int lane)
{
    acc.warp_merge();
    const int slot = (int)((tc - t0) & 31);
    if (lane == slot) kept = acc;
    acc = typename Body::Sum{};
    if (slot == 31 || done)
        if (lane <= slot) a.ylt[tc - slot + lane] = clamp_d(body.total(kept), a.agg_r, a.agg_l);
}

// Analyses trials [t0, t1) (indices relative to trial_begin) and writes
// their losses, one batch at a time.  All 32 lanes of the warp call it with
// the same range.
template <int U, bool FIXED, typename Body>
__device__ __forceinline__ void run_trials(const Trials &a, const Body &body, int64_t t0, int64_t t1,
                                           int lane)
{
    if (t0 >= t1) return;
    typename Body::Sum acc, kept;
    Cursor<U, FIXED> cur(a, t0, t1, lane);
    while (cur.more()) {
        int32_t id[U];
        int cnt;
        int64_t tc;
        bool last;
        cur.take(id, cnt, tc, last);
        if (cnt > 0) body.batch(id, cnt == 32 * U, lane, acc);
        if (last) end_trial(a, body, acc, kept, tc, t0, !cur.more(), lane);
    }
}

}  // namespace rows
}  // namespace are
