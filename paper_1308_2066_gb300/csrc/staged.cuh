// staged.cuh -- the analysis stage with one event per lane and the event's
// table row staged in shared memory (cp.async, coalesced: one L1 wavefront
// per row).  Instantiated by staged64.cu (FP64 tables).
//
// A table entry is the event's financial term in one ELT (formed in FP64 as
// the table is built).  FP64 tables: GB300 issues an FP64 add at about 1/66
// of the FP32 rate and a warp with one active lane costs as much as a full
// one, so each lane marks its event's non-zero columns (an integer test of
// the bit pattern) and adds them in column order: the first is taken as is,
// so an FP64 add is issued only when some event of the warp has two or more.
// Columns with a zero term add an exact 0, which changes nothing, so the
// event loss is the sum over ELTs of step 2 in layer order, as the paper's
// loop forms it.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "are_internal.cuh"

namespace are {
namespace staged {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarps = 8;

__device__ __forceinline__ uint64_t bits(double x) { return (uint64_t)__double_as_longlong(x); }
__device__ __forceinline__ double dbl(uint64_t b) { return __longlong_as_double((long long)b); }

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

// min(max(v, 0), l) on bit patterns, l >= 0 (+inf allowed)
__device__ __forceinline__ double clamp_bits(double v, uint64_t l_bits)
{
    const uint64_t b = bits(v);
    if ((int64_t)b < 0) return 0.0;
    return dbl(b < l_bits ? b : l_bits);
}

// Exact float -> double for finite x >= 0 on the integer pipes.
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

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, int src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
                 "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Physical slot of 16-byte chunk c of row r (CH chunks per row, CH even):
// a per-row rotation that gives the 8 lanes of a shared-memory phase 8
// distinct bank groups for any row length.
template <int CH>
__device__ __forceinline__ int chunk_slot(int c, int r)
{
    const int rot = CH % 8 == 0 ? (r & 7) : CH % 4 == 0 ? ((r >> 1) & 3) : ((r >> 2) & 1);
    const int p = c + rot;
    return p >= CH ? p - CH : p;
}

// Element j of row r in a staged batch.
template <typename T, int JP>
__device__ __forceinline__ T *elem(float4 *buf, int r, int j)
{
    constexpr int VPL = 16 / (int)sizeof(T);
    constexpr int CH = JP / VPL;
    return reinterpret_cast<T *>(buf + r * CH + chunk_slot<CH>(j / VPL, r)) + (j % VPL);
}

struct Batch {
    int64_t t = -1;
    int64_t pos = 0;
    int cnt = 0;
    bool last = false;
};
struct Cursor {
    int64_t t, pos, end;
};

template <bool FIXED>
__device__ __forceinline__ void trial_bounds(const SimArgs &a, int64_t t, int64_t &b, int64_t &e)
{
    const int64_t tt = a.trial_begin + t;
    if (FIXED) {
        b = tt * (int64_t)a.k;
        e = b + a.k;
    } else {
        b = a.off[tt];
        e = a.off[tt + 1];
    }
}

__device__ __forceinline__ double clamp_d(double v, double r, double l)
{
    double x = v - r;
    x = x > 0.0 ? x : 0.0;
    return x < l ? x : l;
}

// The warp's next batch (<= 32 events of one trial); trials without events
// get their outputs written here.
template <bool FIXED>
__device__ __forceinline__ Batch next_batch(const SimArgs &a, Cursor &c, int64_t step, int lane,
                                            double empty_loss)
{
    Batch b;
    while (c.t < a.n_trials) {
        if (c.pos < c.end) {
            b.t = c.t;
            b.pos = c.pos;
            const int64_t left = c.end - c.pos;
            b.cnt = left < 32 ? (int)left : 32;
            c.pos += 32;
            if (c.pos >= c.end) {
                b.last = true;
                c.t += step;
                if (c.t < a.n_trials) trial_bounds<FIXED>(a, c.t, c.pos, c.end);
            }
            return b;
        }
        if (lane == 0 && a.ylt) a.ylt[c.t] = empty_loss;
        c.t += step;
        if (c.t < a.n_trials) trial_bounds<FIXED>(a, c.t, c.pos, c.end);
    }
    return b;
}

template <typename T, int JP>
constexpr int smem_bytes()
{
    return kWarps * 2 * 32 * JP * (int)sizeof(T);   // per warp: two row buffers
}

template <typename T>
using TermsOf = typename std::conditional<sizeof(T) == 4, TermsF32, TermsF64>::type;

// Step 2 for the lane's event: the sum over the layer's ELTs of the terms.
template <int JP>
__device__ __forceinline__ float event_loss(float4 *buf, int lane)
{
    constexpr int CH = JP / 4;
    float g = 0.f;
#pragma unroll
    for (int c = 0; c < CH; ++c) {
        const float4 v = buf[lane * CH + chunk_slot<CH>(c, lane)];
        g = __fadd_rn(__fadd_rn(__fadd_rn(__fadd_rn(g, v.x), v.y), v.z), v.w);
    }
    return g;
}

// FP64: the non-zero columns in column order, an FP64 add only where some
// event of the warp has two or more (see the file comment).
template <int JP>
__device__ __forceinline__ double event_loss64(float4 *buf, int lane)
{
    constexpr int CH = JP / 2;
    uint32_t mask = 0;
#pragma unroll
    for (int c = 0; c < CH; ++c) {
        const double2 v = reinterpret_cast<const double2 *>(buf)[lane * CH + chunk_slot<CH>(c, lane)];
        if (bits(v.x) != 0) mask |= 1u << (2 * c);
        if (bits(v.y) != 0) mask |= 1u << (2 * c + 1);
    }
    double g = 0.0;
    uint32_t m = mask;
    if (m) {
        g = *elem<double, JP>(buf, lane, __ffs(m) - 1);
        m &= m - 1;
    }
    while (__any_sync(kFull, m != 0)) {
        if (m) {
            g = vadd(g, *elem<double, JP>(buf, lane, __ffs(m) - 1));
            m &= m - 1;
        }
    }
    return g;
}

__device__ __forceinline__ float occ_clamp(float g, const TermsF32 &tm)
{
    return fminf(fmaxf(__fsub_rn(g, tm.occ_r), 0.f), tm.occ_l);
}
__device__ __forceinline__ double occ_clamp(double g, const TermsF64 &tm)
{
    const bool need = bits(g) > bits(tm.occ_r);
    double o = 0.0;
    if (__any_sync(kFull, need)) {
        const double d = vsub(g, tm.occ_r);
        if (need) o = clamp_bits(d, bits(tm.occ_l));
    }
    return o;
}

// Trial running sums for the YLT-only outputs.
struct SumF64 {
    double s = 0.0;
    __device__ __forceinline__ void add(double o)
    {
        const bool need = bits(o) != 0;
        if (__any_sync(kFull, need)) {
            const double t = vadd(s, o);
            if (need) s = t;
        }
    }
};

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = __dadd_rn(v, __shfl_xor_sync(kFull, v, off));
    return v;
}
template <typename T, int JP, bool FIXED>
__global__ void __launch_bounds__(kWarps * 32) k_staged(const SimArgs a, const TermsOf<T> tm)
{
    constexpr int VPL = 16 / (int)sizeof(T);
    constexpr int CH = JP / VPL;
    extern __shared__ float4 stage[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float4 *buf0 = stage + (size_t)w * 2 * 32 * CH;
    float4 *buf1 = buf0 + 32 * CH;
    const T *tab = static_cast<const T *>(a.table);
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t step = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const double empty_loss = clamp_d(0.0, a.agg_r, a.agg_l);
    Cursor cur{warp, 0, 0};
    if (cur.t < a.n_trials) trial_bounds<FIXED>(a, cur.t, cur.pos, cur.end);

    auto load_ids = [&](const Batch &b) -> int32_t {
        return lane < b.cnt ? __ldcs(a.ids + b.pos + lane) : 0;
    };
    // (a full batch copies every row unconditionally; a partial one
    // zero-fills the rows past its events)
    auto issue_rows = [&](const Batch &b, int32_t idv, float4 *buf) {
        if (b.cnt == 32) {
#pragma unroll
            for (int i = 0; i < CH; ++i) {
                const int q = lane + 32 * i, r = q / CH, c = q % CH;
                const int32_t id = __shfl_sync(kFull, idv, r);
                cp_async16(smem_addr(buf + r * CH + chunk_slot<CH>(c, r)),
                           reinterpret_cast<const float4 *>(tab + (size_t)id * JP) + c, 16);
            }
        } else {
#pragma unroll
            for (int i = 0; i < CH; ++i) {
                const int q = lane + 32 * i, r = q / CH, c = q % CH;
                const int32_t id = __shfl_sync(kFull, idv, r);
                const bool ok = r < b.cnt;
                const float4 *src = ok ? reinterpret_cast<const float4 *>(tab + (size_t)id * JP) + c
                                       : reinterpret_cast<const float4 *>(tab);
                cp_async16(smem_addr(buf + r * CH + chunk_slot<CH>(c, r)), src, ok ? 16 : 0);
            }
        }
        cp_commit();
    };

    SumF64 sum;   // per-lane running sums of the trial

    auto compute = [&](const Batch &b, float4 *buf) {
        T g;
        if constexpr (sizeof(T) == 8) g = event_loss64<JP>(buf, lane);
        else g = event_loss<JP>(buf, lane);
        const T o = occ_clamp(g, tm);
        if constexpr (sizeof(T) == 8) sum.add(o);
        else sum.add(widen(o));
        if (b.last) {
            const double S = warp_sum(sum.s);
            if (lane == 0) a.ylt[b.t] = clamp_d(S, a.agg_r, a.agg_l);
            sum = SumF64{};
        }
    };

    Batch q0 = next_batch<FIXED>(a, cur, step, lane, empty_loss);
    int32_t i0 = load_ids(q0);
    Batch q1 = next_batch<FIXED>(a, cur, step, lane, empty_loss);
    int32_t i1 = load_ids(q1);
    Batch q2 = next_batch<FIXED>(a, cur, step, lane, empty_loss);
    int32_t i2 = load_ids(q2);
    Batch q3;
    int32_t i3 = 0;
    issue_rows(q0, i0, buf0);

#define ARE_STAGE(QC, QN, IN, QF, IF, BC, BN)                      \
    if (QC.cnt == 0) break;                                        \
    QF = next_batch<FIXED>(a, cur, step, lane, empty_loss);        \
    IF = load_ids(QF);                                             \
    issue_rows(QN, IN, BN);                                        \
    cp_wait1();                                                    \
    __syncwarp();                                                  \
    compute(QC, BC);                                               \
    __syncwarp();
    while (true) {
        ARE_STAGE(q0, q1, i1, q3, i3, buf0, buf1)
        ARE_STAGE(q1, q2, i2, q0, i0, buf1, buf0)
        ARE_STAGE(q2, q3, i3, q1, i1, buf0, buf1)
        ARE_STAGE(q3, q0, i0, q2, i2, buf1, buf0)
    }
#undef ARE_STAGE
    cp_wait0();
}

template <typename T, int JP, bool FIXED>
void launch_staged_t(const SimArgs &a, const TermsOf<T> &tm, int num_sms, cudaStream_t s)
{
    auto kern = k_staged<T, JP, FIXED>;
    constexpr int smem = smem_bytes<T, JP>();
    const int per_sm = fit_blocks(reinterpret_cast<const void *>(kern), kWarps * 32, smem);
    int64_t blocks = (a.n_trials + kWarps - 1) / kWarps;
    const int64_t cap = (int64_t)num_sms * per_sm;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, kWarps * 32, smem, s>>>(a, tm);
    ARE_CUDA_TRY(cudaGetLastError());
}

}  // namespace staged
}  // namespace are
