// select.cu -- filters on the YLT (Section II-C): PML and TVaR.
//
// The paper names PML and TVaR (Section I) without defining them; the
// library reads PML at return period RP as the m-th largest trial loss,
// m = ceil(N / RP), and TVaR at level a as the mean of the m = ceil(N(1-a))
// largest.  Both need only the m-th largest value and the sum of the values
// above it, so no sort is done: an MSB-first radix select over an
// order-preserving 64-bit key of each double finds the m-th largest key
// exactly (8 passes of 8 bits, every target rank in the same pass), then one
// more pass adds the values above it.
//
// Two forms.  The single-YLT selection (launch_select: are_risk_measures,
// the pricing server) runs the passes below in one cooperative launch, with
// a grid-wide barrier between them (details above k_select_coop).  The
// multi-YLT selection (a portfolio's YLTs together) and the allocation-free
// one launch one kernel per pass.
//
// GB300 choices.  Each histogram pass ends with the pick of the next digit,
// done by whichever block of the pass finishes last (a counter and memory
// fences, no waiting), so a radix selection is 10 launches.  Histogram counts are
// aggregated per warp (lanes with the digit of the warp's first active lane
// add once), since early passes send most values to one or two bins.  The tail sum avoids FP64
// arithmetic, which GB300 issues at a small fraction of its integer rate:
// each value above the selected one is scaled by a power of two taken from
// the largest magnitude of the YLT and added as 32-bit limbs to integer
// accumulators, so the sum is exact, and it is rounded to double once.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "are_internal.cuh"

namespace are {
namespace {

namespace cg = cooperative_groups;
constexpr unsigned kFull = 0xffffffffu;
constexpr int kBins = 256;
constexpr int kThreads = 256;
constexpr int kLimbs = 3;                      // 32-bit limbs of one scaled value (< 2^96)
constexpr int kAccWords = 2 * kLimbs + 1;      // per target: positive limbs, negative limbs, count
constexpr int kCtrlWords = 4;                  // blocks arrived, top word of the largest |value|
constexpr int kPre = 8;                        // values a lane loads before it processes them

__device__ __forceinline__ uint64_t key_of(double x)
{
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double value_of(uint64_t k)
{
    const uint64_t b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
    return __longlong_as_double((long long)b);
}

struct Ranks {
    long long m[kMaxTargets];
};

// Scratch of one selection over n_ylt YLTs (blockIdx.y or blockIdx.x picks
// the YLT).
struct Sel {
    const double *single;        // the YLT when there is one
    const double *const *many;   // device array of YLT pointers, or nullptr
    uint32_t *hist;              // per YLT: kMaxTargets x 256 counts
    unsigned long long *state;   // per YLT: kMaxTargets x (key prefix, rank left)
    unsigned int *ctrl;          // per YLT: kCtrlWords
    unsigned long long *acc;     // per YLT: kMaxTargets x kAccWords
    double *result;              // per YLT: kMaxTargets x (m-th largest, mean of the m largest)
    int blocks;                  // blocks per YLT in the histogram and tail passes
};
__device__ __forceinline__ const double *ylt_of(const Sel &s, int y)
{
    return s.many ? s.many[y] : s.single;
}

// ---------------------------------------------------------------------------
// multi-word integers
// ---------------------------------------------------------------------------

struct U192 {
    unsigned long long w0 = 0, w1 = 0, w2 = 0;
};
__device__ __forceinline__ void add192(U192 &a, unsigned long long b0, unsigned long long b1,
                                       unsigned long long b2)
{
    asm("add.cc.u64 %0, %0, %3;\n\t"
        "addc.cc.u64 %1, %1, %4;\n\t"
        "addc.u64 %2, %2, %5;"
        : "+l"(a.w0), "+l"(a.w1), "+l"(a.w2)
        : "l"(b0), "l"(b1), "l"(b2));
}
__device__ __forceinline__ void sub192(U192 &a, const U192 &b)
{
    asm("sub.cc.u64 %0, %0, %3;\n\t"
        "subc.cc.u64 %1, %1, %4;\n\t"
        "subc.u64 %2, %2, %5;"
        : "+l"(a.w0), "+l"(a.w1), "+l"(a.w2)
        : "l"(b.w0), "l"(b.w1), "l"(b.w2));
}
__device__ __forceinline__ bool less192(const U192 &a, const U192 &b)
{
    if (a.w2 != b.w2) return a.w2 < b.w2;
    if (a.w1 != b.w1) return a.w1 < b.w1;
    return a.w0 < b.w0;
}

// |x| * 2^s as a 96-bit integer (lo 64 bits, hi 32 bits), rounding half up
// below the last bit; |x| < 2^(95 - s) keeps it below 2^96.
__device__ __forceinline__ void scaled(double x, int s, unsigned long long &lo, unsigned long long &hi)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
    const int be = (int)(b >> 52);
    unsigned long long m = b & ((1ull << 52) - 1);
    if (be) m |= 1ull << 52;
    const int sh = (be ? be : 1) - 1075 + s;   // |x| = m * 2^(sh - s)
    lo = 0;
    hi = 0;
    if (sh >= 64) {
        hi = m << (sh - 64);
    } else if (sh > 0) {
        lo = m << sh;
        hi = m >> (64 - sh);
    } else if (sh == 0) {
        lo = m;
    } else if (sh >= -53) {
        const int k = -sh;
        lo = (m >> k) + ((m >> (k - 1)) & 1ull);
    }
}

// a * 2^-s rounded once to the nearest double.
__device__ __forceinline__ double to_double(const U192 &a, int s)
{
    int L;
    if (a.w2) L = 192 - __clzll((long long)a.w2);
    else if (a.w1) L = 128 - __clzll((long long)a.w1);
    else if (a.w0) L = 64 - __clzll((long long)a.w0);
    else return 0.0;
    if (L <= 64) return ldexp(__ull2double_rn(a.w0), -s);
    const int r = L - 64;                      // 1 .. 128
    unsigned long long w, sticky;
    if (r < 64) {
        w = (a.w0 >> r) | (a.w1 << (64 - r));
        sticky = a.w0 & ((1ull << r) - 1);
    } else if (r == 64) {
        w = a.w1;
        sticky = a.w0;
    } else if (r < 128) {
        const int q = r - 64;
        w = (a.w1 >> q) | (a.w2 << (64 - q));
        sticky = a.w0 | (a.w1 & ((1ull << q) - 1));
    } else {
        w = a.w2;
        sticky = a.w0 | a.w1;
    }
    // w has its top bit set and a double keeps 53 of its 64 bits: a sticky
    // bit in bit 0 makes the conversion's one rounding the right one
    return ldexp(__ull2double_rn(w | (sticky ? 1ull : 0ull)), r - s);
}

// Scale of a YLT: s = 95 - floor(log2(largest |value|)), from the top 32
// bits of the largest magnitude's bit pattern.
__device__ __forceinline__ int tail_scale(unsigned int mag_hi)
{
    int e = (int)((mag_hi >> 20) & 0x7ff) - 1023;
    if (e < -1022) e = -1022;
    return 95 - e;
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------

// state[2t] = key prefix decided so far, state[2t+1] = rank still to find
// among the keys that share the prefix (1 = the largest of them).
__global__ void k_init(Sel s, Ranks r, int nt)
{
    const int y = blockIdx.x;
    uint32_t *hist = s.hist + (size_t)y * kMaxTargets * kBins;
    unsigned long long *state = s.state + (size_t)y * 2 * kMaxTargets;
    unsigned long long *acc = s.acc + (size_t)y * kMaxTargets * kAccWords;
    for (int i = threadIdx.x; i < nt * kBins; i += blockDim.x) hist[i] = 0;
    for (int i = threadIdx.x; i < nt * kAccWords; i += blockDim.x) acc[i] = 0;
    if (threadIdx.x < kCtrlWords) s.ctrl[(size_t)y * kCtrlWords + threadIdx.x] = 0;
    if (threadIdx.x < nt) {
        state[2 * threadIdx.x] = 0ull;
        state[2 * threadIdx.x + 1] = (unsigned long long)r.m[threadIdx.x];
    }
}

// Adds the lanes with `on` set to bin `bin` of h: the lanes whose bin is the
// first active lane's add once together (the common case: early passes send
// most values to one bin), the others one by one.  Every lane of the warp
// must call it.
__device__ __forceinline__ void hist_add(uint32_t *h, bool on, uint32_t bin, int lane)
{
    const unsigned act = __ballot_sync(kFull, on);
    if (!act) return;
    const int leader = __ffs(act) - 1;
    const uint32_t b0 = __shfl_sync(kFull, bin, leader);
    const unsigned same = __ballot_sync(kFull, on && bin == b0);
    if (lane == leader) atomicAdd(h + b0, (uint32_t)__popc(same));
    else if (on && bin != b0) atomicAdd(h + bin, 1u);
}

// One warp: find the bucket of h (256 counts) that holds the wanted rank,
// counting down from the top bucket, and extend the target's prefix.
__device__ __forceinline__ void pick(const uint32_t *h, unsigned long long *st, int shift, int lane)
{
    uint32_t c[8];
    unsigned long long lane_sum = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        c[i] = __ldcg(h + kBins - 1 - (lane * 8 + i));   // lane 0 holds the top buckets
        lane_sum += c[i];
    }
    unsigned long long incl = lane_sum;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const unsigned long long o = __shfl_up_sync(kFull, incl, off);
        if (lane >= off) incl += o;
    }
    const unsigned long long excl = incl - lane_sum;
    const unsigned long long r = st[1];
    if (excl < r && r <= incl) {
        unsigned long long above = excl;
        int b = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (above + c[i] >= r) {
                b = kBins - 1 - (lane * 8 + i);
                break;
            }
            above += c[i];
        }
        st[0] |= (unsigned long long)b << shift;
        st[1] = r - above;
    }
}

// Histogram pass `pass` (digit bits 56 - 8 pass .. 63 - 8 pass) over the keys
// that share each target's prefix; pass 0 counts every key once for all
// targets and records the largest magnitude.  The last block to finish picks
// every target's digit and clears the histogram for the next pass.
__global__ void __launch_bounds__(kThreads) k_hist(Sel s, int64_t n, int nt, int pass)
{
    const int y = blockIdx.y;
    const double *__restrict__ v = ylt_of(s, y);
    unsigned long long *state = s.state + (size_t)y * 2 * kMaxTargets;
    uint32_t *hist = s.hist + (size_t)y * kMaxTargets * kBins;
    unsigned int *ctrl = s.ctrl + (size_t)y * kCtrlWords;
    __shared__ uint32_t h[kMaxTargets * kBins];
    __shared__ unsigned int s_mag;
    __shared__ int s_last;
    const int rows = pass == 0 ? 1 : nt;
    for (int i = threadIdx.x; i < rows * kBins; i += blockDim.x) h[i] = 0;
    if (threadIdx.x == 0) s_mag = 0;
    const int shift = 56 - 8 * pass;
    uint64_t pre[kMaxTargets];
#pragma unroll
    for (int t = 0; t < kMaxTargets; ++t)   // pass 0 has no prefix yet
        pre[t] = (pass > 0 && t < nt) ? state[2 * t] >> (shift + 8) : 0ull;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    unsigned int mag = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // warp-uniform loop: every lane takes part in the warp's histogram adds;
    // kPre values per lane are loaded before the first is counted
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n;
         base += stride * kPre) {
        double xs[kPre];
#pragma unroll
        for (int u = 0; u < kPre; ++u) {
            const int64_t i = base + u * stride + lane;
            xs[u] = i < n ? v[i] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < kPre; ++u) {
            const bool ok = base + u * stride + lane < n;
            const double x = xs[u];
            const uint64_t k = key_of(x);
            const uint32_t d = (uint32_t)(k >> shift) & 0xffu;
            if (pass == 0) {
                hist_add(h, ok, d, lane);
                const unsigned int m32 =
                    (unsigned int)(((unsigned long long)__double_as_longlong(x) >> 32) & 0x7fffffffu);
                mag = m32 > mag ? m32 : mag;
            } else {
#pragma unroll
                for (int t = 0; t < kMaxTargets; ++t) {
                    if (t >= nt) break;
                    hist_add(h + t * kBins, ok && (k >> (shift + 8)) == pre[t], d, lane);
                }
            }
        }
    }
    if (pass == 0) {
#pragma unroll
        for (int off = 16; off; off >>= 1) {
            const unsigned int o = __shfl_xor_sync(kFull, mag, off);
            mag = o > mag ? o : mag;
        }
        if (lane == 0) atomicMax(&s_mag, mag);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < rows * kBins; i += blockDim.x)
        if (h[i]) atomicAdd(&hist[i], h[i]);
    if (pass == 0 && threadIdx.x == 0 && s_mag) atomicMax(&ctrl[1], s_mag);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&ctrl[0], 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const int t = threadIdx.x >> 5;
    if (t < nt) pick(hist + (pass == 0 ? 0 : t) * kBins, state + 2 * t, shift, lane);
    __syncthreads();
    for (int i = threadIdx.x; i < rows * kBins; i += blockDim.x) hist[i] = 0;
    if (threadIdx.x == 0) ctrl[0] = 0;
}

// Tail pass: every value whose key is above a target's selected key is
// added, scaled, to the target's integer accumulators (positive and
// negative values apart) and counted.  The last block to finish forms each
// target's sum of the m largest -- the values above plus (m - count) times
// the selected value -- and writes (value, sum / m).
__global__ void __launch_bounds__(kThreads) k_tail(Sel s, int64_t n, int nt, Ranks r)
{
    const int y = blockIdx.y;
    const double *__restrict__ v = ylt_of(s, y);
    const unsigned long long *state = s.state + (size_t)y * 2 * kMaxTargets;
    unsigned int *ctrl = s.ctrl + (size_t)y * kCtrlWords;
    unsigned long long *acc = s.acc + (size_t)y * kMaxTargets * kAccWords;
    __shared__ unsigned long long a[kMaxTargets * kAccWords];
    __shared__ int s_last;
    for (int i = threadIdx.x; i < nt * kAccWords; i += blockDim.x) a[i] = 0;
    uint64_t kt[kMaxTargets];
    uint64_t kmin = ~0ull;
#pragma unroll
    for (int t = 0; t < kMaxTargets; ++t) {
        kt[t] = t < nt ? state[2 * t] : ~0ull;
        kmin = kt[t] < kmin ? kt[t] : kmin;
    }
    const int sc = tail_scale(ctrl[1]);
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += stride * kPre) {
        double xs[kPre];   // kPre values loaded before the first is added
#pragma unroll
        for (int u = 0; u < kPre; ++u) xs[u] = i0 + u * stride < n ? v[i0 + u * stride] : 0.0;
#pragma unroll
        for (int u = 0; u < kPre; ++u) {
            if (i0 + u * stride >= n) break;
            const double x = xs[u];
            const uint64_t k = key_of(x);
            if (k > kmin) {
                unsigned long long lo, hi;
                scaled(x, sc, lo, hi);
                const int sign = x < 0.0 ? kLimbs : 0;
                const unsigned long long l0 = lo & 0xffffffffull, l1 = lo >> 32, l2 = hi;
#pragma unroll
                for (int t = 0; t < kMaxTargets; ++t) {
                    if (t < nt && k > kt[t]) {
                        unsigned long long *p = a + t * kAccWords;
                        atomicAdd(p + sign, l0);
                        atomicAdd(p + sign + 1, l1);
                        atomicAdd(p + sign + 2, l2);
                        atomicAdd(p + 2 * kLimbs, 1ull);
                    }
                }
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nt * kAccWords; i += blockDim.x)
        if (a[i]) atomicAdd(&acc[i], a[i]);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&ctrl[0], 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (threadIdx.x < nt) {
        const int t = threadIdx.x;
        const unsigned long long *p = acc + t * kAccWords;
        U192 pos, neg;
        // limb sums -> 192-bit integers: sum_l A_l * 2^(32 l)
        for (int g = 0; g < 2; ++g) {
            U192 &z = g ? neg : pos;
            const unsigned long long A0 = __ldcg(p + g * kLimbs), A1 = __ldcg(p + g * kLimbs + 1),
                                     A2 = __ldcg(p + g * kLimbs + 2);
            add192(z, A0, 0, 0);
            add192(z, A1 << 32, A1 >> 32, 0);
            add192(z, 0, A2, 0);
        }
        const unsigned long long c = __ldcg(p + 2 * kLimbs);
        const double vt = value_of(kt[t]);
        const unsigned long long q = (unsigned long long)r.m[t] - c;   // >= 1: ties at the m-th value
        unsigned long long lo, hi;
        scaled(vt, sc, lo, hi);
        U192 &z = vt < 0.0 ? neg : pos;
        // (hi:lo) * q with hi < 2^32 and q < 2^32
        add192(z, lo * q, __umul64hi(lo, q), 0);
        add192(z, 0, hi * q, __umul64hi(hi, q));
        double sum;
        if (less192(pos, neg)) {
            sub192(neg, pos);
            sum = -to_double(neg, sc);
        } else {
            sub192(pos, neg);
            sum = to_double(pos, sc);
        }
        double *res = s.result + (size_t)y * 2 * kMaxTargets;
        res[2 * t] = vt;
        res[2 * t + 1] = __ddiv_rn(sum, (double)r.m[t]);
    }
    if (threadIdx.x == 0) ctrl[0] = 0;
}

// ---------------------------------------------------------------------------
// Single-YLT selection in one cooperative launch
// ---------------------------------------------------------------------------
//
// One kernel whose blocks are all resident (a cooperative launch), with a
// grid-wide barrier where the radix form has a launch boundary:
// 1. two radix passes find each target's bucket of the top 16 key bits
//    (sign, exponent and four mantissa bits: 1/16 of an octave) and its rank
//    in it;
// 2. one pass keeps the keys of each target's bucket (up to kCand) and adds
//    the values of higher buckets to the target's exact tail sum;
// 3. block t selects among target t's kept keys by their last 48 bits in
//    shared memory and adds the bucket's values above the selected one; if
//    a bucket holds more than kCand keys (a long run of ties), every block
//    runs the remaining six radix passes over the whole YLT instead.
// In a radix pass every block picks every target's next digit itself from
// the pass's global histogram (the same counts give the same digit), so one
// barrier per pass is enough.  The histograms rotate through three buffers:
// the buffer of pass p is cleared by block 0 during pass p + 2, after every
// block has read it (before the barrier of pass p + 1) and before it is
// written again (pass p + 3).

constexpr int kCand = 16384;            // candidate keys kept per target
constexpr int kCoopThreads = 512;

struct SelC {
    const double *v;
    uint32_t *hist;              // 3 x kMaxTargets x kBins counts, zero between calls
    unsigned long long *acc;     // kMaxTargets x kAccWords
    unsigned int *ctrl;          // [1] top word of the largest |value|, zero between calls
    unsigned long long *app;     // per target: keys kept
    unsigned long long *cand;    // per target: kCand keys of its bucket
    double *result;              // per target: value, mean of the m largest
};

// Adds x (scaled by 2^sc) to the accumulator words a (positive and negative
// limbs apart, then a count) in shared memory for the lanes with `on` set,
// summed over the warp first (one set of atomics per warp and sign).  Every
// lane must call it.
__device__ __forceinline__ void acc_add_warp(unsigned long long *a, bool on, double x, int sc, int lane)
{
    if (!__any_sync(kFull, on)) return;
    unsigned long long lo = 0, hi = 0;
    if (on) scaled(x, sc, lo, hi);
    for (int g = 0; g < 2; ++g) {   // positive, then negative values
        const bool mine = on && ((x < 0.0) == (g == 1));
        if (!__any_sync(kFull, mine)) continue;
        unsigned long long w0 = mine ? (lo & 0xffffffffull) : 0, w1 = mine ? lo >> 32 : 0, w2 = mine ? hi : 0;
        unsigned long long c = mine ? 1ull : 0ull;
#pragma unroll
        for (int off = 16; off; off >>= 1) {
            w0 += __shfl_xor_sync(kFull, w0, off);
            w1 += __shfl_xor_sync(kFull, w1, off);
            w2 += __shfl_xor_sync(kFull, w2, off);
            c += __shfl_xor_sync(kFull, c, off);
        }
        if (lane == 0) {
            atomicAdd(a + g * kLimbs, w0);
            atomicAdd(a + g * kLimbs + 1, w1);
            atomicAdd(a + g * kLimbs + 2, w2);
            atomicAdd(a + 2 * kLimbs, c);
        }
    }
}

// (value of key kt, mean of the m largest) from the accumulator words A of
// the values above kt (sum and count, scaled by 2^sc).
__device__ void tail_result(const unsigned long long (&A)[kAccWords], uint64_t kt, long long m, int sc,
                            double *res)
{
    U192 pos, neg;
    for (int g = 0; g < 2; ++g) {
        U192 &z = g ? neg : pos;
        const unsigned long long A0 = A[g * kLimbs], A1 = A[g * kLimbs + 1], A2 = A[g * kLimbs + 2];
        add192(z, A0, 0, 0);
        add192(z, A1 << 32, A1 >> 32, 0);
        add192(z, 0, A2, 0);
    }
    const unsigned long long c = A[2 * kLimbs];
    const double vt = value_of(kt);
    const unsigned long long q = (unsigned long long)m - c;   // >= 1: ties at the m-th value
    unsigned long long lo, hi;
    scaled(vt, sc, lo, hi);
    U192 &z = vt < 0.0 ? neg : pos;
    add192(z, lo * q, __umul64hi(lo, q), 0);
    add192(z, 0, hi * q, __umul64hi(hi, q));
    double sum;
    if (less192(pos, neg)) {
        sub192(neg, pos);
        sum = -to_double(neg, sc);
    } else {
        sub192(pos, neg);
        sum = to_double(pos, sc);
    }
    res[0] = vt;
    res[1] = __ddiv_rn(sum, (double)m);
}

// One warp: the bucket of h (256 counts in shared memory) that holds rank
// rem, counting down from the top bucket; extends the prefix pre.
__device__ __forceinline__ void pick_shared(const uint32_t *h, unsigned long long &pre, unsigned long long &rem,
                                            int shift, int lane)
{
    uint32_t c[8];
    unsigned long long lane_sum = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        c[i] = h[kBins - 1 - (lane * 8 + i)];   // lane 0 holds the top buckets
        lane_sum += c[i];
    }
    unsigned long long incl = lane_sum;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const unsigned long long o = __shfl_up_sync(kFull, incl, off);
        if (lane >= off) incl += o;
    }
    const unsigned long long excl = incl - lane_sum;
    const unsigned long long r = rem;
    __syncwarp();
    if (excl < r && r <= incl) {
        unsigned long long above = excl;
        int b = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (above + c[i] >= r) {
                b = kBins - 1 - (lane * 8 + i);
                break;
            }
            above += c[i];
        }
        pre |= (unsigned long long)b << shift;
        rem = r - above;
    }
}

// One radix pass of the cooperative selection (digit bits shift .. shift + 7)
// over the keys that share each target's prefix st[2t] (pass 0: every key,
// one histogram for all targets), ending with the grid barrier and every
// block's pick of every target's digit.  pass 0 also gathers the largest
// magnitude into ctrl[1].
__device__ void coop_pass(const SelC &s, int64_t n, int nt, int pass, unsigned long long *st, uint32_t *h,
                          unsigned int *s_mag, cg::grid_group &grid)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int shift = 56 - 8 * pass;
    const int rows = pass == 0 ? 1 : nt;
    uint32_t *gh = s.hist + (size_t)(pass % 3) * kMaxTargets * kBins;
    for (int i = threadIdx.x; i < rows * kBins; i += blockDim.x) h[i] = 0;
    if (blockIdx.x == 0 && pass >= 2) {   // the buffer of pass - 2, read by every block already
        uint32_t *old = s.hist + (size_t)((pass - 2) % 3) * kMaxTargets * kBins;
        for (int i = threadIdx.x; i < kMaxTargets * kBins; i += blockDim.x) old[i] = 0;
    }
    if (pass == 0 && threadIdx.x == 0) *s_mag = 0;
    __syncthreads();
    uint64_t pre[kMaxTargets];
#pragma unroll
    for (int t = 0; t < kMaxTargets; ++t) pre[t] = t < nt ? st[2 * t] >> (shift + 8) : 0ull;
    unsigned int mag = 0;
    // warp-uniform loop: every lane takes part in the warp's histogram adds
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n;
         base += stride * kPre) {
        double xs[kPre];
#pragma unroll
        for (int u = 0; u < kPre; ++u) {
            const int64_t i = base + u * stride + lane;
            xs[u] = i < n ? s.v[i] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < kPre; ++u) {
            const bool ok = base + u * stride + lane < n;
            const uint64_t k = key_of(xs[u]);
            const uint32_t d = (uint32_t)(k >> shift) & 0xffu;
            if (pass == 0) {
                hist_add(h, ok, d, lane);
                const unsigned int m32 =
                    (unsigned int)(((unsigned long long)__double_as_longlong(xs[u]) >> 32) & 0x7fffffffu);
                if (ok) mag = m32 > mag ? m32 : mag;
            } else {
#pragma unroll
                for (int t = 0; t < kMaxTargets; ++t) {
                    if (t >= nt) break;
                    hist_add(h + t * kBins, ok && (k >> (shift + 8)) == pre[t], d, lane);
                }
            }
        }
    }
    if (pass == 0) {
#pragma unroll
        for (int off = 16; off; off >>= 1) {
            const unsigned int o = __shfl_xor_sync(kFull, mag, off);
            mag = o > mag ? o : mag;
        }
        if (lane == 0 && mag) atomicMax(s_mag, mag);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < rows * kBins; i += blockDim.x)
        if (h[i]) atomicAdd(&gh[i], h[i]);
    if (pass == 0 && threadIdx.x == 0 && *s_mag) atomicMax(&s.ctrl[1], *s_mag);
    grid.sync();
    // every block picks every target's digit from the pass's histogram
    if (warp < nt) pick(gh + (pass == 0 ? 0 : warp) * kBins, st + 2 * warp, shift, lane);
    __syncthreads();
}

// Block t's exact selection among the n_keys candidate keys of target t's
// bucket (in shared memory): the remaining 48 bits, 8 at a time; returns the
// key and adds the bucket's values above it to a.
__device__ uint64_t finish_in_block(const unsigned long long *keys, int n_keys, unsigned long long *st_t,
                                    uint32_t *h, unsigned long long *a, int sc)
{
    const int lane = threadIdx.x & 31;
    for (int shift = 40; shift >= 0; shift -= 8) {
        for (int i = threadIdx.x; i < kBins; i += blockDim.x) h[i] = 0;
        __syncthreads();
        const uint64_t pre = st_t[0] >> (shift + 8);
        // warp-uniform: the keys share most leading bits, so the warp adds per bin
        for (int base = threadIdx.x & ~31; base < n_keys; base += blockDim.x) {
            const int i = base + lane;
            const bool ok = i < n_keys;
            const uint64_t k = ok ? keys[i] : 0ull;
            hist_add(h, ok && (k >> (shift + 8)) == pre, (uint32_t)(k >> shift) & 0xffu, lane);
        }
        __syncthreads();
        if (threadIdx.x < 32) pick_shared(h, st_t[0], st_t[1], shift, lane);
        __syncthreads();
    }
    const uint64_t kt = st_t[0];
    for (int base = threadIdx.x & ~31; base < n_keys; base += blockDim.x) {
        const int i = base + lane;
        const bool ok = i < n_keys;
        const uint64_t k = ok ? keys[i] : 0ull;
        acc_add_warp(a, ok && k > kt, value_of(k), sc, lane);
    }
    __syncthreads();
    return kt;
}

__global__ void __launch_bounds__(kCoopThreads) k_select_coop(SelC s, int64_t n, int nt, Ranks r)
{
    cg::grid_group grid = cg::this_grid();
    extern __shared__ unsigned long long keys[];   // kCand: the candidates of a block's target
    __shared__ uint32_t h[kMaxTargets * kBins];
    __shared__ unsigned long long st[2 * kMaxTargets];   // per target: key prefix, rank left (the same in every block)
    __shared__ unsigned long long a[kMaxTargets * kAccWords];
    __shared__ unsigned int s_mag;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < nt) {
        st[2 * threadIdx.x] = 0ull;
        st[2 * threadIdx.x + 1] = (unsigned long long)r.m[threadIdx.x];
    }
    if (blockIdx.x == 0) {   // the counters and sums of step 2, used after the next two barriers
        for (int i = threadIdx.x; i < kMaxTargets * kAccWords; i += blockDim.x) s.acc[i] = 0;
        for (int i = threadIdx.x; i < kMaxTargets; i += blockDim.x) s.app[i] = 0;
    }
    __syncthreads();
    // 1. two radix passes: each target's bucket of the top 16 key bits and its rank in it
    coop_pass(s, n, nt, 0, st, h, &s_mag, grid);
    coop_pass(s, n, nt, 1, st, h, &s_mag, grid);
    const int sc = tail_scale(__ldcg(&s.ctrl[1]));
    uint32_t P[kMaxTargets];
#pragma unroll
    for (int t = 0; t < kMaxTargets; ++t) P[t] = t < nt ? (uint32_t)(st[2 * t] >> 48) : 0xffffffffu;
    // 2. the keys of each target's bucket kept (up to kCand); the values of
    //    higher buckets added to the target's exact tail sum
    for (int i = threadIdx.x; i < nt * kAccWords; i += blockDim.x) a[i] = 0;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n;
         base += stride * kPre) {
        double xs[kPre];
#pragma unroll
        for (int u = 0; u < kPre; ++u) {
            const int64_t i = base + u * stride + lane;
            xs[u] = i < n ? s.v[i] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < kPre; ++u) {
            const bool ok = base + u * stride + lane < n;
            const uint64_t k = key_of(xs[u]);
            const uint32_t p = (uint32_t)(k >> 48);
#pragma unroll
            for (int t = 0; t < kMaxTargets; ++t) {
                if (t >= nt) break;
                const bool in = ok && p == P[t];
                const unsigned b = __ballot_sync(kFull, in);
                if (b) {
                    const int leader = __ffs(b) - 1;
                    unsigned long long at = 0;
                    if (lane == leader) at = atomicAdd(s.app + t, (unsigned long long)__popc(b));
                    at = __shfl_sync(kFull, at, leader);
                    const unsigned long long slot = at + (unsigned long long)__popc(b & ((1u << lane) - 1u));
                    if (in && slot < (unsigned long long)kCand) s.cand[(size_t)t * kCand + slot] = k;
                }
                acc_add_warp(a + t * kAccWords, ok && p > P[t], xs[u], sc, lane);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nt * kAccWords; i += blockDim.x)
        if (a[i]) atomicAdd(&s.acc[i], a[i]);
    grid.sync();
    bool fits = true;
    for (int t = 0; t < nt; ++t) fits &= __ldcg(s.app + t) <= (unsigned long long)kCand;
    uint64_t kt[kMaxTargets];
    if (fits) {
        // 3a. block t selects among target t's kept keys in shared memory
        const int t = blockIdx.x;
        if (t < nt) {
            const int n_keys = (int)__ldcg(s.app + t);
            for (int i = threadIdx.x; i < n_keys; i += blockDim.x) keys[i] = __ldcg(s.cand + (size_t)t * kCand + i);
            if (threadIdx.x < kAccWords) a[threadIdx.x] = 0;
            __syncthreads();
            const uint64_t k = finish_in_block(keys, n_keys, st + 2 * t, h, a, sc);
            if (threadIdx.x == 0) {
                unsigned long long A[kAccWords];
                for (int i = 0; i < kAccWords; ++i) A[i] = a[i] + __ldcg(s.acc + t * kAccWords + i);
                tail_result(A, k, r.m[t], sc, s.result + 2 * t);
            }
        }
        if (blockIdx.x == 0) {   // leave the histograms and the magnitude zero for the next call
            __syncthreads();
            for (int i = threadIdx.x; i < 2 * kMaxTargets * kBins; i += blockDim.x) s.hist[i] = 0;   // passes 0, 1
            if (threadIdx.x == 0) s.ctrl[1] = 0;
        }
        return;
    }
    // 3b. a bucket of more than kCand keys: the remaining six radix passes
    //     over the whole YLT, then the buckets' values above the keys
    for (int pass = 2; pass < 8; ++pass) coop_pass(s, n, nt, pass, st, h, &s_mag, grid);
#pragma unroll
    for (int t = 0; t < kMaxTargets; ++t) kt[t] = t < nt ? st[2 * t] : ~0ull;
    for (int i = threadIdx.x; i < nt * kAccWords; i += blockDim.x) a[i] = 0;
    __syncthreads();
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n;
         base += stride * kPre) {
        double xs[kPre];
#pragma unroll
        for (int u = 0; u < kPre; ++u) {
            const int64_t i = base + u * stride + lane;
            xs[u] = i < n ? s.v[i] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < kPre; ++u) {
            const bool ok = base + u * stride + lane < n;
            const uint64_t k = key_of(xs[u]);
            const uint32_t p = (uint32_t)(k >> 48);
#pragma unroll
            for (int t = 0; t < kMaxTargets; ++t) {
                if (t >= nt) break;
                acc_add_warp(a + t * kAccWords, ok && p == P[t] && k > kt[t], xs[u], sc, lane);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nt * kAccWords; i += blockDim.x)
        if (a[i]) atomicAdd(&s.acc[i], a[i]);
    grid.sync();
    if (blockIdx.x != 0) return;
    if (threadIdx.x < nt) {
        const int t = threadIdx.x;
        unsigned long long A[kAccWords];
        for (int i = 0; i < kAccWords; ++i) A[i] = __ldcg(s.acc + t * kAccWords + i);
        tail_result(A, kt[t], r.m[t], sc, s.result + 2 * t);
    }
    __syncthreads();
    // leave the histograms and the magnitude zero for the next call
    for (int i = threadIdx.x; i < 3 * kMaxTargets * kBins; i += blockDim.x) s.hist[i] = 0;
    if (threadIdx.x == 0) s.ctrl[1] = 0;
}

cudaError_t enqueue_coop(const SelC &s, int64_t n, const int64_t *ranks, int nt, int num_sms, cudaStream_t st)
{
    Ranks r{};
    for (int t = 0; t < nt; ++t) r.m[t] = ranks[t];
    const size_t smem = sizeof(unsigned long long) * kCand;
    const int per_sm = fit_blocks(reinterpret_cast<const void *>(k_select_coop), kCoopThreads, smem);
    int64_t blocks = (n + (int64_t)kCoopThreads * kPre - 1) / ((int64_t)kCoopThreads * kPre);
    const int64_t cap = (int64_t)num_sms * per_sm;   // every block resident
    if (blocks > cap) blocks = cap;
    if (blocks < nt) blocks = nt;                    // a block per target for the last step
    SelC sc = s;
    int64_t nn = n;
    int ntt = nt;
    void *args[] = {&sc, &nn, &ntt, &r};
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(k_select_coop), dim3((unsigned)blocks),
                                       dim3(kCoopThreads), args, smem, st);
}

cudaError_t enqueue(const Sel &s, int n_ylt, int64_t n, const int64_t *ranks, int nt,
                    cudaStream_t st)
{
    Ranks r{};
    for (int t = 0; t < nt; ++t) r.m[t] = ranks[t];
    const dim3 grid((unsigned)s.blocks, (unsigned)n_ylt);
    k_init<<<n_ylt, kThreads, 0, st>>>(s, r, nt);
    for (int pass = 0; pass < 8; ++pass) k_hist<<<grid, kThreads, 0, st>>>(s, n, nt, pass);
    k_tail<<<grid, kThreads, 0, st>>>(s, n, nt, r);
    return cudaGetLastError();
}

int blocks_for(int64_t n, int cap)
{
    int64_t b = (n + kThreads * 8 - 1) / (kThreads * 8);
    if (b > cap) b = cap;
    return b < 1 ? 1 : (int)b;
}

}  // namespace

void select_alloc(SelectScratch &s, int num_sms)
{
    s.max_blocks = select_max_blocks(num_sms);
    // three histogram buffers for the cooperative selection
    ARE_CUDA_TRY(cudaMalloc(&s.hist, sizeof(uint32_t) * 3 * kMaxTargets * kBins));
    ARE_CUDA_TRY(cudaMalloc(&s.state, sizeof(unsigned long long) * 2 * kMaxTargets));
    ARE_CUDA_TRY(cudaMalloc(&s.ctrl, sizeof(unsigned int) * kCtrlWords));
    ARE_CUDA_TRY(cudaMalloc(&s.acc, sizeof(unsigned long long) * kMaxTargets * kAccWords));
    ARE_CUDA_TRY(cudaMalloc(&s.result, sizeof(double) * 2 * kMaxTargets));
    ARE_CUDA_TRY(cudaMalloc(&s.app, sizeof(unsigned long long) * kMaxTargets));
    ARE_CUDA_TRY(cudaMalloc(&s.cand, sizeof(unsigned long long) * kCand * kMaxTargets));
    // the cooperative selection leaves these zero at its end
    ARE_CUDA_TRY(cudaMemset(s.hist, 0, sizeof(uint32_t) * 3 * kMaxTargets * kBins));
    ARE_CUDA_TRY(cudaMemset(s.ctrl, 0, sizeof(unsigned int) * kCtrlWords));
    ARE_CUDA_TRY(cudaMemset(s.acc, 0, sizeof(unsigned long long) * kMaxTargets * kAccWords));
}

void select_free(SelectScratch &s)
{
    cudaFree(s.hist);
    cudaFree(s.state);
    cudaFree(s.ctrl);
    cudaFree(s.acc);
    cudaFree(s.result);
    cudaFree(s.app);
    cudaFree(s.cand);
    s = SelectScratch{};
}

// Enqueues the selection kernels; reports launch errors instead of throwing.
cudaError_t select_enqueue(const double *ylt, int64_t n, const int64_t *ranks, int nt,
                           const SelectScratch &s, cudaStream_t st)
{
    Sel sel{ylt, nullptr, s.hist, s.state, s.ctrl, s.acc, s.result, blocks_for(n, s.max_blocks)};
    return enqueue(sel, 1, n, ranks, nt, st);
}

int launch_select(const double *ylt, int64_t n, const int64_t *ranks, int nt, SelectScratch &s,
                  int num_sms, cudaStream_t st)
{
    const SelC sel{ylt, s.hist, s.acc, s.ctrl, s.app, s.cand, s.result};
    ARE_CUDA_TRY(enqueue_coop(sel, n, ranks, nt, num_sms, st));
    return 1;
}

namespace {
int multi_blocks(int n_ylt, int64_t n, int num_sms)
{
    int cap = select_max_blocks(num_sms) / (n_ylt > 0 ? n_ylt : 1);
    return blocks_for(n, cap < 1 ? 1 : cap);
}
size_t align256(size_t x) { return (x + 255) / 256 * 256; }
}  // namespace

size_t select_multi_bytes(int n_ylt, int64_t n, int num_sms)
{
    (void)n;
    (void)num_sms;
    return align256(sizeof(uint32_t) * kMaxTargets * kBins * n_ylt) +
           align256(sizeof(unsigned long long) * 2 * kMaxTargets * n_ylt) +
           align256(sizeof(unsigned int) * kCtrlWords * n_ylt) +
           align256(sizeof(unsigned long long) * kMaxTargets * kAccWords * n_ylt) +
           align256(sizeof(double) * 2 * kMaxTargets * n_ylt);
}

int launch_select_multi(const double *const *ylts, int n_ylt, int64_t n, const int64_t *ranks,
                        int nt, void *scratch, int num_sms, cudaStream_t st, double **result)
{
    unsigned char *p = static_cast<unsigned char *>(scratch);
    Sel sel;
    sel.single = nullptr;
    sel.many = ylts;
    sel.blocks = multi_blocks(n_ylt, n, num_sms);
    sel.hist = reinterpret_cast<uint32_t *>(p);
    p += align256(sizeof(uint32_t) * kMaxTargets * kBins * n_ylt);
    sel.state = reinterpret_cast<unsigned long long *>(p);
    p += align256(sizeof(unsigned long long) * 2 * kMaxTargets * n_ylt);
    sel.ctrl = reinterpret_cast<unsigned int *>(p);
    p += align256(sizeof(unsigned int) * kCtrlWords * n_ylt);
    sel.acc = reinterpret_cast<unsigned long long *>(p);
    p += align256(sizeof(unsigned long long) * kMaxTargets * kAccWords * n_ylt);
    sel.result = reinterpret_cast<double *>(p);
    *result = sel.result;
    ARE_CUDA_TRY(enqueue(sel, n_ylt, n, ranks, nt, st));
    return kSelectLaunches;
}

}  // namespace are

// ---------------------------------------------------------------------------
// Allocation-free PML/TVaR: the same kernels, with their scratch in a
// fixed-size array that lives in the library's device image.
// ---------------------------------------------------------------------------

namespace {

constexpr size_t kStaticHist = 0;                                    // 8 x 256 words
constexpr size_t kStaticState = kStaticHist + sizeof(uint32_t) * are::kMaxTargets * 256;
constexpr size_t kStaticCtrl = kStaticState + 256;                   // 4 words
constexpr size_t kStaticAcc = kStaticCtrl + 256;                     // 8 x 7 words
constexpr size_t kStaticResult = kStaticAcc + 512;                   // 2 x 8 words
static_assert(kStaticResult + 256 <= ARE_STATIC_SCRATCH_BYTES, "static scratch too small");
static_assert(sizeof(unsigned long long) * are::kMaxTargets * 7 <= 512, "accumulator slot too small");

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_static_scratch[ARE_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void *g_static_addr[kMaxDevices];   // device address of g_static_scratch, per device
int g_static_sms[kMaxDevices];
thread_local char t_static_error[192];

are_status static_fail(are_status code, const char *msg)
{
    std::snprintf(t_static_error, sizeof t_static_error, "%s", msg);
    return code;
}

}  // namespace

namespace are {
const char *static_last_error() { return t_static_error; }
}

extern "C" are_status are_risk_measures_static(const double *ylt, int64_t n,
                                               const double *return_periods, int32_t n_rp,
                                               double *pml_out, const double *tvar_levels,
                                               int32_t n_tv, double *tvar_out, void *stream)
{
    using namespace are;
    t_static_error[0] = '\0';
    if (!ylt || n <= 0) return static_fail(ARE_EINVAL, "need a device YLT of n > 0 losses");
    if (n >= (int64_t)UINT32_MAX)
        return static_fail(ARE_EINVAL, "YLT too long for the selection counters");
    if (n_rp < 0 || n_tv < 0 || (n_rp > 0 && (!return_periods || !pml_out)) ||
        (n_tv > 0 && (!tvar_levels || !tvar_out)))
        return static_fail(ARE_EINVAL, "bad PML or TVaR arrays");
    if (n_rp + n_tv > kMaxTargets)
        return static_fail(ARE_EINVAL,
                           "at most 8 return periods and TVaR levels together per call");
    if (n_rp + n_tv == 0) return ARE_OK;
    int64_t ranks[kMaxTargets];
    for (int32_t r = 0; r < n_rp; ++r)
        if ((ranks[r] = rank_for_return_period(n, return_periods[r])) < 1)
            return static_fail(ARE_EINVAL, "return period must be finite and >= 1");
    for (int32_t r = 0; r < n_tv; ++r)
        if ((ranks[n_rp + r] = rank_for_level(n, tvar_levels[r])) < 1)
            return static_fail(ARE_EINVAL, "TVaR level must lie in (0, 1)");

    int dev = 0;
    cudaPointerAttributes attr;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return static_fail(ARE_ECUDA, "no usable current CUDA device");
    }
    if (cudaPointerGetAttributes(&attr, ylt) != cudaSuccess) {
        cudaGetLastError();
        return static_fail(ARE_EINVAL, "ylt is not a CUDA pointer");
    }
    if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)
        return static_fail(ARE_EINVAL, "ylt must be device memory of the current device");
    if (attr.type == cudaMemoryTypeDevice && attr.device != dev)
        return static_fail(ARE_EINVAL, "ylt must be device memory of the current device");

    // Set-up, once per device with that device current: the device address
    // of the scratch array (its name is only a host-side stand-in).
    {
        std::lock_guard<std::mutex> lock(g_static_mu);
        if (!g_static_addr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return static_fail(ARE_ECUDA, "cudaGetSymbolAddress of the static scratch failed");
            }
            int sms = 0;
            if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
                cudaGetLastError();
                return static_fail(ARE_ECUDA, "cannot query the SM count");
            }
            g_static_sms[dev] = sms;
            g_static_addr[dev] = p;
        }
    }
    unsigned char *base = static_cast<unsigned char *>(g_static_addr[dev]);
    SelectScratch sc;
    sc.hist = reinterpret_cast<uint32_t *>(base + kStaticHist);
    sc.state = reinterpret_cast<unsigned long long *>(base + kStaticState);
    sc.ctrl = reinterpret_cast<unsigned int *>(base + kStaticCtrl);
    sc.acc = reinterpret_cast<unsigned long long *>(base + kStaticAcc);
    sc.result = reinterpret_cast<double *>(base + kStaticResult);
    sc.max_blocks = select_max_blocks(g_static_sms[dev]);

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int nt = n_rp + n_tv;
    double res[2 * kMaxTargets];
    cudaError_t e = select_enqueue(ylt, n, ranks, nt, sc, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(res, sc.result, sizeof(double) * 2 * nt, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        std::snprintf(t_static_error, sizeof t_static_error, "CUDA error: %s",
                      cudaGetErrorString(e));
        return ARE_ECUDA;
    }
    for (int32_t r = 0; r < n_rp; ++r) pml_out[r] = res[2 * r];
    for (int32_t r = 0; r < n_tv; ++r) tvar_out[r] = res[2 * (n_rp + r) + 1];
    return ARE_OK;
}
