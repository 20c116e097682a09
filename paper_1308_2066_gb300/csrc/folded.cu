// folded.cu -- the folded layer table: a variant of the analysis stage.
//
// Steps 1-3 of the analysis stage (Section II-B, Algorithm 1: lookup, the
// financial terms, the sum over the layer's ELTs, the occurrence terms) see
// one occurrence at a time: the paper notes that occurrence terms apply to an
// event occurrence independently of the other occurrences of the trial.  So
// the occurrence loss of an event depends on the event and the layer alone,
// and can be computed once per catalog event:
//
//     h[e] = min(max(sum_j share_j * min(max(fx_j x_ej - D_j, 0), Lim_j) - OccR, 0), OccL)
//
// in FP64, ELT by ELT in layer order -- the same operations in the same order
// as the per-occurrence computation, so h[e] equals that occurrence loss
// bit for bit.  Step 4 then needs one value per occurrence instead of J:
// S_i = sum over the trial's occurrences of h[e_d], YLT_i = min(max(S_i - AggR, 0), AggL).
//
// This changes the work per occurrence (one lookup instead of J), so it is a
// variant beside the paper's per-ELT method, not a replacement for it.
//
// The sum.  GB300 issues FP64 adds at a small fraction of its integer rate,
// and most occurrences have h = 0.  So (a) a bitmap of the events with h > 0,
// held in shared memory, decides which occurrences need a value at all, and
// (b) the values that do are added as fixed-point integers: h * 2^s becomes a
// 128-bit integer, the trial sum is kept in 160 bits with carries (exact, in
// any order), and the total is rounded to double once.  The scale s is taken
// from the largest h of the layer, so no sum can overflow and every h of
// 2^-52 of the largest or more converts exactly.
//
// Work mapping: one warp per trial, persistent grid of one 1024-thread CTA
// per SM.  A lane loads its share of the trial's ids as 16-byte vectors, up
// to 1024 ids per trial pass issued before any is used; each lane parks its
// ids in its own shared-memory slots, marks those with h > 0 from the bitmap
// and gathers their values, two per round.
#include <cuda_runtime.h>

#include "are_internal.cuh"
#include "fixed.cuh"

namespace are {
namespace {

using namespace fixed;

constexpr unsigned kFull = 0xffffffffu;
constexpr int kFoldThreads = 1024;
constexpr int kFoldWarps = kFoldThreads / 32;
constexpr int kPass = 1024;            // ids per trial pass (32 per lane, two rounds of 16)
constexpr int kSlots = 17;             // a lane's id slots per round: 16 used, odd stride spreads banks

__device__ __forceinline__ double net(double v, double r, double l)
{
    double a = __dsub_rn(v, r);
    if (!(a > 0.0)) a = 0.0;
    if (a > l) a = l;
    return a;
}

// ---------------------------------------------------------------------------
// fold: h[e], the bitmap of h > 0 and the largest h (as bits)
//
// h starts at +0 and receives ELT j's term share_j * min(max(fx_j x - D_j,
// 0), Lim_j) for each of its entries, one launch per ELT in layer order (an
// ELT holds an event once, so no two threads of a launch touch one event).
// Events absent from an ELT would add +0, which leaves the sum unchanged, so
// skipping them keeps the sum equal to the one over all ELTs in order.
// ---------------------------------------------------------------------------

__global__ void k_fold_elt(const int32_t *__restrict__ ids, const double *__restrict__ loss,
                           int32_t n, double fx, double ded, double lim, double share,
                           double *__restrict__ h, int hstride)
{
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double *p = h + (int64_t)ids[i] * hstride;
        *p = __dadd_rn(*p, __dmul_rn(share, net(__dmul_rn(fx, loss[i]), ded, lim)));
    }
}

__global__ void k_fold_finish(int32_t catalog, double occ_r, double occ_l, double *__restrict__ h,
                              int hstride, uint32_t *__restrict__ bits, int32_t words,
                              unsigned long long *__restrict__ hmax)
{
    const int lane = threadIdx.x & 31;
    unsigned long long best = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)words * 32;
         e += stride) {
        double o = 0.0;
        if (e < catalog) {
            o = net(h[e * hstride], occ_r, occ_l);
            h[e * hstride] = o;
        }
        const unsigned long long b = (unsigned long long)__double_as_longlong(o);
        best = b > best ? b : best;
        const uint32_t m = __ballot_sync(kFull, o > 0.0);
        if (lane == 0) bits[e >> 5] = m;
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) {
        const unsigned long long o = __shfl_xor_sync(kFull, best, off);
        best = o > best ? o : best;
    }
    if (lane == 0 && best) atomicMax(hmax, best);
}

// ---------------------------------------------------------------------------
// exact fixed-point sums (fixed.cuh)
// ---------------------------------------------------------------------------

// The scale of a layer: s = 125 - floor(log2(max h)) (0 when every h is 0).
__device__ __forceinline__ int fold_scale(unsigned long long hmax_bits)
{
    return hmax_bits ? 125 - ilog2_bits(hmax_bits) : 0;
}

// F[e] = h[e] * 2^s in place: h[e] sits in the low word of F[e].
__global__ void k_fold_fixed(int32_t catalog, ulonglong2 *__restrict__ F,
                             const unsigned long long *__restrict__ hmax)
{
    const int s = fold_scale(*hmax);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < catalog;
         e += (int64_t)gridDim.x * blockDim.x) {
        const double h = __longlong_as_double((long long)F[e].x);
        ulonglong2 f;
        to_fixed(h, s, f.x, f.y);
        F[e] = f;
    }
}

// ---------------------------------------------------------------------------
// the trial pass
// ---------------------------------------------------------------------------

template <bool FIXED, bool SBITS>
__global__ void __launch_bounds__(kFoldThreads, 1) k_folded(const FoldArgs a)
{
    extern __shared__ __align__(16) uint32_t smem[];
    uint32_t *lists = smem;                                  // kFoldThreads x kSlots ids
    uint32_t *sbits = smem + kFoldThreads * kSlots;          // bitmap (SBITS)
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    if (SBITS) {
        const uint4 *src = reinterpret_cast<const uint4 *>(a.bits);
        uint4 *dst = reinterpret_cast<uint4 *>(sbits);
        for (int i = threadIdx.x; i < a.words / 4; i += blockDim.x) dst[i] = __ldg(src + i);
        __syncthreads();
    }
    const uint32_t *bm = SBITS ? sbits : a.bits;
    uint32_t *mine = lists + (wib * 32 + lane) * kSlots;     // the lane's slots
    const int s = fold_scale(*a.hmax);
    const ulonglong2 *F = a.F;

    // lane j keeps the exact sum of the j-th trial of the warp's current
    // batch of 32; a batch is finished (rounded to double, aggregate terms)
    // with one instruction sequence for its 32 trials
    unsigned long long klo = 0, khi = 0;
    uint32_t ktop = 0;
    int nb = 0;
    // a contiguous block of trials per warp, so the warp's events are one
    // contiguous run of the YET and the ids after the current pass can be
    // prefetched into L2 without knowing where the next trial starts
    const int64_t nw = (int64_t)gridDim.x * kFoldWarps, w = (int64_t)blockIdx.x * kFoldWarps + wib;
    const int t_end = (int)(a.n_trials * (w + 1) / nw);   // trial counts are below 2^31
    int tb = (int)(a.n_trials * w / nw);
    const int32_t *const ids_end = a.ids + a.n_events;
    for (int t = tb; t < t_end; ++t) {
        const int64_t tt = a.trial_begin + t;
        int64_t b, e;
        if (FIXED) {
            b = tt * a.k;
            e = b + a.k;
        } else {
            b = a.off[tt];
            e = a.off[tt + 1];
        }
        Acc acc;
        for (int64_t c0 = b & ~(int64_t)3; c0 < e; c0 += kPass) {
            // positions relative to c0: this pass covers [lo, hi)
            const int64_t rem = e - c0;
            const int hi = rem < kPass ? (int)rem : kPass;
            const int lo = b > c0 ? (int)(b - c0) : 0;   // 0..3 on the first pass, 0 after
            const unsigned span = (unsigned)(hi - lo);
            // the 1024 ids after this pass (the rest of this trial or the
            // next trials of the warp) on their way to L2, a line per lane
            {
                const int32_t *pf = a.ids + c0 + hi + 32 * lane;
                if (pf < ids_end) asm volatile("prefetch.global.L2 [%0];" ::"l"(pf));
            }
            // all of this pass's ids in flight before any is used
            int4 q[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int p = 4 * (lane + 32 * u);
                q[u] = p < hi ? __ldcs(reinterpret_cast<const int4 *>(a.ids + c0 + p))
                              : make_int4(0, 0, 0, 0);
            }
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                // which of the lane's 16 ids have h > 0; the ids go to the
                // lane's own slots, so none of this waits on another id
                uint32_t mark = 0;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int4 v4 = q[4 * half + u];
#pragma unroll
                    for (int w = 0; w < 4; ++w) {
                        const int id = w == 0 ? v4.x : w == 1 ? v4.y : w == 2 ? v4.z : v4.w;
                        const int p = 4 * (lane + 32 * (4 * half + u)) + w;
                        const uint32_t word = SBITS ? bm[(uint32_t)id >> 5] : __ldg(bm + ((uint32_t)id >> 5));
                        const uint32_t bit = __funnelshift_r(word, 0u, id) & ((unsigned)(p - lo) < span);
                        mark |= bit << (4 * u + w);
                        mine[4 * u + w] = (uint32_t)id;
                    }
                }
                // gather and add the marked ones, two per lane per round
                while (__any_sync(kFull, mark != 0)) {
                    const int k0 = __ffs(mark) - 1;
                    mark &= mark - 1;
                    const int k1 = __ffs(mark) - 1;
                    mark &= mark - 1;
                    const ulonglong2 f0 = k0 >= 0 ? __ldg(F + mine[k0]) : make_ulonglong2(0, 0);
                    const ulonglong2 f1 = k1 >= 0 ? __ldg(F + mine[k1]) : make_ulonglong2(0, 0);
                    acc.add(f0.x, f0.y, 0);
                    acc.add(f1.x, f1.y, 0);
                }
            }
        }
        warp_sum(acc);
        if (lane == nb) {
            klo = acc.lo;
            khi = acc.hi;
            ktop = acc.top;
        }
        if (++nb == 32 || t == t_end - 1) {
            if (lane < nb) {
                Acc x;
                x.lo = klo;
                x.hi = khi;
                x.top = ktop;
                a.ylt[tb + lane] = net(to_double(x, s), a.agg_r, a.agg_l);
            }
            nb = 0;
            tb = t + 1;
        }
    }
}

template <bool FIXED, bool SBITS>
int launch_folded_t(const FoldArgs &a, int num_sms, cudaStream_t st)
{
    const size_t smem = sizeof(uint32_t) * ((size_t)kFoldThreads * kSlots + (SBITS ? a.words : 0));
    ARE_CUDA_TRY(cudaFuncSetAttribute(k_folded<FIXED, SBITS>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int grid = num_sms;
    const int64_t need = (a.n_trials + kFoldWarps - 1) / kFoldWarps;
    if (need < grid) grid = (int)need;
    k_folded<FIXED, SBITS><<<grid, kFoldThreads, smem, st>>>(a);
    ARE_CUDA_TRY(cudaGetLastError());
    return 1;
}

}  // namespace

// Bitmap words of a catalog: a multiple of 4 (16-byte copies into shared memory).
int32_t folded_words(int32_t catalog)
{
    return (int32_t)((((int64_t)catalog + 127) / 128) * 4);
}

// Largest bitmap kept in shared memory beside the per-warp lists.
bool folded_bits_in_smem(int32_t words)
{
    return (size_t)words * 4 + sizeof(uint32_t) * kFoldThreads * kSlots <= 220u * 1024u;
}

int launch_fold(const ScatterArgs &elts, double occ_r, double occ_l, int32_t catalog, ulonglong2 *F,
                uint32_t *bits, unsigned long long *hmax, int num_sms, cudaStream_t s)
{
    const int32_t words = folded_words(catalog);
    double *h = reinterpret_cast<double *>(F);   // h[e] accumulates in the low word of F[e]
    ARE_CUDA_TRY(cudaMemsetAsync(hmax, 0, sizeof *hmax, s));
    ARE_CUDA_TRY(cudaMemsetAsync(F, 0, sizeof(ulonglong2) * (size_t)catalog, s));
    int launches = 0;
    for (int j = 0; j < elts.n_elts; ++j) {
        if (elts.n[j] == 0) continue;
        int blocks = (elts.n[j] + 255) / 256;
        if (blocks > num_sms * 8) blocks = num_sms * 8;
        k_fold_elt<<<blocks, 256, 0, s>>>(elts.ids[j], elts.loss[j], elts.n[j], elts.fx[j],
                                          elts.ded[j], elts.lim[j], elts.share[j], h, 2);
        ARE_CUDA_TRY(cudaGetLastError());
        ++launches;
    }
    int64_t blocks = ((int64_t)words * 32 + 255) / 256;
    if (blocks > (int64_t)num_sms * 16) blocks = (int64_t)num_sms * 16;
    k_fold_finish<<<(unsigned)blocks, 256, 0, s>>>(catalog, occ_r, occ_l, h, 2, bits, words, hmax);
    ARE_CUDA_TRY(cudaGetLastError());
    k_fold_fixed<<<(unsigned)blocks, 256, 0, s>>>(catalog, F, hmax);
    ARE_CUDA_TRY(cudaGetLastError());
    return launches + 2;
}

int launch_folded(const FoldArgs &a, int num_sms, cudaStream_t s)
{
    if (a.n_trials == 0) return 0;
    const bool sb = folded_bits_in_smem(a.words);
    if (a.off)
        return sb ? launch_folded_t<false, true>(a, num_sms, s) : launch_folded_t<false, false>(a, num_sms, s);
    return sb ? launch_folded_t<true, true>(a, num_sms, s) : launch_folded_t<true, false>(a, num_sms, s);
}

}  // namespace are
