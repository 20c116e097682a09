// select.cu -- filters on the YLT (Section II-C): PML and TVaR.
//
// The paper names PML and TVaR (Section I) without defining them; the
// library reads PML at return period RP as the m-th largest trial loss,
// m = ceil(N / RP), and TVaR at level a as the mean of the m = ceil(N(1-a))
// largest.  Both need only the m-th largest value and the sum of the values
// above it, so no sort is done: an MSB-first radix select over an
// order-preserving 64-bit key of each double finds the m-th largest key
// exactly (8 passes of 8 bits, every target rank in the same pass), then one
// more pass adds the values above it with compensated (two-sum) FP64
// arithmetic.  Everything is enqueued on one stream with the per-pass state
// in device memory, so the host waits only for the final values.
#include <cuda_runtime.h>

#include "are_internal.cuh"

namespace are {
namespace {

constexpr int kBins = 256;
constexpr int kThreads = 256;

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

// Error-free sum of two doubles (Knuth's TwoSum).
__device__ __forceinline__ void two_sum(double a, double b, double &s, double &e)
{
    s = __dadd_rn(a, b);
    const double bb = __dsub_rn(s, a);
    e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
}
struct DD {
    double hi = 0.0, lo = 0.0;
    __device__ __forceinline__ void add(double x)
    {
        double s, e;
        two_sum(hi, x, s, e);
        hi = s;
        lo = __dadd_rn(lo, e);
    }
    __device__ __forceinline__ void add(const DD &o)
    {
        double s, e;
        two_sum(hi, o.hi, s, e);
        hi = s;
        lo = __dadd_rn(lo, __dadd_rn(e, o.lo));
    }
};

struct Ranks {
    long long m[kMaxTargets];
};

// state[2t] = key prefix decided so far, state[2t+1] = rank still to find
// among the keys that share the prefix (1 = the largest of them).
__global__ void k_init(unsigned long long *state, uint32_t *hist, Ranks r, int nt)
{
    for (int i = threadIdx.x; i < nt * kBins; i += blockDim.x) hist[i] = 0;
    if (threadIdx.x < nt) {
        state[2 * threadIdx.x] = 0ull;
        state[2 * threadIdx.x + 1] = (unsigned long long)r.m[threadIdx.x];
    }
}

__global__ void __launch_bounds__(kThreads) k_hist(const double *__restrict__ y, int64_t n,
                                                   const unsigned long long *__restrict__ state,
                                                   int nt, int pass, uint32_t *hist)
{
    __shared__ uint32_t h[kMaxTargets * kBins];
    for (int i = threadIdx.x; i < nt * kBins; i += blockDim.x) h[i] = 0;
    const int shift = 56 - 8 * pass;
    uint64_t pre[kMaxTargets];
#pragma unroll
    for (int t = 0; t < kMaxTargets; ++t) pre[t] = t < nt ? state[2 * t] : 0ull;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint64_t k = key_of(y[i]);
        const uint32_t d = (uint32_t)(k >> shift) & 0xffu;
#pragma unroll
        for (int t = 0; t < kMaxTargets; ++t) {
            if (t >= nt) break;
            const bool match = pass == 0 || (k >> (shift + 8)) == (pre[t] >> (shift + 8));
            if (match) atomicAdd(&h[t * kBins + d], 1u);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nt * kBins; i += blockDim.x)
        if (h[i]) atomicAdd(&hist[i], h[i]);
}

// One warp per target: find the bucket that holds the wanted rank, descending.
__global__ void k_pick(unsigned long long *state, uint32_t *hist, int nt, int pass)
{
    const int t = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (t >= nt) return;
    const int shift = 56 - 8 * pass;
    uint32_t *h = hist + t * kBins;
    uint32_t c[8];
    unsigned long long lane_sum = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        c[i] = h[kBins - 1 - (lane * 8 + i)];  // lane 0 holds the top buckets
        lane_sum += c[i];
    }
    unsigned long long incl = lane_sum;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const unsigned long long o = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += o;
    }
    const unsigned long long excl = incl - lane_sum;
    const unsigned long long r = state[2 * t + 1];
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 8; ++i) h[kBins - 1 - (lane * 8 + i)] = 0;
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
        state[2 * t] |= (unsigned long long)b << shift;
        state[2 * t + 1] = r - above;
    }
}

// Per block and target: compensated sum and count of the values whose key
// is above the selected key.
__global__ void __launch_bounds__(kThreads) k_tail(const double *__restrict__ y, int64_t n,
                                                   const unsigned long long *__restrict__ state,
                                                   int nt, double *partial)
{
    uint64_t kt[kMaxTargets];
    DD acc[kMaxTargets];
    unsigned long long cnt[kMaxTargets];
#pragma unroll
    for (int t = 0; t < kMaxTargets; ++t) {
        kt[t] = t < nt ? state[2 * t] : ~0ull;
        cnt[t] = 0;
    }
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const double v = y[i];
        const uint64_t k = key_of(v);
#pragma unroll
        for (int t = 0; t < kMaxTargets; ++t)
            if (k > kt[t]) {
                acc[t].add(v);
                ++cnt[t];
            }
    }
    __shared__ double sh[kThreads / 32][kMaxTargets][3];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int t = 0; t < kMaxTargets; ++t) {
        for (int off = 16; off > 0; off >>= 1) {
            DD o;
            o.hi = __shfl_down_sync(0xffffffffu, acc[t].hi, off);
            o.lo = __shfl_down_sync(0xffffffffu, acc[t].lo, off);
            cnt[t] += __shfl_down_sync(0xffffffffu, cnt[t], off);
            acc[t].add(o);
        }
        if (lane == 0) {
            sh[w][t][0] = acc[t].hi;
            sh[w][t][1] = acc[t].lo;
            sh[w][t][2] = (double)cnt[t];
        }
    }
    __syncthreads();
    if (threadIdx.x < nt) {
        const int t = threadIdx.x;
        DD s;
        double c = 0.0;
        for (int i = 0; i < kThreads / 32; ++i) {
            DD o;
            o.hi = sh[i][t][0];
            o.lo = sh[i][t][1];
            s.add(o);
            c += sh[i][t][2];
        }
        double *p = partial + ((size_t)blockIdx.x * kMaxTargets + t) * 3;
        p[0] = s.hi;
        p[1] = s.lo;
        p[2] = c;
    }
}

// One warp per target: adds the blocks' partial sums in block order, then
// the ties at the selected value, and writes (value, mean of the m largest).
__global__ void k_final(const unsigned long long *state, const double *partial, int n_blocks,
                        Ranks r, int nt, double *result)
{
    const int t = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (t >= nt) return;
    DD s;
    double c = 0.0;
    for (int b = lane; b < n_blocks; b += 32) {
        const double *p = partial + ((size_t)b * kMaxTargets + t) * 3;
        DD o;
        o.hi = p[0];
        o.lo = p[1];
        s.add(o);
        c += p[2];
    }
    for (int off = 16; off > 0; off >>= 1) {
        DD o;
        o.hi = __shfl_down_sync(0xffffffffu, s.hi, off);
        o.lo = __shfl_down_sync(0xffffffffu, s.lo, off);
        c += __shfl_down_sync(0xffffffffu, c, off);
        s.add(o);
    }
    if (lane == 0) {
        const double v = value_of(state[2 * t]);
        const double m = (double)r.m[t];
        s.add(__dmul_rn(m - c, v));
        result[2 * t] = v;
        result[2 * t + 1] = __ddiv_rn(__dadd_rn(s.hi, s.lo), m);
    }
}

}  // namespace

void select_alloc(SelectScratch &s, int num_sms)
{
    s.max_blocks = num_sms * 4;
    ARE_CUDA_TRY(cudaMalloc(&s.hist, sizeof(uint32_t) * kMaxTargets * kBins));
    ARE_CUDA_TRY(cudaMalloc(&s.state, sizeof(unsigned long long) * 2 * kMaxTargets));
    ARE_CUDA_TRY(cudaMalloc(&s.partial, sizeof(double) * 3 * kMaxTargets * s.max_blocks));
    ARE_CUDA_TRY(cudaMalloc(&s.result, sizeof(double) * 2 * kMaxTargets));
}

void select_free(SelectScratch &s)
{
    cudaFree(s.hist);
    cudaFree(s.state);
    cudaFree(s.partial);
    cudaFree(s.result);
    s = SelectScratch{};
}

int launch_select(const double *ylt, int64_t n, const int64_t *ranks, int nt, SelectScratch &s,
                   int num_sms, cudaStream_t st)
{
    Ranks r{};
    for (int t = 0; t < nt; ++t) r.m[t] = ranks[t];
    int64_t blocks = (n + kThreads * 8 - 1) / (kThreads * 8);
    if (blocks > s.max_blocks) blocks = s.max_blocks;
    if (blocks < 1) blocks = 1;
    (void)num_sms;
    k_init<<<1, kThreads, 0, st>>>(s.state, s.hist, r, nt);
    for (int pass = 0; pass < 8; ++pass) {
        k_hist<<<(unsigned)blocks, kThreads, 0, st>>>(ylt, n, s.state, nt, pass, s.hist);
        k_pick<<<1, 32 * kMaxTargets, 0, st>>>(s.state, s.hist, nt, pass);
    }
    k_tail<<<(unsigned)blocks, kThreads, 0, st>>>(ylt, n, s.state, nt, s.partial);
    k_final<<<1, 32 * kMaxTargets, 0, st>>>(s.state, s.partial, (int)blocks, r, nt, s.result);
    ARE_CUDA_TRY(cudaGetLastError());
    return 2 + 2 * 8 + 2;
}

}  // namespace are
