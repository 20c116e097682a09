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

#include <cstdio>
#include <mutex>

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

// Scratch of one selection over n_ylt YLTs (blockIdx.y or blockIdx.x picks
// the YLT): per YLT 8 x 256 histogram words, 8 x (prefix, rank) state words,
// blocks x 8 x 3 partial sums, 8 x 2 results.
struct Sel {
    const double *single;        // the YLT when there is one
    const double *const *many;   // device array of YLT pointers, or nullptr
    uint32_t *hist;
    unsigned long long *state;
    double *partial;
    double *result;
    int blocks;                  // blocks per YLT in the histogram and tail passes
};
__device__ __forceinline__ const double *ylt_of(const Sel &s, int y)
{
    return s.many ? s.many[y] : s.single;
}

// state[2t] = key prefix decided so far, state[2t+1] = rank still to find
// among the keys that share the prefix (1 = the largest of them).
__global__ void k_init(Sel s, Ranks r, int nt)
{
    const int y = blockIdx.x;
    uint32_t *hist = s.hist + (size_t)y * kMaxTargets * kBins;
    unsigned long long *state = s.state + (size_t)y * 2 * kMaxTargets;
    for (int i = threadIdx.x; i < nt * kBins; i += blockDim.x) hist[i] = 0;
    if (threadIdx.x < nt) {
        state[2 * threadIdx.x] = 0ull;
        state[2 * threadIdx.x + 1] = (unsigned long long)r.m[threadIdx.x];
    }
}

__global__ void __launch_bounds__(kThreads) k_hist(Sel s, int64_t n, int nt, int pass)
{
    const int y = blockIdx.y;
    const double *__restrict__ v = ylt_of(s, y);
    const unsigned long long *state = s.state + (size_t)y * 2 * kMaxTargets;
    uint32_t *hist = s.hist + (size_t)y * kMaxTargets * kBins;
    __shared__ uint32_t h[kMaxTargets * kBins];
    for (int i = threadIdx.x; i < nt * kBins; i += blockDim.x) h[i] = 0;
    const int shift = 56 - 8 * pass;
    uint64_t pre[kMaxTargets];
#pragma unroll
    for (int t = 0; t < kMaxTargets; ++t) pre[t] = t < nt ? state[2 * t] : 0ull;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint64_t k = key_of(v[i]);
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
__global__ void k_pick(Sel s, int nt, int pass)
{
    const int y = blockIdx.x;
    const int t = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (t >= nt) return;
    unsigned long long *state = s.state + (size_t)y * 2 * kMaxTargets;
    const int shift = 56 - 8 * pass;
    uint32_t *h = s.hist + ((size_t)y * kMaxTargets + t) * kBins;
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
__global__ void __launch_bounds__(kThreads) k_tail(Sel s, int64_t n, int nt)
{
    const int y = blockIdx.y;
    const double *__restrict__ v = ylt_of(s, y);
    const unsigned long long *state = s.state + (size_t)y * 2 * kMaxTargets;
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
        const double x = v[i];
        const uint64_t k = key_of(x);
#pragma unroll
        for (int t = 0; t < kMaxTargets; ++t)
            if (k > kt[t]) {
                acc[t].add(x);
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
        DD sum;
        double c = 0.0;
        for (int i = 0; i < kThreads / 32; ++i) {
            DD o;
            o.hi = sh[i][t][0];
            o.lo = sh[i][t][1];
            sum.add(o);
            c += sh[i][t][2];
        }
        double *p = s.partial + (((size_t)y * s.blocks + blockIdx.x) * kMaxTargets + t) * 3;
        p[0] = sum.hi;
        p[1] = sum.lo;
        p[2] = c;
    }
}

// One warp per target: adds the blocks' partial sums in block order, then
// the ties at the selected value, and writes (value, mean of the m largest).
__global__ void k_final(Sel s, Ranks r, int nt)
{
    const int y = blockIdx.x;
    const int t = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (t >= nt) return;
    const unsigned long long *state = s.state + (size_t)y * 2 * kMaxTargets;
    DD sum;
    double c = 0.0;
    for (int b = lane; b < s.blocks; b += 32) {
        const double *p = s.partial + (((size_t)y * s.blocks + b) * kMaxTargets + t) * 3;
        DD o;
        o.hi = p[0];
        o.lo = p[1];
        sum.add(o);
        c += p[2];
    }
    for (int off = 16; off > 0; off >>= 1) {
        DD o;
        o.hi = __shfl_down_sync(0xffffffffu, sum.hi, off);
        o.lo = __shfl_down_sync(0xffffffffu, sum.lo, off);
        c += __shfl_down_sync(0xffffffffu, c, off);
        sum.add(o);
    }
    if (lane == 0) {
        const double v = value_of(state[2 * t]);
        const double m = (double)r.m[t];
        sum.add(__dmul_rn(m - c, v));
        double *res = s.result + (size_t)y * 2 * kMaxTargets;
        res[2 * t] = v;
        res[2 * t + 1] = __ddiv_rn(__dadd_rn(sum.hi, sum.lo), m);
    }
}

cudaError_t enqueue(const Sel &s, int n_ylt, int64_t n, const int64_t *ranks, int nt,
                    cudaStream_t st)
{
    Ranks r{};
    for (int t = 0; t < nt; ++t) r.m[t] = ranks[t];
    const dim3 grid((unsigned)s.blocks, (unsigned)n_ylt);
    k_init<<<n_ylt, kThreads, 0, st>>>(s, r, nt);
    for (int pass = 0; pass < 8; ++pass) {
        k_hist<<<grid, kThreads, 0, st>>>(s, n, nt, pass);
        k_pick<<<n_ylt, 32 * kMaxTargets, 0, st>>>(s, nt, pass);
    }
    k_tail<<<grid, kThreads, 0, st>>>(s, n, nt);
    k_final<<<n_ylt, 32 * kMaxTargets, 0, st>>>(s, r, nt);
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

// Enqueues the selection kernels; reports launch errors instead of throwing.
cudaError_t select_enqueue(const double *ylt, int64_t n, const int64_t *ranks, int nt,
                           const SelectScratch &s, cudaStream_t st)
{
    Sel sel{ylt, nullptr, s.hist, s.state, s.partial, s.result, blocks_for(n, s.max_blocks)};
    return enqueue(sel, 1, n, ranks, nt, st);
}

int launch_select(const double *ylt, int64_t n, const int64_t *ranks, int nt, SelectScratch &s,
                  int num_sms, cudaStream_t st)
{
    (void)num_sms;
    ARE_CUDA_TRY(select_enqueue(ylt, n, ranks, nt, s, st));
    return kSelectLaunches;
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
    const size_t blocks = (size_t)multi_blocks(n_ylt, n, num_sms);
    return align256(sizeof(uint32_t) * kMaxTargets * kBins * n_ylt) +
           align256(sizeof(unsigned long long) * 2 * kMaxTargets * n_ylt) +
           align256(sizeof(double) * 3 * kMaxTargets * blocks * n_ylt) +
           align256(sizeof(double) * 2 * kMaxTargets * n_ylt);
}

int launch_select_multi(const double *const *ylts, int n_ylt, int64_t n, const int64_t *ranks,
                        int nt, void *scratch, int num_sms, cudaStream_t st, double **result)
{
    const int blocks = multi_blocks(n_ylt, n, num_sms);
    unsigned char *p = static_cast<unsigned char *>(scratch);
    Sel sel;
    sel.single = nullptr;
    sel.many = ylts;
    sel.blocks = blocks;
    sel.hist = reinterpret_cast<uint32_t *>(p);
    p += align256(sizeof(uint32_t) * kMaxTargets * kBins * n_ylt);
    sel.state = reinterpret_cast<unsigned long long *>(p);
    p += align256(sizeof(unsigned long long) * 2 * kMaxTargets * n_ylt);
    sel.partial = reinterpret_cast<double *>(p);
    p += align256(sizeof(double) * 3 * kMaxTargets * (size_t)blocks * n_ylt);
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
constexpr size_t kStaticResult = kStaticState + 256;                 // 2 x 8 words
constexpr size_t kStaticPartial = kStaticResult + 256;               // blocks x 8 x 3 doubles
constexpr int kStaticMaxBlocks = 1024;
static_assert(kStaticPartial + sizeof(double) * 3 * are::kMaxTargets * kStaticMaxBlocks <=
                  ARE_STATIC_SCRATCH_BYTES,
              "static scratch too small for its block limit");

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
    sc.result = reinterpret_cast<double *>(base + kStaticResult);
    sc.partial = reinterpret_cast<double *>(base + kStaticPartial);
    sc.max_blocks = select_max_blocks(g_static_sms[dev]);
    if (sc.max_blocks > kStaticMaxBlocks) sc.max_blocks = kStaticMaxBlocks;

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
