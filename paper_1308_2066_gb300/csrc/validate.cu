// validate.cu -- device-side checks of a YET as it is loaded: event ids in
// [0, catalog), CSR offsets starting at 0, non-decreasing and ending at the
// event count, timestamps non-decreasing within each trial.  The YET is
// gigabytes at paper scale (Section III-B: 800M-1500M ids), so it is checked
// where it lands rather than on the host.  A kernel that finds a violation
// sets *flag; the host reads the flag after the kernels.
#include <cuda_runtime.h>

#include "are_internal.cuh"

namespace are {
namespace {

constexpr int kBlocks = 4096;

__global__ void k_check_ids(const int32_t *__restrict__ ids, int64_t n, int32_t catalog,
                            int *flag)
{
    int bad = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int32_t v = __ldcs(ids + i);
        bad |= (v < 0) | (v >= catalog);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

// The same check on ids that a kernel is about to read: an id outside the
// catalog is replaced by 0, so no table read goes out of bounds, and flagged.
__global__ void k_sanitize_ids(int32_t *__restrict__ ids, int64_t n, int32_t catalog, int *flag)
{
    int bad = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int32_t v = ids[i];
        if (v < 0 || v >= catalog) {
            ids[i] = 0;
            bad = 1;
        }
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

// Ids of `bits` bits each (1 .. 32), packed little-endian into 32-bit
// words: id j starts at bit bit0 + j * bits of `words`, which must be
// readable one word past the last id.  Writes them as int32 to out; an id
// outside [0, catalog) is written as 0 and sets bit 0 of *flag.
__global__ void k_unpack_ids(const uint32_t *__restrict__ words, int64_t bit0, int bits, int64_t n,
                             int32_t catalog, int32_t *__restrict__ out, int *flag)
{
    int bad = 0;
    const uint64_t mask = bits >= 32 ? 0xffffffffull : ((1ull << bits) - 1ull);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int64_t b = bit0 + i * bits;
        const int64_t w = b >> 5;
        const uint64_t x = (((uint64_t)__ldg(words + w + 1) << 32) | __ldg(words + w)) >> (b & 31);
        const uint32_t v = (uint32_t)(x & mask);
        const bool ok = v < (uint32_t)catalog;
        __stcs(out + i, ok ? (int32_t)v : 0);
        bad |= !ok;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

__global__ void k_check_offsets(const int64_t *__restrict__ off, int64_t n_trials,
                                int64_t n_events, int *flag)
{
    int bad = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_trials; i += stride)
        bad |= off[i + 1] < off[i];
    if (blockIdx.x == 0 && threadIdx.x == 0) bad |= (off[0] != 0) | (off[n_trials] != n_events);
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 2);
}

__global__ void k_check_ts(const float *__restrict__ ts, const int64_t *__restrict__ off,
                           int64_t n_trials, int32_t k, int *flag)
{
    int bad = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n_trials; t += stride) {
        const int64_t b = off ? off[t] : t * (int64_t)k;
        const int64_t e = off ? off[t + 1] : b + k;
        for (int64_t i = b + 1; i < e; ++i) bad |= !(ts[i] >= ts[i - 1]);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 4);
}

unsigned blocks_for(int64_t n)
{
    int64_t b = (n + 255) / 256;
    if (b > kBlocks) b = kBlocks;
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

int launch_check_ids(const int32_t *ids, int64_t n, int32_t catalog, int *flag, cudaStream_t s)
{
    if (n <= 0) return 0;
    k_check_ids<<<blocks_for(n), 256, 0, s>>>(ids, n, catalog, flag);
    ARE_CUDA_TRY(cudaGetLastError());
    return 1;
}

int launch_check_offsets(const int64_t *off, int64_t n_trials, int64_t n_events, int *flag,
                          cudaStream_t s)
{
    k_check_offsets<<<blocks_for(n_trials), 256, 0, s>>>(off, n_trials, n_events, flag);
    ARE_CUDA_TRY(cudaGetLastError());
    return 1;
}

int launch_check_timestamps(const float *ts, const int64_t *off, int64_t n_trials, int32_t k,
                             int *flag, cudaStream_t s)
{
    if (n_trials <= 0) return 0;
    k_check_ts<<<blocks_for(n_trials), 256, 0, s>>>(ts, off, n_trials, k, flag);
    ARE_CUDA_TRY(cudaGetLastError());
    return 1;
}

int launch_unpack_ids(const uint32_t *words, int64_t bit0, int bits, int64_t n, int32_t catalog, int32_t *out,
                      int *flag, cudaStream_t s)
{
    if (n <= 0) return 0;
    k_unpack_ids<<<blocks_for(n), 256, 0, s>>>(words, bit0, bits, n, catalog, out, flag);
    ARE_CUDA_TRY(cudaGetLastError());
    return 1;
}

int launch_sanitize_ids(int32_t *ids, int64_t n, int32_t catalog, int *flag, cudaStream_t s)
{
    if (n <= 0) return 0;
    k_sanitize_ids<<<blocks_for(n), 256, 0, s>>>(ids, n, catalog, flag);
    ARE_CUDA_TRY(cudaGetLastError());
    return 1;
}

}  // namespace are
