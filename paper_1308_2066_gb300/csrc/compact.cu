// compact.cu -- the compact layer table (FP32): a row index row_of[catalog]
// and rows only for the events present in at least one of the layer's ELTs.
//
// The direct-access layout (Section III-B) spends a row on every catalog
// event.  When the catalog is large and the ELTs sparse -- 2,000,000 events
// and 32 ELTs of 20,000 entries: 256 MB of rows, twice the L2, for 640,000
// entries -- the rows of the events that occur in some ELT are enough: here
// 560,000 rows (72 MB) and a 8 MB index, which stay in L2.  An event without
// a row has a zero loss in every ELT.  The build runs on the device: mark
// the present events, number them with an exclusive scan over the catalog
// (per-tile counts, one scan of the counts, per-tile numbering), then
// scatter each ELT entry into its row.
#include <cuda_runtime.h>

#include "are_internal.cuh"

namespace are {
namespace {

constexpr int kScanThreads = 1024;
constexpr int kPerThread = 4;
constexpr int kTile = kScanThreads * kPerThread;   // catalog events per scan block

__global__ void k_mark_present(const ScatterArgs a, int32_t *__restrict__ row_of)
{
    const int j = blockIdx.y;
    const int32_t *ids = a.ids[j];
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n[j]; i += gridDim.x * blockDim.x)
        row_of[ids[i]] = 0;
}

// Inclusive scan of one value per thread over a block of kScanThreads.
__device__ __forceinline__ int block_scan(int v, int *warp_sums)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int o = __shfl_up_sync(0xffffffffu, v, off);
        if (lane >= off) v += o;
    }
    if (lane == 31) warp_sums[w] = v;
    __syncthreads();
    if (w == 0) {
        int s = lane < kScanThreads / 32 ? warp_sums[lane] : 0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int o = __shfl_up_sync(0xffffffffu, s, off);
            if (lane >= off) s += o;
        }
        warp_sums[lane] = s;
    }
    __syncthreads();
    const int add = w > 0 ? warp_sums[w - 1] : 0;
    __syncthreads();
    return v + add;
}

__global__ void __launch_bounds__(kScanThreads) k_count_present(const int32_t *__restrict__ row_of,
                                                                 int32_t catalog, int32_t *counts)
{
    __shared__ int warp_sums[32];
    const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kPerThread;
    int c = 0;
#pragma unroll
    for (int k = 0; k < kPerThread; ++k) c += base + k < catalog && row_of[base + k] >= 0;
    const int incl = block_scan(c, warp_sums);
    if (threadIdx.x == kScanThreads - 1) counts[blockIdx.x] = incl;
}

// Exclusive scan of the per-tile counts in place (one block).
__global__ void __launch_bounds__(kScanThreads) k_scan_counts(int32_t *counts, int n)
{
    __shared__ int warp_sums[32];
    const int per = (n + kScanThreads - 1) / kScanThreads;
    const int b = threadIdx.x * per;
    int s = 0;
    for (int i = 0; i < per; ++i)
        if (b + i < n) s += counts[b + i];
    const int excl = block_scan(s, warp_sums) - s;
    int run = excl;
    for (int i = 0; i < per; ++i)
        if (b + i < n) {
            const int v = counts[b + i];
            counts[b + i] = run;
            run += v;
        }
}

__global__ void __launch_bounds__(kScanThreads) k_number_rows(int32_t *__restrict__ row_of, int32_t catalog,
                                                               const int32_t *__restrict__ offsets)
{
    __shared__ int warp_sums[32];
    const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kPerThread;
    int f[kPerThread], c = 0;
#pragma unroll
    for (int k = 0; k < kPerThread; ++k) {
        f[k] = base + k < catalog && row_of[base + k] >= 0;
        c += f[k];
    }
    int row = offsets[blockIdx.x] + block_scan(c, warp_sums) - c;
#pragma unroll
    for (int k = 0; k < kPerThread; ++k)
        if (f[k]) row_of[base + k] = row++;
}

__global__ void k_scatter_compact(float *__restrict__ rows, const int32_t *__restrict__ row_of,
                                  const ScatterArgs a)
{
    const int j = blockIdx.y;
    const int32_t *ids = a.ids[j];
    const double *loss = a.loss[j];
    const double fx = a.fx[j], ded = a.ded[j], lim = a.lim[j], share = a.share[j];
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n[j]; i += gridDim.x * blockDim.x)
        rows[(size_t)row_of[ids[i]] * a.jp + j] = (float)fin_term(loss[i], fx, ded, lim, share);
}

}  // namespace

int64_t compact_scan_blocks(int32_t catalog) { return ((int64_t)catalog + kTile - 1) / kTile; }

// row_of: catalog int32; counts: compact_scan_blocks(catalog) int32 scratch;
// rows: max_rows x a.jp floats (max_rows >= the number of present events).
int launch_build_compact(int32_t *row_of, int32_t *counts, float *rows, size_t rows_bytes,
                         int32_t catalog, const ScatterArgs &a, cudaStream_t s)
{
    ARE_CUDA_TRY(cudaMemsetAsync(row_of, 0xff, sizeof(int32_t) * (size_t)catalog, s));
    ARE_CUDA_TRY(cudaMemsetAsync(rows, 0, rows_bytes, s));
    int32_t nmax = 0;
    for (int j = 0; j < a.n_elts; ++j) nmax = a.n[j] > nmax ? a.n[j] : nmax;
    int launches = 0;
    if (nmax > 0 && a.n_elts > 0) {
        dim3 grid((unsigned)((nmax + 255) / 256), (unsigned)a.n_elts);
        if (grid.x > 4096) grid.x = 4096;
        k_mark_present<<<grid, 256, 0, s>>>(a, row_of);
        ARE_CUDA_TRY(cudaGetLastError());
        const int64_t nb = compact_scan_blocks(catalog);
        k_count_present<<<(unsigned)nb, kScanThreads, 0, s>>>(row_of, catalog, counts);
        k_scan_counts<<<1, kScanThreads, 0, s>>>(counts, (int)nb);
        k_number_rows<<<(unsigned)nb, kScanThreads, 0, s>>>(row_of, catalog, counts);
        k_scatter_compact<<<grid, 256, 0, s>>>(rows, row_of, a);
        ARE_CUDA_TRY(cudaGetLastError());
        launches = 5;
    }
    return launches;
}

}  // namespace are
