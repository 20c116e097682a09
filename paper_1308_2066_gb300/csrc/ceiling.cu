// ceiling.cu -- the gather ceiling: a measurement helper, not a step of the
// method.
//
// The analysis stage reads, per event occurrence, the event's id from the
// YET (streamed from HBM) and the event's row of the layer's direct-access
// table (gathered; the table is small enough to stay in L2).  The ceiling
// kernel does exactly these reads and nothing else -- no financial or layer
// terms, no sums beyond a checksum that keeps the loads alive -- with each
// warp load instruction covering whole rows (16 bytes per lane).  Its rate,
// best over a few launch shapes, is the denominator of the analysis
// kernels' gather roofline.
#include <cuda_runtime.h>

#include "are_internal.cuh"

namespace are {
namespace {

template <int RB, int U>
__global__ void __launch_bounds__(256) k_gather(const int32_t *__restrict__ ids, int64_t n,
                                                const float4 *__restrict__ tab, float *__restrict__ out)
{
    constexpr int R = RB / 16, RPW = 32 / R;   // lanes per row, rows per warp load
    const int lane = threadIdx.x & 31, row = lane / R, col = lane % R;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    float acc = 0.f;
    for (int64_t base = warp * RPW * U; base < n; base += nw * RPW * U) {
        float4 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t e = base + u * RPW + row;
            const int id = e < n ? __ldcs(ids + e) : 0;
            v[u] = __ldg(tab + (int64_t)id * R + col);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) acc += v[u].x + v[u].y + v[u].z + v[u].w;
    }
    out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

template <int RB, int U>
float time_gather(const int32_t *ids, int64_t n, const float4 *tab, float *out, int blocks,
                  int reps, cudaStream_t s, cudaEvent_t a, cudaEvent_t b)
{
    float best = 1e30f;
    for (int r = 0; r < reps + 1; ++r) {       // the first launch warms L2
        ARE_CUDA_TRY(cudaEventRecord(a, s));
        k_gather<RB, U><<<blocks, 256, 0, s>>>(ids, n, tab, out);
        ARE_CUDA_TRY(cudaGetLastError());
        ARE_CUDA_TRY(cudaEventRecord(b, s));
        ARE_CUDA_TRY(cudaEventSynchronize(b));
        float ms = 0.f;
        ARE_CUDA_TRY(cudaEventElapsedTime(&ms, a, b));
        if (r > 0 && ms < best) best = ms;
    }
    return best;
}

}  // namespace

// Best time (ms) of one gather pass over n ids with rows of row_bytes (32,
// 64 or 128) from `table`; `out` holds num_sms * 8 * 256 floats.  Adds the
// launches made to `launches`.
float gather_ceiling_ms(const int32_t *ids, int64_t n, int row_bytes, int reps, int num_sms,
                        const void *table, float *out, cudaStream_t s, uint64_t &launches)
{
    cudaEvent_t a, b;
    ARE_CUDA_TRY(cudaEventCreate(&a));
    ARE_CUDA_TRY(cudaEventCreate(&b));
    float best = 1e30f;
    const float4 *tab = static_cast<const float4 *>(table);
    try {
        for (int bps : {4, 8}) {
            const int blocks = num_sms * bps;
            float ms;
            if (row_bytes == 32) {
                ms = time_gather<32, 4>(ids, n, tab, out, blocks, reps, s, a, b);
                best = ms < best ? ms : best;
                ms = time_gather<32, 8>(ids, n, tab, out, blocks, reps, s, a, b);
            } else if (row_bytes == 64) {
                ms = time_gather<64, 4>(ids, n, tab, out, blocks, reps, s, a, b);
                best = ms < best ? ms : best;
                ms = time_gather<64, 8>(ids, n, tab, out, blocks, reps, s, a, b);
            } else {
                ms = time_gather<128, 4>(ids, n, tab, out, blocks, reps, s, a, b);
                best = ms < best ? ms : best;
                ms = time_gather<128, 8>(ids, n, tab, out, blocks, reps, s, a, b);
            }
            best = ms < best ? ms : best;
            launches += 2 * (reps + 1);
        }
    } catch (...) {
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        throw;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return best;
}

}  // namespace are
