// ceiling.cu -- the gather ceiling: a measurement helper, not a step of the
// method.
//
// The analysis stage reads, per event occurrence, the event's id from the
// YET (streamed from HBM) and the event's row of the layer's direct-access
// table (gathered; the table is small enough to stay in L2).  The ceiling
// kernels do exactly these reads and nothing else -- no terms, no sums
// beyond a checksum that keeps the loads alive -- in three shapes, each over
// a range of rows in flight and blocks per SM:
//   0  16-byte loads, row_bytes/16 lanes per row, each lane reading its
//      row's id itself;
//   1  32-byte loads, row_bytes/32 lanes per row, ids read once per 32
//      events with one coalesced load and passed by shuffles (the shape of
//      the register-rows analysis kernel);
//   2  rows copied global -> shared with 16-byte cp.async, whole rows per
//      copy instruction (the shape of the staged analysis kernels), then
//      one value of each row read back.
// The best rate over all shapes is the denominator of the analysis
// kernels' gather roofline.
#include <cuda_runtime.h>

#include <vector>

#include "are_internal.cuh"

namespace are {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kThreads = 256;

struct F8 {
    float v[8];
};

__device__ __forceinline__ F8 load8(const float *p)
{
    F8 r;
    asm volatile("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=f"(r.v[0]), "=f"(r.v[1]), "=f"(r.v[2]), "=f"(r.v[3]), "=f"(r.v[4]),
                   "=f"(r.v[5]), "=f"(r.v[6]), "=f"(r.v[7])
                 : "l"(p));
    return r;
}

__device__ __forceinline__ float4 load4(const float4 *p)
{
    float4 r;
    asm volatile("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
                 : "l"(p));
    return r;
}

// shape 0: lane (row, col) reads its row's id and one 16-byte piece, U rows
// per lane in flight (the loads are issued before any is used).
template <int RB, int U>
__global__ void __launch_bounds__(kThreads) k_gather(const int32_t *__restrict__ ids, int64_t n,
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
            v[u] = load4(tab + (int64_t)id * R + col);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) acc += v[u].x + v[u].y + v[u].z + v[u].w;
    }
    out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

// shape 1: U groups of 32 events per batch; a group's ids in one coalesced
// load, its rows read by RB/32 lanes each with 32-byte loads.
template <int RB, int U>
__global__ void __launch_bounds__(kThreads) k_gather_rows(const int32_t *__restrict__ ids, int64_t n,
                                                          const float *__restrict__ tab,
                                                          float *__restrict__ out)
{
    constexpr int R = RB / 32, RPW = 32 / R;
    const int lane = threadIdx.x & 31, row = lane / R, col = lane % R;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    float acc = 0.f;
    for (int64_t base = warp * 32 * U; base < n; base += nw * 32 * U) {
        int32_t id[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t e = base + u * 32 + lane;
            id[u] = e < n ? __ldcs(ids + e) : 0;
        }
        F8 v[U][R];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int32_t e = __shfl_sync(kFull, id[u], q * RPW + row);
                v[u][q] = load8(tab + (size_t)(uint32_t)e * (RB / 4) + col * 8);
            }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int q = 0; q < R; ++q)
#pragma unroll
                for (int i = 0; i < 8; ++i) acc += v[u][q].v[i];
    }
    out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}

// shape 2: each warp copies the rows of 32 * U events into its shared
// buffer with cp.async (a copy instruction covers 32 / (RB / 16) whole rows),
// waits, and reads one value per row back.
template <int RB, int U>
__global__ void __launch_bounds__(kThreads) k_gather_staged(const int32_t *__restrict__ ids, int64_t n,
                                                            const char *__restrict__ tab,
                                                            float *__restrict__ out)
{
    constexpr int CH = RB / 16;                 // 16-byte chunks per row
    constexpr int ROWS = 32 * U;
    extern __shared__ float4 stage[];
    const int lane = threadIdx.x & 31;
    float4 *buf = stage + (size_t)(threadIdx.x >> 5) * ROWS * CH;
    const uint32_t sbuf = (uint32_t)__cvta_generic_to_shared(buf);
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    float acc = 0.f;
    for (int64_t base = warp * ROWS; base < n; base += nw * ROWS) {
        int32_t id[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t e = base + u * 32 + lane;
            id[u] = e < n ? __ldcs(ids + e) : 0;
        }
#pragma unroll
        for (int i = 0; i < ROWS * CH / 32; ++i) {
            const int q = lane + 32 * i, r = q / CH, c = q % CH;
            const int32_t src = U == 1 ? id[0] : ((r >> 5) ? id[U - 1] : id[0]);
            const int32_t e = __shfl_sync(kFull, src, r & 31);
            cp_async16(sbuf + (uint32_t)(r * CH + c) * 16u, tab + (size_t)(uint32_t)e * RB + c * 16);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncwarp();
#pragma unroll
        for (int u = 0; u < U; ++u) acc += buf[(u * 32 + lane) * CH].x;
        __syncwarp();
    }
    out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

template <typename F>
float best_ms(F launch, int reps, cudaStream_t s, cudaEvent_t a, cudaEvent_t b)
{
    float best = 1e30f;
    for (int r = 0; r < reps + 1; ++r) {       // the first launch warms L2
        ARE_CUDA_TRY(cudaEventRecord(a, s));
        launch();
        ARE_CUDA_TRY(cudaGetLastError());
        ARE_CUDA_TRY(cudaEventRecord(b, s));
        ARE_CUDA_TRY(cudaEventSynchronize(b));
        float ms = 0.f;
        ARE_CUDA_TRY(cudaEventElapsedTime(&ms, a, b));
        if (r > 0 && ms < best) best = ms;
    }
    return best;
}

// Every shape of one row size.  Each kernel's blocks per SM are tried up to
// what fits.
template <int RB>
void sweep(const int32_t *ids, int64_t n, const void *table, float *out, int reps, int num_sms,
           cudaStream_t s, cudaEvent_t a, cudaEvent_t b, std::vector<CeilingShape> &res,
           uint64_t &launches)
{
    auto run = [&](int kind, int u, const void *kern, size_t smem, auto launch) {
        const int fit = fit_blocks(kern, kThreads, smem);
        for (int bps : {3, 4, 6, 8, 0}) {
            if (bps == 0) {   // a shape that fits fewer than 3 blocks: as many as fit
                if (fit >= 3) break;
                bps = fit;
            } else if (bps > fit) {
                continue;
            }
            const int blocks = num_sms * bps;
            const float ms = best_ms([&] { launch(blocks); }, reps, s, a, b);
            launches += (uint64_t)reps + 1;
            res.push_back(CeilingShape{kind, u, bps, (double)n / ((double)ms * 1e-3)});
        }
    };
    const float4 *t4 = static_cast<const float4 *>(table);
    const float *tf = static_cast<const float *>(table);
    const char *tc = static_cast<const char *>(table);
    run(0, 4, reinterpret_cast<const void *>(k_gather<RB, 4>), 0,
        [&](int g) { k_gather<RB, 4><<<g, kThreads, 0, s>>>(ids, n, t4, out); });
    run(0, 8, reinterpret_cast<const void *>(k_gather<RB, 8>), 0,
        [&](int g) { k_gather<RB, 8><<<g, kThreads, 0, s>>>(ids, n, t4, out); });
    run(0, 16, reinterpret_cast<const void *>(k_gather<RB, 16>), 0,
        [&](int g) { k_gather<RB, 16><<<g, kThreads, 0, s>>>(ids, n, t4, out); });
    run(1, 1, reinterpret_cast<const void *>(k_gather_rows<RB, 1>), 0,
        [&](int g) { k_gather_rows<RB, 1><<<g, kThreads, 0, s>>>(ids, n, tf, out); });
    run(1, 2, reinterpret_cast<const void *>(k_gather_rows<RB, 2>), 0,
        [&](int g) { k_gather_rows<RB, 2><<<g, kThreads, 0, s>>>(ids, n, tf, out); });
    constexpr int U4 = RB <= 64 ? 4 : 2;   // 128-byte rows: as many registers as U = 2 at 64
    if (RB <= 64)
        run(1, U4, reinterpret_cast<const void *>(k_gather_rows<RB, U4>), 0,
            [&](int g) { k_gather_rows<RB, U4><<<g, kThreads, 0, s>>>(ids, n, tf, out); });
    for (int u : {1, 2}) {
        const size_t smem = (size_t)(kThreads / 32) * 32 * u * RB;
        const void *k = u == 1 ? reinterpret_cast<const void *>(k_gather_staged<RB, 1>)
                               : reinterpret_cast<const void *>(k_gather_staged<RB, 2>);
        run(2, u, k, smem, [&](int g) {
            if (u == 1) k_gather_staged<RB, 1><<<g, kThreads, smem, s>>>(ids, n, tc, out);
            else k_gather_staged<RB, 2><<<g, kThreads, smem, s>>>(ids, n, tc, out);
        });
    }
}

}  // namespace

// Every shape's rate (rows per second) of one gather pass over n ids with
// rows of row_bytes (32, 64 or 128) from `table`; `out` holds num_sms * 8 *
// 256 floats.  Adds the launches made to `launches`.
std::vector<CeilingShape> gather_ceiling(const int32_t *ids, int64_t n, int row_bytes, int reps,
                                         int num_sms, const void *table, float *out, cudaStream_t s,
                                         uint64_t &launches)
{
    cudaEvent_t a, b;
    ARE_CUDA_TRY(cudaEventCreate(&a));
    ARE_CUDA_TRY(cudaEventCreate(&b));
    std::vector<CeilingShape> res;
    try {
        if (row_bytes == 32) sweep<32>(ids, n, table, out, reps, num_sms, s, a, b, res, launches);
        else if (row_bytes == 64) sweep<64>(ids, n, table, out, reps, num_sms, s, a, b, res, launches);
        else sweep<128>(ids, n, table, out, reps, num_sms, s, a, b, res, launches);
    } catch (...) {
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        throw;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return res;
}

}  // namespace are
