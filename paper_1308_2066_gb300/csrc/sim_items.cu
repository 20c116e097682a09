// sim_items.cu -- the analysis stage (Basic Algorithm, Section II-B) for any
// number of layers in one persistent launch (the algorithm's outer loop over
// layers), FP32 table paths.
//
// Work is a list of items (layer, tile of trials), ordered layer by layer so
// the table of one layer at a time is hot in L2 while the YET streams by;
// warps claim items from a device counter until none are left.  Inside an
// item a warp walks its trials in steps of B = (32/R)*U events: the table row
// of an event (jp floats, jp/4 16-byte chunks) is read by R = jp/4 lanes with
// one 16-byte load each, every lane holding U rows in flight.  Each lane
// applies the financial terms of its 4 columns (step 2); a reduce-scatter
// across the R lanes of a row sums the ELTs (end of step 2) and leaves each lane
// with whole events, whose occurrence terms (step 3) and compensated running
// sum (step 4) it then does alone.  At the end of a trial the warp adds its
// lanes' sums and applies the aggregate terms.
#include <cuda_runtime.h>

#include <cstdlib>
#include <type_traits>

#include "are_internal.cuh"

namespace are {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = __dadd_rn(v, __shfl_xor_sync(kFull, v, off));
    return v;
}

__device__ __forceinline__ double clamp_d(double v, double r, double l)
{
    double a = v - r;
    a = a > 0.0 ? a : 0.0;
    return a < l ? a : l;
}

// Exact float -> double for finite x >= 0 on the integer pipes (the FP64
// pipe is the scarce unit on this chip); subnormal inputs take the FP64
// conversion in a warp-uniform branch.
__device__ __forceinline__ double widen(float x)
{
    const uint32_t u = __float_as_uint(x);
    double d = __longlong_as_double(u ? (long long)(((unsigned long long)u << 29) +
                                                    (896ull << 52))
                                      : 0ll);
    const bool sub = u != 0 && u < 0x00800000u;
    if (__any_sync(kFull, sub)) {
        double c;
        asm volatile("cvt.f64.f32 %0, %1;" : "=d"(c) : "f"(x));
        if (sub) d = c;
    }
    return d;
}

struct AccKahan {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float o)
    {
        const float y = __fsub_rn(o, c);
        const float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
    __device__ __forceinline__ double total() const { return (double)s - (double)c; }
};
struct AccF64 {
    double s = 0.0;
    __device__ __forceinline__ void add(float o)
    {
        double r;
        asm volatile("add.rn.f64 %0, %1, %2;" : "=d"(r) : "d"(s), "d"(widen(o)));
        s = r;
    }
    __device__ __forceinline__ double total() const { return s; }
};

template <bool FIXED>
__device__ __forceinline__ void bounds(const ItemWork &w, int64_t t, int64_t &b, int64_t &e)
{
    const int64_t tt = w.trial_begin + t;
    if (FIXED) {
        b = tt * (int64_t)w.k;
        e = b + w.k;
    } else {
        b = w.off[tt];
        e = w.off[tt + 1];
    }
}

// Runs the trials [t0, t1) of one layer.  JP = table columns; U = rows per
// lane in flight.
template <int JP, int U, int ACC, bool FIXED>
__device__ __forceinline__ void run_item(const ItemWork &w, const LayerF32 &L, int64_t t0,
                                         int64_t t1, int lane)
{
    constexpr int R = JP / 4;       // lanes per row
    constexpr int RPW = 32 / R;     // rows per warp load
    constexpr int B = RPW * U;      // events per step
    constexpr int KEEP = U / R;     // events each lane finishes per step
    static_assert(U % R == 0 && (R & (R - 1)) == 0, "U must be a multiple of R, R a power of 2");
    const int row = lane / R, col = lane % R;

    float lim[4], shr[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        lim[c] = L.lim[col * 4 + c];
        shr[c] = L.share[col * 4 + c];
    }
    const float occ_r = L.occ_r, occ_l = L.occ_l;
    const bool any_share = L.any_share != 0;
    const float4 *tab = reinterpret_cast<const float4 *>(L.table);
    typename std::conditional<ACC == ARE_FP32_KAHAN, AccKahan, AccF64>::type acc;
    const double empty_loss = clamp_d(0.0, L.agg_r, L.agg_l);

    // cursor over the item's trials, in steps of B events
    int64_t t = t0, pos = 0, end = 0;
    if (t < t1) bounds<FIXED>(w, t, pos, end);
    auto skip_empty = [&] {
        while (t < t1 && pos >= end) {
            if (lane == 0) L.ylt[t] = empty_loss;
            ++t;
            if (t < t1) bounds<FIXED>(w, t, pos, end);
        }
    };
    skip_empty();
    auto load_ids = [&](int32_t (&id)[U], int64_t p, int64_t e) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t ev = p + u * RPW + row;
            id[u] = ev < e ? __ldcs(w.ids + ev) : -1;
        }
    };
    int32_t nid[U];
    if (t < t1) load_ids(nid, pos, end);

    while (t < t1) {
        int32_t id[U];
#pragma unroll
        for (int u = 0; u < U; ++u) id[u] = nid[u];
        const int64_t cur_t = t;
        pos += B;
        const bool last = pos >= end;
        if (last) {
            ++t;
            if (t < t1) bounds<FIXED>(w, t, pos, end);
            skip_empty();
        }
        float4 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
            v[u] = id[u] >= 0 ? __ldg(tab + (size_t)id[u] * R + col) : make_float4(0.f, 0.f, 0.f, 0.f);
        if (t < t1) load_ids(nid, pos, end);

        // step 2 for this lane's 4 columns of each row in flight (the table
        // holds each loss's excess over the deductible)
        float part[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            float n0 = fminf(fmaxf(v[u].x, 0.f), lim[0]);
            float n1 = fminf(fmaxf(v[u].y, 0.f), lim[1]);
            float n2 = fminf(fmaxf(v[u].z, 0.f), lim[2]);
            float n3 = fminf(fmaxf(v[u].w, 0.f), lim[3]);
            if (any_share) {
                n0 = __fmul_rn(n0, shr[0]);
                n1 = __fmul_rn(n1, shr[1]);
                n2 = __fmul_rn(n2, shr[2]);
                n3 = __fmul_rn(n3, shr[3]);
            }
            part[u] = __fadd_rn(__fadd_rn(n0, n1), __fadd_rn(n2, n3));
        }
        // reduce-scatter over the R lanes of a row: each lane keeps KEEP
        // whole-row sums (slots col*KEEP .. col*KEEP + KEEP - 1)
#pragma unroll
        for (int m = R / 2, half = U / 2; m >= 1; m >>= 1, half >>= 1) {
            const bool up = (col & m) != 0;
#pragma unroll
            for (int i = 0; i < half; ++i) {
                const float send = up ? part[i] : part[i + half];
                const float keep = up ? part[i + half] : part[i];
                part[i] = __fadd_rn(keep, __shfl_xor_sync(kFull, send, m));
            }
        }
        // steps 3-4 for this lane's events
#pragma unroll
        for (int i = 0; i < KEEP; ++i) acc.add(fminf(fmaxf(__fsub_rn(part[i], occ_r), 0.f), occ_l));
        if (last) {
            const double S = warp_sum(acc.total());
            if (lane == 0) L.ylt[cur_t] = clamp_d(S, L.agg_r, L.agg_l);
            acc = decltype(acc){};
        }
    }
}

template <int JP, int U, int ACC, bool FIXED>
__global__ void __launch_bounds__(256) k_sim_items(const __grid_constant__ ItemWork w)
{
    const int lane = threadIdx.x & 31;
    const unsigned long long warp = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned long long n_warps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
    for (unsigned long long k = 0;; ++k) {
        unsigned long long item = warp + k * n_warps;   // static split without a counter
        if (w.counter) {
            if (lane == 0) item = atomicAdd(w.counter, 1ull);
            item = __shfl_sync(kFull, item, 0);
        }
        if (item >= (unsigned long long)w.n_items) break;
        // layer of the item: last layer whose first item is <= item
        int lo = 0;
        if (w.layers) {
            int hi = w.n_layers - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if ((unsigned long long)w.layers[mid].item_begin <= item) lo = mid;
                else hi = mid - 1;
            }
        }
        const LayerF32 &L = w.layers ? w.layers[lo] : w.one;
        const int64_t t0 = L.t0 + (int64_t)(item - L.item_begin) * w.trials_per_item;
        int64_t t1 = t0 + w.trials_per_item;
        if (t1 > L.t0 + L.nt) t1 = L.t0 + L.nt;
        run_item<JP, U, ACC, FIXED>(w, L, t0, t1, lane);
    }
}

// U per row width: U must be a multiple of the lanes per row (jp/4).
template <int JP>
constexpr int u_for(int u)
{
    return JP == 32 ? 8 : (u == 4 ? 4 : 8);
}

template <int JP, int U, int ACC, bool FIXED>
const void *kernel_ptr()
{
    return reinterpret_cast<const void *>(k_sim_items<JP, U, ACC, FIXED>);
}

template <int JP, int U, int ACC, bool FIXED>
int max_blocks_t()
{
    return fit_blocks(kernel_ptr<JP, U, ACC, FIXED>(), 256, 0);
}

template <int JP, int U, int ACC, bool FIXED>
void launch_items_t(const ItemWork &w, int blocks_per_sm, int num_sms, cudaStream_t s)
{
    const int per_sm = max_blocks_t<JP, U, ACC, FIXED>();
    if (blocks_per_sm <= 0 || blocks_per_sm > per_sm) blocks_per_sm = per_sm;
    int64_t blocks = (int64_t)num_sms * blocks_per_sm;
    const int64_t need = (w.n_items + 7) / 8;
    if (blocks > need) blocks = need < 1 ? 1 : need;
    k_sim_items<JP, U, ACC, FIXED><<<(unsigned)blocks, 256, 0, s>>>(w);
    ARE_CUDA_TRY(cudaGetLastError());
}

template <int JP, int ACC, bool FIXED>
void launch_jp(const ItemWork &w, const ItemConfig &cfg, int num_sms, cudaStream_t s)
{
    if (u_for<JP>(cfg.rows_in_flight) == 4)
        launch_items_t<JP, (JP == 32 ? 8 : 4), ACC, FIXED>(w, cfg.blocks_per_sm, num_sms, s);
    else
        launch_items_t<JP, 8, ACC, FIXED>(w, cfg.blocks_per_sm, num_sms, s);
}

template <int ACC, bool FIXED>
void launch_acc(const ItemWork &w, int jp, const ItemConfig &cfg, int num_sms, cudaStream_t s)
{
    switch (jp) {
    case 8: return launch_jp<8, ACC, FIXED>(w, cfg, num_sms, s);
    case 16: return launch_jp<16, ACC, FIXED>(w, cfg, num_sms, s);
    case 32: return launch_jp<32, ACC, FIXED>(w, cfg, num_sms, s);
    }
    throw Error{ARE_EINVAL, "no persistent kernel for table width " + std::to_string(jp)};
}

}  // namespace

int launch_items(const ItemWork &w, int jp, const ItemConfig &cfg, are_precision prec,
                 int num_sms, cudaStream_t s)
{
    ARE_CHECK(prec == ARE_FP32_KAHAN || prec == ARE_FP32_FP64AGG, ARE_EINVAL,
              "the persistent item kernel runs the FP32 table paths");
    const bool fixed = w.off == nullptr;
    if (prec == ARE_FP32_KAHAN)
        fixed ? launch_acc<ARE_FP32_KAHAN, true>(w, jp, cfg, num_sms, s)
              : launch_acc<ARE_FP32_KAHAN, false>(w, jp, cfg, num_sms, s);
    else
        fixed ? launch_acc<ARE_FP32_FP64AGG, true>(w, jp, cfg, num_sms, s)
              : launch_acc<ARE_FP32_FP64AGG, false>(w, jp, cfg, num_sms, s);
    return 1;
}

}  // namespace are
