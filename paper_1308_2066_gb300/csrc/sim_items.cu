// sim_items.cu -- the analysis stage (Basic Algorithm, Section II-B) for any
// number of layers in one persistent launch (the algorithm's outer loop over
// layers), FP32 table paths.
//
// Work is a list of items (layer, tile of trials), ordered layer by layer so
// the table of one layer at a time is hot in L2 while the YET streams by;
// warps claim items from a device counter until none are left (or take
// every n-th item when no counter is given).  An item's trials run through
// the register-rows core of rows.cuh: each event's table row of terms read
// by jp/8 lanes with one 32-byte load each, the sum over ELTs closed by a
// reduce-scatter across a row's lanes, the occurrence terms and the running
// sum per lane, the aggregate terms for up to 32 trials at once.
#include <cuda_runtime.h>

#include <string>

#include "are_internal.cuh"
#include "rows.cuh"

namespace are {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// Blocks per SM the register budget is set for (as the single-layer kernel).
__host__ __device__ constexpr int items_min_blocks(int jp, int u)
{
    return jp * u <= 16 ? 5 : jp * u <= 32 ? 4 : 2;
}

template <int JP, int U, int ACC, bool FIXED>
__global__ void __launch_bounds__(256, items_min_blocks(JP, U)) k_sim_items(const __grid_constant__ ItemWork w)
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
        rows::Trials a;
        a.ids = w.ids;
        a.off = w.off;
        a.k = w.k;
        a.trial_begin = w.trial_begin;
        a.ylt = L.ylt;
        a.agg_r = L.agg_r;
        a.agg_l = L.agg_l;
        rows::BodyF32<JP, U, ACC> body;
        body.table = L.table;
        body.occ_r = L.occ_r;
        body.occ_l = L.occ_l;
        rows::run_trials<U, FIXED>(a, body, t0, t1, lane);
    }
}

template <int JP, int U, int ACC, bool FIXED>
void launch_items_t(const ItemWork &w, int blocks_per_sm, int num_sms, cudaStream_t s)
{
    const int per_sm = fit_blocks(reinterpret_cast<const void *>(k_sim_items<JP, U, ACC, FIXED>), 256, 0);
    if (blocks_per_sm <= 0 || blocks_per_sm > per_sm) blocks_per_sm = per_sm;
    int64_t blocks = (int64_t)num_sms * blocks_per_sm;
    const int64_t need = (w.n_items + 7) / 8;
    if (blocks > need) blocks = need < 1 ? 1 : need;
    k_sim_items<JP, U, ACC, FIXED><<<(unsigned)blocks, 256, 0, s>>>(w);
    ARE_CUDA_TRY(cudaGetLastError());
}

// cfg.rows_in_flight: groups of 32 events per batch (1 or 2)
template <int JP, int ACC, bool FIXED>
void launch_jp(const ItemWork &w, const ItemConfig &cfg, int num_sms, cudaStream_t s)
{
    if (cfg.rows_in_flight == 1)
        launch_items_t<JP, 1, ACC, FIXED>(w, cfg.blocks_per_sm, num_sms, s);
    else
        launch_items_t<JP, 2, ACC, FIXED>(w, cfg.blocks_per_sm, num_sms, s);
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
