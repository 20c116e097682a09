// rows64.cu -- the FP64 analysis stage (Basic Algorithm, Section II-B) for
// one layer, with the table rows held in registers (rows.cuh, BodyP64).
//
// The FP64 terms are read from the layer's packed FP64 table: one 32- or
// 64-byte row per catalog event holding the mask of the ELTs whose term is
// not 0 and up to 3 or 7 of those terms in column order (a longer row's
// terms are all in an overflow array).  At the paper's sizes a dense FP64 row (8 bytes per
// ELT: 128 MB at 1M events x 16 ELTs, the size of L2) would come half from
// HBM, and a non-zero term is a few per cent of the entries.  Every
// occurrence reads its event's whole row; the terms are added in column
// order as the oracle adds them, so every event loss and occurrence loss is
// the oracle's bit for bit.  The trial's running sum is exact (fixed-point
// integers, fixed.cuh) and rounded to double once: within the rounding of
// the oracle's own sequential sum of it, and with no FP64 instruction per
// occurrence beyond the few events with two or more non-zero terms or a
// loss above the occurrence retention.
#include <cuda_runtime.h>

#include <string>

#include "are_internal.cuh"
#include "rows.cuh"

namespace are {
namespace {

// Blocks per SM the register budget is set for: the most that leave at most
// a word of spill for RW * U words per lane in flight (a ragged YET's cursor
// needs a few registers more).
__host__ __device__ constexpr int rows64_min_blocks(int rw, int u, bool fixed)
{
    return !fixed ? (rw * u <= 4 ? 5 : rw * u <= 8 ? 4 : rw * u <= 16 ? 3 : 2)
                  : rw == 4 ? (u == 1 ? 6 : 5) : rw * u <= 8 ? 4 : rw * u <= 16 ? 3 : 2;
}

template <int RW, int U, bool FIXED>
__global__ void __launch_bounds__(256, rows64_min_blocks(RW, U, FIXED))
    k_rows64(const rows::Trials a, const rows::BodyP64<RW, U> body, const int64_t n_trials)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    rows::run_trials<U, FIXED>(a, body, warp * n_trials / nw, (warp + 1) * n_trials / nw, lane);
}

template <int RW, int U, bool FIXED>
void launch_t(const SimArgs &a, const TermsF64 &tm, int scale, int num_sms, cudaStream_t s)
{
    auto kern = k_rows64<RW, U, FIXED>;
    const int per_sm = fit_blocks(reinterpret_cast<const void *>(kern), 256, 0);
    int64_t blocks = (a.n_trials + 7) / 8;
    const int64_t cap = (int64_t)num_sms * per_sm;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    rows::Trials t;
    t.ids = a.ids;
    t.off = a.off;
    t.k = a.k;
    t.trial_begin = a.trial_begin;
    t.ylt = a.ylt;
    t.agg_r = a.agg_r;
    t.agg_l = a.agg_l;
    rows::BodyP64<RW, U> body;
    body.rows = static_cast<const unsigned long long *>(a.table);
    body.ovf = static_cast<const double *>(a.table2);
    body.scale = scale;
    body.occ_r = tm.occ_r;
    body.occ_l = tm.occ_l;
    kern<<<(unsigned)blocks, 256, 0, s>>>(t, body, a.n_trials);
    ARE_CUDA_TRY(cudaGetLastError());
}

template <int RW>
void go(const SimArgs &a, const TermsF64 &tm, int scale, int num_sms, cudaStream_t s)
{
    const bool two = a.epl != 1;
    if (a.off)
        two ? launch_t<RW, 2, false>(a, tm, scale, num_sms, s) : launch_t<RW, 1, false>(a, tm, scale, num_sms, s);
    else
        two ? launch_t<RW, 2, true>(a, tm, scale, num_sms, s) : launch_t<RW, 1, true>(a, tm, scale, num_sms, s);
}

}  // namespace

// a.table: the packed FP64 table (row_words 64-bit words per row); a.table2:
// its overflow terms; a.epl: groups of 32 events per batch.
int launch_rows64(const SimArgs &a, int row_words, const TermsF64 &t, int scale, int num_sms, cudaStream_t s)
{
    if (a.n_trials <= 0) return 0;
    if (row_words == 4) {
        go<4>(a, t, scale, num_sms, s);
        return 1;
    }
    if (row_words == 8) {
        go<8>(a, t, scale, num_sms, s);
        return 1;
    }
    throw Error{ARE_EINVAL, "no FP64 register-rows kernel for packed rows of " + std::to_string(row_words) +
                                " words"};
}

}  // namespace are
