// screen64.cu -- the FP64 analysis stage with an FP32 screen.
//
// The FP64 table of a layer (8 bytes per event and ELT) is as large as L2 at
// the paper's sizes (1M events x 16 ELTs = 128 MB), so the FP64 staged
// kernel takes about half of its table rows from HBM.  Here each event's row
// is read from an FP32 copy of the table instead (half the bytes: it stays
// in L2), whose entries are the FP64 terms rounded up.  A term is >= 0 and
// rounding up keeps a non-zero term non-zero, so a column is marked when its
// FP32 copy is > 0, exactly where the FP64 term is not 0.  Only the marked
// entries -- a few per cent at the paper's sizes -- are read from the FP64
// table: each lane reads its own in column order (the first two together)
// and adds them, the first taken as is, with an FP64 add only where some
// event of the warp has two or more.  An unmarked column's term is exactly 0
// and adding an exact 0 changes nothing, so the event losses equal the FP64
// staged kernel's (and the oracle's) bit for bit.
#include "staged.cuh"

namespace are {
namespace {

using namespace staged;

template <int JP>
__host__ __device__ constexpr int screen_smem_bytes()
{
    return kWarps * 2 * 32 * JP * 4;   // per warp: two FP32 row buffers
}

template <int JP, bool FIXED>
__global__ void __launch_bounds__(kWarps * 32) k_screen64(const SimArgs a, const TermsF64 tm)
{
    constexpr int CH = JP / 4;   // 16-byte chunks of an FP32 row
    extern __shared__ float4 stage[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float4 *buf0 = stage + (size_t)w * 2 * 32 * CH;
    float4 *buf1 = buf0 + 32 * CH;
    const float *tab = static_cast<const float *>(a.table2);
    const double *t64 = static_cast<const double *>(a.table);
    const int jp64 = a.jp64;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t step = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const double empty_loss = clamp_d(0.0, a.agg_r, a.agg_l);
    Cursor cur{warp, 0, 0};
    if (cur.t < a.n_trials) trial_bounds<FIXED>(a, cur.t, cur.pos, cur.end);

    auto load_ids = [&](const Batch &b) -> int32_t {
        return lane < b.cnt ? __ldcs(a.ids + b.pos + lane) : 0;
    };
    // (a full batch copies every row unconditionally; a partial one
    // zero-fills the rows past its events)
    auto issue_rows = [&](const Batch &b, int32_t idv, float4 *buf) {
        if (b.cnt == 32) {
#pragma unroll
            for (int i = 0; i < CH; ++i) {
                const int q = lane + 32 * i, r = q / CH, c = q % CH;
                const int32_t id = __shfl_sync(kFull, idv, r);
                cp_async16(smem_addr(buf + r * CH + chunk_slot<CH>(c, r)),
                           reinterpret_cast<const float4 *>(tab + (size_t)id * JP) + c, 16);
            }
        } else {
#pragma unroll
            for (int i = 0; i < CH; ++i) {
                const int q = lane + 32 * i, r = q / CH, c = q % CH;
                const int32_t id = __shfl_sync(kFull, idv, r);
                const bool ok = r < b.cnt;
                const float4 *src = ok ? reinterpret_cast<const float4 *>(tab + (size_t)id * JP) + c
                                       : reinterpret_cast<const float4 *>(tab);
                cp_async16(smem_addr(buf + r * CH + chunk_slot<CH>(c, r)), src, ok ? 16 : 0);
            }
        }
        cp_commit();
    };

    SumF64 sum;

    auto compute = [&](const Batch &b, int32_t idv, float4 *buf) {
        // mark the columns that can carry a loss (padding columns hold 0)
        uint32_t mask = 0;
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const float4 v = buf[lane * CH + chunk_slot<CH>(c, lane)];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float x = e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w;
                const int j = c * 4 + e;
                mask |= (uint32_t)(x > 0.f) << j;
            }
        }
        if (lane >= b.cnt) mask = 0;
        // the marked columns' FP64 terms in column order (evict-first: the
        // sparse FP64 reads must not push the screen out of L2), the first
        // two read together, an FP64 add only where an event has two or more
        double g = 0.0;
        const double *row = t64 + (size_t)(uint32_t)idv * jp64;
        uint32_t m = mask;
        const uint32_t m1 = m & (m - 1);
        const int j0 = m ? __ffs(m) - 1 : 0, j1 = m1 ? __ffs(m1) - 1 : 0;
        const double x0 = m ? __ldcs(row + j0) : 0.0, x1 = m1 ? __ldcs(row + j1) : 0.0;
        if (m) g = x0;
        if (__any_sync(kFull, m1 != 0)) {
            if (m1) g = vadd(g, x1);
        }
        m = m1 & (m1 - 1);
        while (__any_sync(kFull, m != 0)) {
            if (m) {
                g = vadd(g, __ldcs(row + __ffs(m) - 1));
                m &= m - 1;
            }
        }
        // occurrence terms and the trial's running sum
        sum.add(occ_clamp(g, tm));
        if (b.last) {
            const double S = warp_sum(sum.s);
            if (lane == 0) a.ylt[b.t] = clamp_d(S, a.agg_r, a.agg_l);
            sum = SumF64{};
        }
    };

    Batch q0 = next_batch<FIXED>(a, cur, step, lane, empty_loss);
    int32_t i0 = load_ids(q0);
    Batch q1 = next_batch<FIXED>(a, cur, step, lane, empty_loss);
    int32_t i1 = load_ids(q1);
    Batch q2 = next_batch<FIXED>(a, cur, step, lane, empty_loss);
    int32_t i2 = load_ids(q2);
    Batch q3;
    int32_t i3 = 0;
    issue_rows(q0, i0, buf0);

#define ARE_SCREEN_STAGE(QC, IC, QN, IN, QF, IF, BC, BN)           \
    if (QC.cnt == 0) break;                                        \
    QF = next_batch<FIXED>(a, cur, step, lane, empty_loss);        \
    IF = load_ids(QF);                                             \
    issue_rows(QN, IN, BN);                                        \
    cp_wait1();                                                    \
    __syncwarp();                                                  \
    compute(QC, IC, BC);                                           \
    __syncwarp();
    while (true) {
        ARE_SCREEN_STAGE(q0, i0, q1, i1, q3, i3, buf0, buf1)
        ARE_SCREEN_STAGE(q1, i1, q2, i2, q0, i0, buf1, buf0)
        ARE_SCREEN_STAGE(q2, i2, q3, i3, q1, i1, buf0, buf1)
        ARE_SCREEN_STAGE(q3, i3, q0, i0, q2, i2, buf1, buf0)
    }
#undef ARE_SCREEN_STAGE
    cp_wait0();
}

template <int JP, bool FIXED>
void launch_screen_t(const SimArgs &a, const TermsF64 &tm, int num_sms, cudaStream_t s)
{
    auto kern = k_screen64<JP, FIXED>;
    constexpr int smem = screen_smem_bytes<JP>();
    const int per_sm = fit_blocks(reinterpret_cast<const void *>(kern), kWarps * 32, smem);
    int64_t blocks = (a.n_trials + kWarps - 1) / kWarps;
    const int64_t cap = (int64_t)num_sms * per_sm;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, kWarps * 32, smem, s>>>(a, tm);
    ARE_CUDA_TRY(cudaGetLastError());
}

template <int JP>
void go(const SimArgs &a, const TermsF64 &t, int num_sms, cudaStream_t s)
{
    if (a.off) launch_screen_t<JP, false>(a, t, num_sms, s);
    else launch_screen_t<JP, true>(a, t, num_sms, s);
}

}  // namespace

// a.table: the FP64 table (a.jp64 columns); a.table2: the FP32 screen
// (jp32 columns, the FP64 values rounded up).
int launch_screen64(const SimArgs &a, int jp32, const TermsF64 &t, int num_sms, cudaStream_t s)
{
    if (a.n_trials <= 0) return 0;
    switch (jp32) {
    case 8: go<8>(a, t, num_sms, s); return 1;
    case 16: go<16>(a, t, num_sms, s); return 1;
    case 32: go<32>(a, t, num_sms, s); return 1;
    }
    throw Error{ARE_EINVAL, "no screened FP64 kernel for table width " + std::to_string(jp32)};
}

}  // namespace are
