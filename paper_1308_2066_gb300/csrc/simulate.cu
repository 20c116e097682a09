// simulate.cu -- the analysis stage (Basic Algorithm, Section II-B) for one
// layer over a range of trials with an FP32 layer table (each entry an
// event's financial term in one ELT, built by repack.cu).  Two kernels:
//
//  * k_rows (the default): rows held in registers, see rows.cuh; over packed
//    rows (k_rows_packed) where a layer of more than 8 ELTs holds few entries
//    per catalog event.
//  * k_simulate_staged (a tuning candidate, and the compact layout's
//    kernel): one event per lane, rows staged in shared memory.
//
// The trial loss is the aggregate-clamped total: with non-negative
// occurrence losses the de-cumulated marginals of step 4 telescope to it, so
// the YLT needs no per-event scan.
#include <cuda_runtime.h>

#include <string>
#include <type_traits>

#include "are_internal.cuh"
#include "rows.cuh"

namespace are {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// Two FP32 additions in one packed instruction (sm_100 and later), used by
// the FP32 + Kahan staged kernel.
__device__ __forceinline__ float2 add2(float2 a, float2 b)
{
    unsigned long long ra, rb, rd;
    asm("mov.b64 %0, {%1, %2};" : "=l"(ra) : "f"(a.x), "f"(a.y));
    asm("mov.b64 %0, {%1, %2};" : "=l"(rb) : "f"(b.x), "f"(b.y));
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
    float2 d;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(d.x), "=f"(d.y) : "l"(rd));
    return d;
}

// FP64 add that the compiler may not hoist out of the warp-uniform branch
// below (every FP64 instruction is expensive on this chip).
__device__ __forceinline__ double vadd(double a, double b)
{
    double r;
    asm volatile("add.rn.f64 %0, %1, %2;" : "=d"(r) : "d"(a), "d"(b));
    return r;
}

// Per-lane running sums of occurrence losses (step 4) for the staged FP32
// kernel, one flavour per precision mode.
struct AccKahan {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float o)
    {
        const float y = __fsub_rn(o, c);
        const float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
    // s - c exactly in double: c is within a few ulps of s's last bit
    __device__ __forceinline__ double total() const { return (double)s - (double)c; }
};
struct AccF32F64 {
    double s = 0.0;
    __device__ __forceinline__ void add(float o)
    {
        const bool need = o != 0.f;
        if (__any_sync(kFull, need)) {
            const double t = vadd(s, (double)o);
            if (need) s = t;
        }
    }
    __device__ __forceinline__ double total() const { return s; }
};

__device__ __forceinline__ double warp_total(double v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = __dadd_rn(v, __shfl_xor_sync(kFull, v, off));
    return v;
}

__device__ __forceinline__ double net_d(double v, double r, double l)
{
    double a = v - r;
    a = a > 0.0 ? a : 0.0;
    return a < l ? a : l;
}

// ---------------------------------------------------------------------------
// FP32 paths, staged: one event per lane.
//
// A warp takes its trials in batches of up to 32 events (a batch never spans
// two trials).  The 32 table rows of a batch are copied global -> shared with
// cp.async in a coalesced pattern (the lanes of one copy instruction cover
// 32/CH whole rows, so each row costs one L1 wavefront), then every lane
// reads its own event's row from shared memory and does all of the event's
// arithmetic: the sum over ELTs of the row's terms, the
// occurrence terms and the compensated running sum.  Row chunks are rotated
// per row so the lanes' 16-byte shared reads hit distinct banks.  Event ids
// are loaded three batches ahead and rows one batch ahead (double buffer).
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, int src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
                 "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Physical slot of 16-byte chunk c of row r (CH chunks per row): a rotation
// that gives the 8 lanes of each shared-memory phase 8 distinct bank groups.
template <int CH>
__device__ __forceinline__ int chunk_slot(int c, int r)
{
    const int rot = CH == 2 ? (r >> 2) & 1 : CH == 4 ? (r >> 1) & 3 : CH == 6 ? (r >> 2) & 1 : r & 7;
    const int p = c + rot;
    return p >= CH ? p - CH : p;
}

// A batch in the pipeline: its trial (index into the launch's range) and a
// packed count of events (bits 0-6, 0 = no more work) and last-of-trial flag
// (bit 7).  Kept small: four of them live in registers.
struct Batch {
    int32_t t = -1;
    int32_t info = 0;
    __device__ __forceinline__ int cnt() const { return info & 127; }
    __device__ __forceinline__ bool last() const { return (info & 128) != 0; }
};

// Where a warp is in its trials: current trial, its next event and the
// number of its events not yet handed out.
struct Cursor {
    int32_t t;
    int32_t rem;
    int64_t pos;
};

template <bool FIXED>
__device__ __forceinline__ void trial_start(const SimArgs &a, Cursor &c)
{
    const int64_t tt = a.trial_begin + c.t;
    if (FIXED) {
        c.pos = tt * (int64_t)a.k;
        c.rem = a.k;
    } else {
        c.pos = a.off[tt];
        c.rem = (int32_t)(a.off[tt + 1] - c.pos);
    }
}

// The warp's next batch of up to BS events of one trial (its first event in
// *pos); trials without events get their loss written here.
template <bool FIXED, int BS>
__device__ __forceinline__ Batch next_batch(const SimArgs &a, Cursor &c, int32_t step, int lane,
                                            double empty_loss, int64_t &pos)
{
    Batch b;
    while (c.t < a.n_trials) {
        if (c.rem > 0) {
            b.t = c.t;
            pos = c.pos;
            b.info = c.rem < BS ? c.rem : BS;
            c.pos += BS;
            c.rem -= BS;
            if (c.rem <= 0) {
                b.info |= 128;
                c.t += step;
                if (c.t < a.n_trials) trial_start<FIXED>(a, c);
            }
            return b;
        }
        if (lane == 0) a.ylt[c.t] = empty_loss;
        c.t += step;
        if (c.t < a.n_trials) trial_start<FIXED>(a, c);
    }
    return b;
}

constexpr int kStagedWarps = 8;

template <int JP, int EPL>
constexpr int staged_smem_bytes()
{
    return kStagedWarps * 2 * 32 * EPL * JP * 4;
}

template <int EPL>
struct Ids {
    int32_t v[EPL];
};

// EPL = events per lane in a batch (a batch is 32 * EPL events of a trial).
// CMP: compact table -- each id is turned into its row (a.table2) one stage
// before the row is copied, and an event without a row reads as zeros.
template <int JP, int ACC, bool FIXED, int EPL, bool CMP = false>
__global__ void __launch_bounds__(kStagedWarps * 32)
    k_simulate_staged(const SimArgs a, const TermsF32 tm)
{
    constexpr int CH = JP / 4;              // 16-byte chunks per row
    constexpr int ROWS = 32 * EPL;          // rows per batch
    constexpr int NC = CH * EPL;            // row chunks each lane copies per batch
    extern __shared__ float4 stage[];
    const int lane = threadIdx.x & 31;
    float4 *buf0 = stage + (size_t)(threadIdx.x >> 5) * 2 * ROWS * CH;
    float4 *buf1 = buf0 + ROWS * CH;
    const uint32_t sbuf0 = smem_addr(buf0), sbuf1 = smem_addr(buf1);
    const char *tab = static_cast<const char *>(a.table);

    const int32_t warp = (int32_t)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int32_t step = (int32_t)((gridDim.x * blockDim.x) >> 5);
    const double empty_loss = net_d(0.0, a.agg_r, a.agg_l);
    Cursor cur{warp, 0, 0};
    if (cur.t < a.n_trials) trial_start<FIXED>(a, cur);

    auto load_ids = [&](const Batch &b, int64_t pos) {
        Ids<EPL> r;
#pragma unroll
        for (int e = 0; e < EPL; ++e)
            r.v[e] = 32 * e + lane < b.cnt() ? __ldcs(a.ids + pos + 32 * e + lane) : 0;
        return r;
    };
    // copy i of a lane moves chunk (lane + 32 i) % CH of row (lane + 32 i) / CH
    // (a full batch of a direct table copies every row unconditionally; the
    // other batches zero-fill the rows past their events and, with compact
    // tables, the rows of events that have none)
    auto issue_rows = [&](const Batch &b, const Ids<EPL> &idv, uint32_t sbuf) {
        if (!CMP && b.cnt() == ROWS) {
#pragma unroll
            for (int i = 0; i < NC; ++i) {
                const int q = lane + 32 * i, r = q / CH, c = q % CH;
                const int32_t id = __shfl_sync(kFull, idv.v[i / CH], r & 31);
                cp_async16(sbuf + (uint32_t)(r * CH + chunk_slot<CH>(c, r)) * 16u,
                           tab + (size_t)(uint32_t)id * (JP * 4) + c * 16, 16);
            }
        } else {
#pragma unroll
            for (int i = 0; i < NC; ++i) {
                const int q = lane + 32 * i, r = q / CH, c = q % CH;
                const int32_t id = __shfl_sync(kFull, idv.v[i / CH], r & 31);
                const bool ok = r < b.cnt() && (!CMP || id >= 0);
                const char *src = tab + (ok ? (size_t)(uint32_t)id * (JP * 4) + c * 16 : 0);
                cp_async16(sbuf + (uint32_t)(r * CH + chunk_slot<CH>(c, r)) * 16u, src, ok ? 16 : 0);
            }
        }
        cp_commit();
    };
    auto to_rows = [&](Ids<EPL> &v) {
        if (CMP) {
#pragma unroll
            for (int e = 0; e < EPL; ++e) v.v[e] = __ldg(static_cast<const int32_t *>(a.table2) + v.v[e]);
        }
    };

    typename std::conditional<ACC == ARE_FP32_KAHAN, AccKahan, AccF32F64>::type acc;
    auto compute = [&](const Batch &b, const float4 *buf) {
#pragma unroll
        for (int e = 0; e < EPL; ++e) {
            const int r = lane + 32 * e;
            // the sum over ELTs of the row's terms in packed FP32x2 pairs:
            // partial sums over the columns j mod 4, added at the end
            float2 g01 = make_float2(0.f, 0.f), g23 = make_float2(0.f, 0.f);
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const float4 v = buf[r * CH + chunk_slot<CH>(c, r)];
                g01 = add2(g01, make_float2(v.x, v.y));
                g23 = add2(g23, make_float2(v.z, v.w));
            }
            const float g = __fadd_rn(__fadd_rn(g01.x, g01.y), __fadd_rn(g23.x, g23.y));
            acc.add(fminf(fmaxf(__fsub_rn(g, tm.occ_r), 0.f), tm.occ_l));
        }
        if (b.last()) {
            const double S = warp_total(acc.total());
            if (lane == 0) a.ylt[b.t] = net_d(S, a.agg_r, a.agg_l);
            acc = decltype(acc){};
        }
    };

    int64_t pos = 0;
    Batch q0 = next_batch<FIXED, ROWS>(a, cur, step, lane, empty_loss, pos);
    Ids<EPL> i0 = load_ids(q0, pos);
    Batch q1 = next_batch<FIXED, ROWS>(a, cur, step, lane, empty_loss, pos);
    Ids<EPL> i1 = load_ids(q1, pos);
    Batch q2 = next_batch<FIXED, ROWS>(a, cur, step, lane, empty_loss, pos);
    Ids<EPL> i2 = load_ids(q2, pos);
    Batch q3;
    Ids<EPL> i3{};
    to_rows(i0);
    to_rows(i1);
    issue_rows(q0, i0, sbuf0);

    // Each stage: ids three batches ahead, (compact tables) rows of the ids
    // two batches ahead, row copies one batch ahead, compute.
#define ARE_STAGE(QC, QN, IN, IT, QF, IF, BC, BN, SN)                     \
    if (QC.cnt() == 0) break;                                             \
    QF = next_batch<FIXED, ROWS>(a, cur, step, lane, empty_loss, pos);    \
    IF = load_ids(QF, pos);                                               \
    to_rows(IT);                                                          \
    issue_rows(QN, IN, SN);                                               \
    cp_wait1();                                                           \
    __syncwarp();                                                         \
    compute(QC, BC);                                                      \
    __syncwarp();
    while (true) {
        ARE_STAGE(q0, q1, i1, i2, q3, i3, buf0, buf1, sbuf1)
        ARE_STAGE(q1, q2, i2, i3, q0, i0, buf1, buf0, sbuf0)
        ARE_STAGE(q2, q3, i3, i0, q1, i1, buf0, buf1, sbuf1)
        ARE_STAGE(q3, q0, i0, i1, q2, i2, buf1, buf0, sbuf0)
    }
#undef ARE_STAGE
    cp_wait0();
}

template <int JP, int ACC, bool FIXED, int EPL, bool CMP = false>
void launch_staged(const SimArgs &a, const TermsF32 &terms, int num_sms, cudaStream_t s)
{
    auto kern = k_simulate_staged<JP, ACC, FIXED, EPL, CMP>;
    constexpr int smem = staged_smem_bytes<JP, EPL>();
    const int per_sm = fit_blocks(reinterpret_cast<const void *>(kern), kStagedWarps * 32, smem);
    int64_t blocks = (a.n_trials + kStagedWarps - 1) / kStagedWarps;
    const int64_t cap = (int64_t)num_sms * per_sm;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, kStagedWarps * 32, smem, s>>>(a, terms);
    ARE_CUDA_TRY(cudaGetLastError());
}

template <int JP, int ACC>
void launch_staged_fx(const SimArgs &a, const TermsF32 &terms, int num_sms, cudaStream_t s)
{
    if (a.kernel == 4) {   // compact table: two events per lane with Kahan sums, one with FP64 sums
        constexpr int E = ACC == ARE_FP32_KAHAN ? 2 : 1;
        if (a.off) launch_staged<JP, ACC, false, E, true>(a, terms, num_sms, s);
        else launch_staged<JP, ACC, true, E, true>(a, terms, num_sms, s);
        return;
    }
    const bool two = a.epl == 2;
    if (a.off)
        two ? launch_staged<JP, ACC, false, 2>(a, terms, num_sms, s)
            : launch_staged<JP, ACC, false, 1>(a, terms, num_sms, s);
    else
        two ? launch_staged<JP, ACC, true, 2>(a, terms, num_sms, s)
            : launch_staged<JP, ACC, true, 1>(a, terms, num_sms, s);
}

// ---------------------------------------------------------------------------
// FP32 paths, rows in registers (rows.cuh): a warp takes a contiguous block
// of the launch's trials.
// ---------------------------------------------------------------------------

// Blocks per SM the register budget is set for: the row pieces in flight
// (JP * U floats per lane) decide it.  One 32-byte piece per lane runs best
// at 6 blocks (40 registers, no spill): 7 or 8 blocks force 32 registers and
// a slower loop, 5 leave fewer rows in flight.
__host__ __device__ constexpr int rows_min_blocks(int jp, int u)
{
    return jp * u <= 8 ? 6 : jp * u <= 16 ? 5 : jp * u <= 32 ? 4 : 2;
}

template <int JP, int U, int ACC, bool FIXED>
__global__ void __launch_bounds__(256, rows_min_blocks(JP, U))
    k_rows(const rows::Trials a, const rows::BodyF32<JP, U, ACC> body, const int64_t n_trials)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    rows::run_trials<U, FIXED>(a, body, warp * n_trials / nw, (warp + 1) * n_trials / nw, lane);
}

template <int JP, int U, int ACC, bool FIXED>
void launch_rows_t(const SimArgs &a, const TermsF32 &tm, int num_sms, cudaStream_t s)
{
    auto kern = k_rows<JP, U, ACC, FIXED>;
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
    rows::BodyF32<JP, U, ACC> body;
    body.table = static_cast<const float *>(a.table);
    body.occ_r = tm.occ_r;
    body.occ_l = tm.occ_l;
    kern<<<(unsigned)blocks, 256, 0, s>>>(t, body, a.n_trials);
    ARE_CUDA_TRY(cudaGetLastError());
}

// Packed FP32 rows of PW words (8 or 16): a.table the rows, a.table2 the
// overflow terms.
template <int PW, int U, int ACC, bool FIXED>
__global__ void __launch_bounds__(256, rows_min_blocks(PW, U))
    k_rows_packed(const rows::Trials a, const rows::BodyPackedF32<PW, U, ACC> body, const int64_t n_trials)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    rows::run_trials<U, FIXED>(a, body, warp * n_trials / nw, (warp + 1) * n_trials / nw, lane);
}

template <int PW, int U, int ACC, bool FIXED>
void launch_packed_t(const SimArgs &a, const TermsF32 &tm, int num_sms, cudaStream_t s)
{
    auto kern = k_rows_packed<PW, U, ACC, FIXED>;
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
    rows::BodyPackedF32<PW, U, ACC> body;
    body.rows = static_cast<const float *>(a.table);
    body.ovf = static_cast<const float *>(a.table2);
    body.occ_r = tm.occ_r;
    body.occ_l = tm.occ_l;
    kern<<<(unsigned)blocks, 256, 0, s>>>(t, body, a.n_trials);
    ARE_CUDA_TRY(cudaGetLastError());
}

template <int PW, int ACC>
void launch_packed(const SimArgs &a, const TermsF32 &tm, int num_sms, cudaStream_t s)
{
    const bool two = a.epl == 0 ? PW > 8 : a.epl != 1;
    if (a.off)
        two ? launch_packed_t<PW, 2, ACC, false>(a, tm, num_sms, s)
            : launch_packed_t<PW, 1, ACC, false>(a, tm, num_sms, s);
    else
        two ? launch_packed_t<PW, 2, ACC, true>(a, tm, num_sms, s)
            : launch_packed_t<PW, 1, ACC, true>(a, tm, num_sms, s);
}

template <int JP, int ACC>
void launch_rows(const SimArgs &a, const TermsF32 &tm, int num_sms, cudaStream_t s)
{
    const bool two = a.epl == 0 ? JP > 8 : a.epl != 1;
    if (a.off)
        two ? launch_rows_t<JP, 2, ACC, false>(a, tm, num_sms, s)
            : launch_rows_t<JP, 1, ACC, false>(a, tm, num_sms, s);
    else
        two ? launch_rows_t<JP, 2, ACC, true>(a, tm, num_sms, s)
            : launch_rows_t<JP, 1, ACC, true>(a, tm, num_sms, s);
}

template <int ACC>
int launch_fp32(const SimArgs &a, int jp, const TermsF32 &tm, int num_sms, cudaStream_t s)
{
    if (a.kernel == 5) {   // register rows over packed FP32 rows of jp words
        if (jp == 8) launch_packed<8, ACC>(a, tm, num_sms, s);
        else if (jp == 16) launch_packed<16, ACC>(a, tm, num_sms, s);
        else throw Error{ARE_EINVAL, "packed FP32 rows are 8 or 16 words"};
        return 1;
    }
    const bool staged = a.kernel == 1 || a.kernel == 4;   // 4: the compact table's rows
    switch (jp) {
    case 8: staged ? launch_staged_fx<8, ACC>(a, tm, num_sms, s) : launch_rows<8, ACC>(a, tm, num_sms, s); return 1;
    case 16: staged ? launch_staged_fx<16, ACC>(a, tm, num_sms, s) : launch_rows<16, ACC>(a, tm, num_sms, s); return 1;
    case 32: staged ? launch_staged_fx<32, ACC>(a, tm, num_sms, s) : launch_rows<32, ACC>(a, tm, num_sms, s); return 1;
    }
    throw Error{ARE_EINVAL, "no FP32 simulate kernel for table width " + std::to_string(jp)};
}

}  // namespace

// FP32: the register-rows kernel unless a.kernel names the staged one (1,
// or 4 for the compact layout) or the packed rows (5).  (FP64 analyses run
// in staged64.cu, screen64.cu and rows64.cu.)
int launch_simulate(const SimArgs &a, are_precision prec, int jp, const TermsF32 *t32,
                     const TermsF64 *, int num_sms, cudaStream_t s)
{
    if (a.n_trials <= 0) return 0;
    if (prec == ARE_FP32_KAHAN) return launch_fp32<ARE_FP32_KAHAN>(a, jp, *t32, num_sms, s);
    if (prec == ARE_FP32_FP64AGG) return launch_fp32<ARE_FP32_FP64AGG>(a, jp, *t32, num_sms, s);
    throw Error{ARE_EINVAL, "no FP32 simulate kernel for this precision"};
}

}  // namespace are
