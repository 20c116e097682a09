// repack.cu -- preprocessing (Section II-B, stage 1): the layer's ELTs become
// one event-major direct-access table.
//
// The paper keeps one catalog-sized loss array per ELT (Section III-B: a
// 2M-event catalog and 15 ELTs give 30M event-loss pairs), so an event costs
// one random access per ELT.  Here row e of a single table holds event e's
// entries in all J ELTs of the layer, in layer order, padded to a whole
// number of 32-byte sectors (jp columns, zeros past J): one event's lookups
// in every ELT become one row read.
//
// Each entry is the event's financial term in that ELT (Section II-B step 2
// before its sum over ELTs): f_j(x) = share_j * min(max(fx_j * x - D_j, 0),
// Lim_j), formed in FP64 in exactly the operations and order the terms
// define (fx * x, less D, clamped, times the share) and rounded once to the
// table type.  A term depends only on the event and the ELT, never on the
// trial, so it is formed once per ELT entry here instead of once per
// occurrence; every occurrence still reads its event's whole row.  An event
// the ELT does not hold has x = 0 and stores f_j(0) = 0.
#include <cuda_runtime.h>

#include "are_internal.cuh"

namespace are {
namespace {

template <typename T, bool RU>
__global__ void k_scatter(T *__restrict__ tab, const ScatterArgs a)
{
    const int j = blockIdx.y;
    const int32_t n = a.n[j];
    const int32_t *ids = a.ids[j];
    const double *loss = a.loss[j];
    const double fx = a.fx[j], ded = a.ded[j], lim = a.lim[j], share = a.share[j];
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double x = fin_term(loss[i], fx, ded, lim, share);
        tab[(size_t)ids[i] * a.jp + j] = RU ? (T)__double2float_ru(x) : (T)x;
    }
}

// Packed FP64 rows (rw = 4 or 8 words: 32 or 64 bytes): row e holds the
// mask of its non-zero columns (low 32 bits of word 0) and those terms in
// column order (words 1 .. rw - 1).  A row with more non-zero terms than
// that keeps the first rw - 1 inline and all of them in a block of the
// overflow array, whose offset goes to the high 32 bits of word 0 (blocks
// are handed out by an atomic counter; each block holds its row's terms in
// column order).  Built straight from the ELT entries in three passes (grid.y
// = ELT j), each entry's term formed as k_scatter forms it; ELT ids are
// unique, so each (row, column) is one entry's alone.
// 1. the mask;
__global__ void k_pack64_mask(const ScatterArgs a, unsigned long long *__restrict__ rows, int rw)
{
    const int j = blockIdx.y;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n[j]; i += gridDim.x * blockDim.x) {
        const double x = fin_term(a.loss[j][i], a.fx[j], a.ded[j], a.lim[j], a.share[j]);
        if (__double_as_longlong(x) != 0) atomicOr(rows + (size_t)a.ids[j][i] * rw, 1ull << j);
    }
}

// 2. the inline terms at their rank; in a row that overflows, the entry of
//    rank 0 takes the row's overflow block and writes its offset;
__global__ void k_pack64_place(const ScatterArgs a, unsigned long long *__restrict__ rows, int rw,
                               unsigned long long *__restrict__ ovf_used)
{
    const int j = blockIdx.y;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n[j]; i += gridDim.x * blockDim.x) {
        const double x = fin_term(a.loss[j][i], a.fx[j], a.ded[j], a.lim[j], a.share[j]);
        if (__double_as_longlong(x) == 0) continue;
        unsigned long long *row = rows + (size_t)a.ids[j][i] * rw;
        const uint32_t mask = (uint32_t)row[0];
        const int cnt = __popc(mask), r = __popc(mask & ((1u << j) - 1u));
        if (r < rw - 1) row[1 + r] = (unsigned long long)__double_as_longlong(x);
        if (cnt > rw - 1 && r == 0) {
            const unsigned long long off = atomicAdd(ovf_used, (unsigned long long)cnt);
            atomicOr(row, off << 32);
        }
    }
}

// 3. every term of an overflowing row into its block.
__global__ void k_pack64_over(const ScatterArgs a, const unsigned long long *__restrict__ rows, int rw,
                              double *__restrict__ ovf)
{
    const int j = blockIdx.y;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n[j]; i += gridDim.x * blockDim.x) {
        const unsigned long long h = rows[(size_t)a.ids[j][i] * rw];
        const uint32_t mask = (uint32_t)h;
        if (__popc(mask) <= rw - 1 || !((mask >> j) & 1u)) continue;
        const int r = __popc(mask & ((1u << j) - 1u));
        ovf[(uint32_t)(h >> 32) + r] = fin_term(a.loss[j][i], a.fx[j], a.ded[j], a.lim[j], a.share[j]);
    }
}

// Packed FP32 rows (pw = 8 or 16 words: 32 or 64 bytes): word 0 holds the
// mask of the ELT columns whose term is not 0, words 1 .. pw - 1 those terms
// in column order (the rest 0).  A row of more than pw - 1 non-zero terms
// keeps the first pw - 2 inline and in word pw - 1 the offset of a block of
// the overflow array (handed out by an atomic counter) that holds the rest
// in column order.
// They are built straight from the ELT entries (no dense table): three
// passes over the entries of every ELT (grid.y = ELT j), each entry's term
// formed and rounded as k_scatter forms it.  ELT ids are
// unique, so each (row, column) is one entry's alone.
// 1. the mask: bit j of word 0 of the entry's row where its term is not 0;
__global__ void k_pack32_mask(const ScatterArgs a, uint32_t *__restrict__ rows, int pw)
{
    const int j = blockIdx.y;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n[j]; i += gridDim.x * blockDim.x) {
        const float f = (float)fin_term(a.loss[j][i], a.fx[j], a.ded[j], a.lim[j], a.share[j]);
        if (__float_as_uint(f) != 0u) atomicOr(rows + (size_t)a.ids[j][i] * pw, 1u << j);
    }
}

// 2. the inline terms: rank r (the set mask bits below j) goes to word 1 + r;
//    in a row that overflows, the entry of the first rank past the inline
//    ones takes the row's overflow block and writes its offset to the last
//    word;
__global__ void k_pack32_place(const ScatterArgs a, uint32_t *__restrict__ rows, int pw, float *__restrict__ ovf,
                               unsigned long long *__restrict__ ovf_used)
{
    const int j = blockIdx.y;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n[j]; i += gridDim.x * blockDim.x) {
        const float f = (float)fin_term(a.loss[j][i], a.fx[j], a.ded[j], a.lim[j], a.share[j]);
        if (__float_as_uint(f) == 0u) continue;
        uint32_t *row = rows + (size_t)a.ids[j][i] * pw;
        const uint32_t mask = row[0];
        const int cnt = __popc(mask), r = __popc(mask & ((1u << j) - 1u));
        const bool over = cnt > pw - 1;
        const int inl = over ? pw - 2 : cnt;
        if (r < inl) {
            row[1 + r] = __float_as_uint(f);
        } else if (r == inl) {
            const uint32_t off = (uint32_t)atomicAdd(ovf_used, (unsigned long long)(cnt - inl));
            row[pw - 1] = off;
            ovf[off] = f;
        }
    }
}

// 3. the other terms past the inline ones, at their rank in the row's block.
__global__ void k_pack32_over(const ScatterArgs a, const uint32_t *__restrict__ rows, int pw,
                              float *__restrict__ ovf)
{
    const int j = blockIdx.y;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n[j]; i += gridDim.x * blockDim.x) {
        const uint32_t *row = rows + (size_t)a.ids[j][i] * pw;
        const uint32_t mask = row[0];
        const int cnt = __popc(mask), inl = pw - 2;
        if (cnt <= pw - 1) continue;   // no overflow in this row
        const int r = __popc(mask & ((1u << j) - 1u));
        if (!((mask >> j) & 1u) || r <= inl) continue;
        ovf[row[pw - 1] + (r - inl)] = (float)fin_term(a.loss[j][i], a.fx[j], a.ded[j], a.lim[j], a.share[j]);
    }
}

}  // namespace

// Packed FP32 rows (pw words) straight from the layer's ELT entries: rows
// catalog x pw words, ovf room for every entry, ovf_used a device counter.
// Three launches, no dense table.
int launch_pack32_direct(const ScatterArgs &a, int32_t catalog, int pw, uint32_t *rows, float *ovf,
                         unsigned long long *ovf_used, cudaStream_t s)
{
    if (pw != 8 && pw != 16) throw Error{ARE_EINVAL, "packed FP32 rows are 8 or 16 words"};
    ARE_CUDA_TRY(cudaMemsetAsync(ovf_used, 0, sizeof *ovf_used, s));
    if (catalog <= 0) return 0;
    ARE_CUDA_TRY(cudaMemsetAsync(rows, 0, sizeof(uint32_t) * (size_t)catalog * pw, s));
    int32_t nmax = 0;
    for (int j = 0; j < a.n_elts; ++j) nmax = a.n[j] > nmax ? a.n[j] : nmax;
    if (nmax == 0 || a.n_elts == 0) return 0;
    dim3 grid((unsigned)((nmax + 255) / 256), (unsigned)a.n_elts);
    if (grid.x > 4096) grid.x = 4096;
    k_pack32_mask<<<grid, 256, 0, s>>>(a, rows, pw);
    k_pack32_place<<<grid, 256, 0, s>>>(a, rows, pw, ovf, ovf_used);
    k_pack32_over<<<grid, 256, 0, s>>>(a, rows, pw, ovf);
    ARE_CUDA_TRY(cudaGetLastError());
    return 3;
}

// Words per packed row for a layer whose ELTs hold `terms_per_event`
// entries per catalog event on average (an upper bound of the mean count of
// non-zero terms in a row), or 0 for the dense FP32 row.  32-byte rows (one
// sector, one lane per row) where the rows that overflow them are rare: FP32
// (7 terms inline) up to 2 entries per event for tables of more than 8 ELTs
// (8 or fewer already have 32-byte dense rows); FP64 (3 terms inline) up to
// 0.5.  Otherwise FP32 keeps the dense 64-byte row up to 16 ELTs and packs
// wider tables into 64-byte rows (15 terms inline), and FP64 packs into
// 64-byte rows (7 terms inline).
int packed_row_words(int n_elts, double terms_per_event, bool fp32)
{
    if (fp32) {
        if (n_elts <= 8) return 0;
        if (terms_per_event <= 2.0) return 8;
        return n_elts > 16 ? 16 : 0;
    }
    return terms_per_event <= 0.5 ? 4 : 8;
}

// Packed FP64 rows (rw words) straight from the layer's ELT entries: rows
// catalog x rw words, ovf room for every entry, ovf_used a device counter.
// Three launches, no dense table.
int launch_pack64_direct(const ScatterArgs &a, int32_t catalog, int rw, unsigned long long *rows, double *ovf,
                         unsigned long long *ovf_used, cudaStream_t s)
{
    if (rw != 4 && rw != 8) throw Error{ARE_EINVAL, "packed FP64 rows are 4 or 8 words"};
    ARE_CUDA_TRY(cudaMemsetAsync(ovf_used, 0, sizeof *ovf_used, s));
    if (catalog <= 0) return 0;
    ARE_CUDA_TRY(cudaMemsetAsync(rows, 0, sizeof(unsigned long long) * (size_t)catalog * rw, s));
    int32_t nmax = 0;
    for (int j = 0; j < a.n_elts; ++j) nmax = a.n[j] > nmax ? a.n[j] : nmax;
    if (nmax == 0 || a.n_elts == 0) return 0;
    dim3 grid((unsigned)((nmax + 255) / 256), (unsigned)a.n_elts);
    if (grid.x > 4096) grid.x = 4096;
    k_pack64_mask<<<grid, 256, 0, s>>>(a, rows, rw);
    k_pack64_place<<<grid, 256, 0, s>>>(a, rows, rw, ovf_used);
    k_pack64_over<<<grid, 256, 0, s>>>(a, rows, rw, ovf);
    ARE_CUDA_TRY(cudaGetLastError());
    return 3;
}

// Columns per row: J rounded up so a row fills whole 32-byte sectors; FP32
// rows are 8, 16 or 32 floats (a power of two, so the lanes that share a row
// pair up by halving), FP64 rows any multiple of 4 doubles.
int table_jp(int n_elts, bool fp32)
{
    if (fp32) return n_elts <= 8 ? 8 : n_elts <= 16 ? 16 : 32;
    int jp = (n_elts + 3) / 4 * 4;
    return jp < 4 ? 4 : jp;
}

// round_up (FP32 only): each value rounded towards +infinity -- the FP32
// screen of an FP64 table, never below the value it stands for (so positive
// exactly where the FP64 entry is).
int launch_scatter_table(void *table, bool fp32, const ScatterArgs &a, cudaStream_t s, bool round_up)
{
    int32_t nmax = 0;
    for (int j = 0; j < a.n_elts; ++j) nmax = a.n[j] > nmax ? a.n[j] : nmax;
    if (nmax == 0 || a.n_elts == 0) return 0;
    dim3 grid((unsigned)((nmax + 255) / 256), (unsigned)a.n_elts);
    if (grid.x > 4096) grid.x = 4096;
    if (fp32 && round_up)
        k_scatter<float, true><<<grid, 256, 0, s>>>(static_cast<float *>(table), a);
    else if (fp32)
        k_scatter<float, false><<<grid, 256, 0, s>>>(static_cast<float *>(table), a);
    else
        k_scatter<double, false><<<grid, 256, 0, s>>>(static_cast<double *>(table), a);
    ARE_CUDA_TRY(cudaGetLastError());
    return 1;
}

}  // namespace are
