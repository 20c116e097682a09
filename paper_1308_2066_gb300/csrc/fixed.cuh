// fixed.cuh -- exact sums of non-negative doubles as fixed-point integers.
//
// GB300 issues FP64 adds at a small fraction of its integer rate.  A value
// h >= 0 scaled by 2^s (s chosen from an upper bound of the values, so that
// each scaled value is below 2^126) is a 128-bit integer; sums of such
// integers are kept in 160 bits with carries, exact in any order and for up
// to 2^34 terms, and rounded to double once at the end.  Every value of at
// least 2^-73 times the bound converts without error; a smaller one is
// rounded (half up) at 2^-s.
#pragma once

#include <cuda_runtime.h>

#include <stdint.h>

namespace are {
namespace fixed {

constexpr unsigned kFixedFull = 0xffffffffu;

struct Acc {   // top:hi:lo, 160 bits
    unsigned long long lo = 0, hi = 0;
    uint32_t top = 0;
    __device__ __forceinline__ void add(unsigned long long blo, unsigned long long bhi, uint32_t btop)
    {
        asm("add.cc.u64 %0, %0, %3;\n\t"
            "addc.cc.u64 %1, %1, %4;\n\t"
            "addc.u32 %2, %2, %5;"
            : "+l"(lo), "+l"(hi), "+r"(top)
            : "l"(blo), "l"(bhi), "r"(btop));
    }
};

// floor(log2(x)) of a positive finite double given by its bits.
__device__ __forceinline__ int ilog2_bits(unsigned long long b)
{
    const int e = (int)((b >> 52) & 0x7ff);
    if (e) return e - 1023;
    return (63 - __clzll((long long)b)) - 1074;   // subnormal
}

// h * 2^s as a 128-bit integer (round half up below the last bit).  With
// s = 125 - floor(log2(hmax)) and h <= hmax the result is below 2^126.
__device__ __forceinline__ void to_fixed(double h, int s, unsigned long long &lo, unsigned long long &hi)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(h);
    const int be = (int)((b >> 52) & 0x7ff);
    unsigned long long m = b & ((1ull << 52) - 1);
    if (be) m |= 1ull << 52;
    const int sh = (be ? be : 1) - 1075 + s;    // value = m * 2^sh
    lo = 0;
    hi = 0;
    if (sh >= 64) {
        hi = m << (sh - 64);
    } else if (sh > 0) {
        lo = m << sh;
        hi = m >> (64 - sh);
    } else if (sh == 0) {
        lo = m;
    } else if (sh >= -53) {
        const int n = -sh;
        lo = (m >> n) + ((m >> (n - 1)) & 1ull);
    }
}

// (top:hi:lo) * 2^-s rounded once to the nearest double.
__device__ __forceinline__ double to_double(const Acc &a, int s)
{
    int L;   // bit length
    if (a.top) L = 160 - __clz((int)a.top);
    else if (a.hi) L = 128 - __clzll((long long)a.hi);
    else if (a.lo) L = 64 - __clzll((long long)a.lo);
    else return 0.0;
    if (L <= 64) return ldexp(__ull2double_rn(a.lo), -s);
    const int r = L - 64;            // 1 .. 96
    unsigned long long w, sticky;
    if (r < 64) {
        w = (a.lo >> r) | (a.hi << (64 - r));
        sticky = a.lo & ((1ull << r) - 1);
    } else if (r == 64) {
        w = a.hi;
        sticky = a.lo;
    } else {
        const int q = r - 64;        // 1 .. 32
        w = (a.hi >> q) | ((unsigned long long)a.top << (64 - q));
        sticky = a.lo | (a.hi & ((1ull << q) - 1));
    }
    // w has its top bit set; a double keeps 53 of its 64 bits, so a sticky
    // bit in bit 0 makes the one rounding of the conversion the right one
    return ldexp(__ull2double_rn(w | (sticky ? 1ull : 0ull)), r - s);
}

__device__ __forceinline__ void warp_sum(Acc &a)
{
#pragma unroll
    for (int off = 16; off; off >>= 1) {
        const unsigned long long lo = __shfl_xor_sync(kFixedFull, a.lo, off);
        const unsigned long long hi = __shfl_xor_sync(kFixedFull, a.hi, off);
        const uint32_t top = __shfl_xor_sync(kFixedFull, a.top, off);
        a.add(lo, hi, top);
    }
}

}  // namespace fixed
}  // namespace are
