// Exact, order-independent sums of non-negative values for sum(r).
//
// Terms are added in 128-bit fixed point whose last bit is worth 2^(E-100),
// where 2^E bounds every term: E comes from the previous sum(r), which
// bounds every new rank because the PageRank update never increases the
// total (Sec. IV-D: mass leaks through dangling rows and removed columns, and
// is never created).  Any grouping of the same terms gives the same bits, so
// a sum does not depend on which block or warp added which term, and only
// terms below 2^(E-100) lose bits.  Conversions read the float bits with
// integer instructions only (the FP64 pipe of GB300 is narrow).
#pragma once

#include "pp_common.cuh"

namespace pp {

struct Fx128 {
    uint64_t hi, lo;
};

__device__ __forceinline__ void fx_add(Fx128 &a, uint64_t h, uint64_t l) {
    a.lo += l;
    a.hi += h + (a.lo < l ? 1ull : 0ull);
}

// m * 2^sh as a 128-bit integer (m < 2^53; the caller's bound on E keeps
// sh + 53 <= 128), integer instructions only.
__device__ __forceinline__ void fx_add_shifted(Fx128 &a, uint64_t m, int sh) {
    uint64_t h = 0, l = 0;
    if (sh <= -64) {
        return;
    } else if (sh < 0) {
        l = m >> (-sh);
    } else if (sh == 0) {
        l = m;
    } else if (sh < 64) {
        l = m << sh;
        h = m >> (64 - sh);
    } else {
        h = m << (sh - 64);
    }
    fx_add(a, h, l);
}

// x * 2^(100-E) from the bits of x (x >= 0; 0, negative and NaN add nothing).
__device__ __forceinline__ void fx_add(Fx128 &a, double x, int E) {
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    if ((long long)b <= 0) return;
    const int e = (int)(b >> 52);
    if (e == 0x7ff) return;
    const uint64_t m = (b & ((1ull << 52) - 1)) | (e ? (1ull << 52) : 0ull);
    fx_add_shifted(a, m, (e ? e : 1) - 1075 + 100 - E);  // x = m * 2^((e?e:1) - 1075)
}

__device__ __forceinline__ void fx_add(Fx128 &a, float x, int E) {
    const uint32_t b = __float_as_uint(x);
    if ((int)b <= 0) return;
    const int e = (int)(b >> 23);
    if (e == 0xff) return;
    const uint64_t m = (b & 0x7fffffu) | (e ? 0x800000u : 0u);
    fx_add_shifted(a, m, (e ? e : 1) - 150 + 100 - E);  // x = m * 2^((e?e:1) - 150)
}

// x * 2^(100-E) for 0 <= x < 2^(E-1), without branches (the binary64 column
// sums of Kernel 3, one per matrix entry): the bound keeps the shift at most
// 46 bits left; bits below 2^(E-100) are dropped.
__device__ __forceinline__ void fx_add_term(Fx128 &a, double x, int E) {
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    const int e = (int)(b >> 52) & 0x7ff;
    const uint64_t m = (b & ((1ull << 52) - 1)) | (e ? (1ull << 52) : 0ull);
    const int sh = (e ? e : 1) - 1075 + 100 - E;
    const uint64_t l = sh >= 0 ? (m << sh) : (sh > -64 ? (m >> -sh) : 0ull);
    const uint64_t h = sh > 0 ? (m >> (64 - sh)) : 0ull;
    fx_add(a, h, l);
}

// a * 2^(E-100) rounded to the nearest binary64 (ties to even), from integer
// instructions only; the value must be 0 or in the normal range.
__device__ __forceinline__ double fx_to_double(Fx128 a, int E) {
    if (!(a.hi | a.lo)) return 0.0;
    const int lz = a.hi ? __clzll((long long)a.hi) : 64 + __clzll((long long)a.lo);
    uint64_t hi = a.hi, lo = a.lo;
    if (lz >= 64) {
        hi = lo << (lz - 64);
        lo = 0;
    } else if (lz > 0) {
        hi = (hi << lz) | (lo >> (64 - lz));
        lo <<= lz;
    }
    // the leading one is now bit 63 of hi: 53 bits of mantissa, then the rest
    uint64_t mant = hi >> 11;
    const uint64_t rest = hi & 0x7ffull;
    const bool half = (rest >> 10) & 1ull, sticky = (rest & 0x3ffull) || lo;
    if (half && (sticky || (mant & 1ull))) ++mant;
    int ex = 127 - lz + E - 100;  // value = mant * 2^(ex - 52)
    if (mant >> 53) {
        mant >>= 1;
        ++ex;
    }
    return __longlong_as_double((long long)((((uint64_t)(ex + 1023)) << 52) | (mant & ((1ull << 52) - 1))));
}

// Exact sum over a warp, in lane 0.
__device__ __forceinline__ Fx128 fx_warp_sum(Fx128 a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t h = __shfl_down_sync(0xffffffffu, a.hi, o);
        const uint64_t l = __shfl_down_sync(0xffffffffu, a.lo, o);
        fx_add(a, h, l);
    }
    return a;
}

__device__ __forceinline__ double fx_value(uint64_t hi, uint64_t lo, int E) {
    return ldexp((double)hi, E - 36) + ldexp((double)lo, E - 100);
}

// Exponent for the next accumulator: 2^E > S >= any rank of the next iterate.
__device__ __forceinline__ int fx_exponent(double S) {
    int e = 0;
    frexp(S, &e);
    return e + 1;
}

template <int THREADS_>
__device__ __forceinline__ Fx128 fx_block_sum(Fx128 a, uint64_t *scratch /* 2 * warps */) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t h = __shfl_down_sync(0xffffffffu, a.hi, o);
        const uint64_t l = __shfl_down_sync(0xffffffffu, a.lo, o);
        fx_add(a, h, l);
    }
    if (lane == 0) {
        scratch[2 * warp] = a.hi;
        scratch[2 * warp + 1] = a.lo;
    }
    __syncthreads();
    Fx128 t{0, 0};
    if (threadIdx.x == 0)
        for (int w = 0; w < THREADS_ / 32; ++w) fx_add(t, scratch[2 * w], scratch[2 * w + 1]);
    __syncthreads();
    return t;
}

// Adds v to the 128-bit accumulator acc[0] (hi), acc[1] (lo).  The two words
// are updated by separate atomics, so only the final value (after every
// contribution) is meaningful.
__device__ __forceinline__ void fx_atomic_add(unsigned long long *acc, Fx128 v) {
    const unsigned long long old = atomicAdd(acc + 1, (unsigned long long)v.lo);
    const unsigned long long carry = (old + v.lo < old) ? 1ull : 0ull;
    if (v.hi + carry) atomicAdd(acc, (unsigned long long)(v.hi + carry));
}

}  // namespace pp
