// Deterministic accumulation: exact 128-bit fixed-point sums.
//
// Every block class adds its contributions into shared outputs (g, the
// spreading grids, the moments) from many CTAs.  With FP64 atomics the order
// of those additions, and so the last bits of the result, changes from run
// to run.  In the deterministic mode each contribution v is instead rounded
// once to the integer round(v 2^s) and added to a signed 128-bit two's
// complement accumulator (two 64-bit words, the carry out of the low word
// added to the high word).  Integer addition is associative, so the sum, and
// the double it is converted to at the end, is the same whatever order the
// additions happen in.  Every call scales its input vector by a power of two
// so that its largest magnitude lies in [1, 2) (input_exponent); the scale s is
// then fixed (kFxScale): every partial sum stays below 2^126 and one
// contribution's rounding is at most 2^-(s+1), 2^-54 of the largest input.
#pragma once

#include <climits>
#include <cstdint>

namespace nuht {

// ProbParams::fxs value that selects FP64 atomics (the default mode).
constexpr int kFxOff = INT_MIN;

struct Fx128 {
    unsigned long long lo, hi;
};

// round(v 2^s) as a 128-bit two's complement integer (lo, hi), by integer
// operations on the bits of v.  |v| 2^s must stay below 2^126 (the scale
// guarantees it); rounding is to nearest, ties away from zero.
__device__ __forceinline__ void fx_encode(double v, int s, unsigned long long& lo, unsigned long long& hi)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int e = (int)((b >> 52) & 0x7ff);
    unsigned long long mant = b & 0xfffffffffffffull;
    if (e) mant |= 1ull << 52;
    const int sh = (e ? e : 1) - 1075 + s;   // |v| 2^s = mant 2^sh
    lo = 0;
    hi = 0;
    if (mant == 0) return;
    if (sh >= 0) {
        if (sh == 0) {
            lo = mant;
        } else if (sh < 64) {
            lo = mant << sh;
            hi = mant >> (64 - sh);
        } else if (sh < 74) {
            hi = mant << (sh - 64);
        } else {
            hi = 0x3fffffffffffffffull;   // out of range: saturate (not reached with a valid scale)
        }
    } else if (sh > -64) {
        const int rs = -sh;
        lo = (mant + (1ull << (rs - 1))) >> rs;
    }
    if (b >> 63) {   // negate
        lo = ~lo + 1ull;
        hi = ~hi + (lo == 0 ? 1ull : 0ull);
    }
}

// *p += (lo, hi) modulo 2^128 (global or shared memory).  The low word's
// carry is exact: the old value returned by the atomic tells whether this
// addition wrapped, and the wraps of all additions sum to the same count in
// any order.
static __device__ __noinline__ void fx_add_words(Fx128* p, unsigned long long lo, unsigned long long hi)
{
    if (lo) {
        const unsigned long long old = atomicAdd(&p->lo, lo);
        if (old + lo < old) hi += 1ull;
    }
    if (hi) atomicAdd(&p->hi, hi);
}

// Not inlined: the hot kernels call it only in the deterministic mode, and
// keeping it out of line keeps their default (FP64 atomic) path's registers.
static __device__ __noinline__ void fx_add(Fx128* p, double v, int s)
{
    unsigned long long lo, hi;
    fx_encode(v, s, lo, hi);
    fx_add_words(p, lo, hi);
}

// The double nearest (within an ulp) to the accumulator times 2^-s.
__device__ __forceinline__ double fx_decode(Fx128 a, int s)
{
    const bool neg = (long long)a.hi < 0;
    if (neg) {
        a.lo = ~a.lo + 1ull;
        a.hi = ~a.hi + (a.lo == 0 ? 1ull : 0ull);
    }
    const double v = scalbn(fma((double)a.hi, 18446744073709551616.0, (double)a.lo), -s);
    return neg ? -v : v;
}

// E with v in [2^E, 2^(E+1)) for the bit pattern b of a non-negative double v
// (0 for v = 0): the execute kernels see their inputs scaled by 2^-E of the
// largest input magnitude, so that it lies in [1, 2).
__device__ __forceinline__ int input_exponent(unsigned long long b)
{
    if (b == 0) return 0;
    const int ebits = (int)((b >> 52) & 0x7ff);
    if (ebits) return ebits - 1023;
    return -1023 - (__clzll((long long)(b & 0xfffffffffffffull)) - 12);   // subnormal: its leading bit
}

// Deterministic-mode scale of the fixed-point sums: with inputs scaled into
// [1, 2) in magnitude, a sum of at most 2^31 of them, each carried with a
// factor of at most 2^40 (every expansion and grid value of the transform
// stays far below that), is below 2^125 times 2^-53, so round(v 2^53) stays in
// the signed 128-bit range, and one contribution rounds by at most 2^-54.
constexpr int kFxScale = 53;

// An accumulation target: an FP64 array (FP64 atomics), or in the
// deterministic mode an Fx128 array with the same element indices.
struct Accum {
    double* p;
    int fxs;
    __device__ __forceinline__ void add(int64_t i, double v) const
    {
        if (fxs == kFxOff) atomicAdd(p + i, v);
        else fx_add(reinterpret_cast<Fx128*>(p) + i, v, fxs);
    }
    __device__ __forceinline__ bool det() const { return fxs != kFxOff; }
    // the same target from element off on
    __device__ __forceinline__ Accum at(int64_t off) const
    {
        return Accum{fxs == kFxOff ? p + off : reinterpret_cast<double*>(reinterpret_cast<Fx128*>(p) + off), fxs};
    }
};

// The two modes as compile-time targets with Accum's interface, for kernels
// instantiated once per mode (the spreading kernel: the out-of-line
// fixed-point call would otherwise cost the FP64 path registers).
struct AccumF64 {
    double* p;
    int fxs;
    __device__ __forceinline__ void add(int64_t i, double v) const { atomicAdd(p + i, v); }
    __device__ __forceinline__ AccumF64 at(int64_t off) const { return AccumF64{p + off, fxs}; }
};

struct AccumFx {
    double* p;
    int fxs;
    __device__ __forceinline__ void add(int64_t i, double v) const
    {
        fx_add(reinterpret_cast<Fx128*>(p) + i, v, fxs);
    }
    __device__ __forceinline__ AccumFx at(int64_t off) const
    {
        return AccumFx{reinterpret_cast<double*>(reinterpret_cast<Fx128*>(p) + off), fxs};
    }
};

template <bool DET>
struct AccumOf {
    using type = AccumF64;
};
template <>
struct AccumOf<true> {
    using type = AccumFx;
};

}  // namespace nuht
