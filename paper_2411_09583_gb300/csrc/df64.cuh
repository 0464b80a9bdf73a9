// Double-float arithmetic: a value is the unevaluated sum hi + lo of two
// floats (about 48 significant bits).  GB300 issues FP32 operations 64 times
// faster than FP64 ones, so the hot loops of the tap arithmetic (kernel-tap
// polynomials and tap accumulations) run in this format.
//
// Built from the classical error-free transformations: TwoSum (Knuth),
// FastTwoSum (Dekker) and TwoProduct by fused multiply-add; compensated Horner
// evaluation (Graillat, Langlois & Louvet, 2005) and the compensated dot
// product Dot2 (Ogita, Rump & Oishi, 2005).
#pragma once

#include <cstdint>

namespace nuht {

struct df {
    float h, l;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ df fast_two_sum(float a, float b)
{
    const float s = a + b;
    return df{s, b - (s - a)};
}

__device__ __forceinline__ df df_from(double x)
{
    const float h = (float)x;
    return df{h, (float)(x - (double)h)};
}

__device__ __forceinline__ double df_to(df a) { return (double)a.h + (double)a.l; }

__device__ __forceinline__ df df_mul(df a, df b)
{
    const float p = a.h * b.h;
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ df df_add(df a, df b)
{
    float s, e;
    two_sum(a.h, b.h, s, e);
    e += a.l + b.l;
    return fast_two_sum(s, e);
}

// Compensated Horner: p(v) = sum_k c_k v^k with double-float coefficients
// c[k] = (h, l) and the argument v = vh + vl (|vl| <= ulp(vh)/2).  The main
// sum runs in FP32 with its rounding errors (TwoProduct, TwoSum) and the low
// coefficient parts gathered in a correction polynomial; the low part of the
// argument enters through the first-order term vl p'(vh).
__device__ __forceinline__ df horner_comp(const float2* __restrict__ c, int deg, float vh, float vl)
{
    float s = c[deg].x, r = c[deg].y, dp = 0.0f;
    for (int k = deg - 1; k >= 0; --k) {
        dp = fmaf(dp, vh, s);                    // derivative by Horner, FP32 is enough
        const float p = s * vh;
        const float pi = fmaf(s, vh, -p);
        float s2, sg;
        two_sum(p, c[k].x, s2, sg);
        r = fmaf(r, vh, pi + sg + c[k].y);
        s = s2;
    }
    return fast_two_sum(s, fmaf(vl, dp, r));
}

// Compensated accumulator of products of double-float numbers (Dot2 style):
// the running sum s carries FP32 rounding errors into c.
struct acc2 {
    float s, c;
};

__device__ __forceinline__ void acc_fma(acc2& A, df a, df b)
{
    const float p = a.h * b.h;
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    float s, q;
    two_sum(A.s, p, s, q);
    A.s = s;
    A.c += q + e;
}

__device__ __forceinline__ double acc_value(acc2 A) { return (double)A.s + (double)A.c; }

}  // namespace nuht
