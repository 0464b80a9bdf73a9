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
//
// Degrees above kc (whose coefficients are so small that FP32 rounding of
// their partial sum stays far below the target accuracy) are summed first in
// plain FP32; kc >= deg makes every step compensated.
__device__ __forceinline__ df horner_comp(const float2* __restrict__ c, int deg, float vh, float vl,
                                          int kc = 1 << 30)
{
    float s = c[deg].x, r = kc >= deg ? c[deg].y : 0.0f, dp = 0.0f;
    int k = deg - 1;
    for (; k > kc; --k) {
        dp = fmaf(dp, vh, s);
        s = fmaf(s, vh, c[k].x);
    }
    for (; k >= 0; --k) {
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

namespace nuht {

__device__ __forceinline__ df df_negate(df a) { return df{-a.h, -a.l}; }

// Three-term step a t1 - t0 in double-float (a Chebyshev recurrence with
// a = 2x), as one
// compensated multiply-subtract: the product's rounding error and the low
// parts enter the correction, only the result is renormalised.
__device__ __forceinline__ df cheb_step(df a, df t1, df t0)
{
    const float P = a.h * t1.h;
    const float Pe = fmaf(a.l, t1.h, fmaf(a.h, t1.l, fmaf(a.h, t1.h, -P)));
    float sm, e;
    two_sum(P, -t0.h, sm, e);
    return fast_two_sum(sm, e + (Pe - t0.l));
}

// 1/a by one Newton step from the FP32 reciprocal (error ~ 2^-47).
__device__ __forceinline__ df df_recip(df a)
{
    const float y0 = 1.0f / a.h;
    const df p = df_mul(a, df{y0, 0.0f});
    const float e = (1.0f - p.h) - p.l;
    return fast_two_sum(y0, y0 * e);
}

// sqrt(a), a > 0, by one Newton step from the FP32 square root.
__device__ __forceinline__ df df_sqrt(df a)
{
    const float y0 = sqrtf(a.h);
    const float ph = y0 * y0;
    const float pl = fmaf(y0, y0, -ph);
    const float r = ((a.h - ph) - pl) + a.l;
    return fast_two_sum(y0, r * (0.5f / y0));
}

// sin and cos of x + q pi/2 for |x| <= pi/4 (double-float): the Taylor
// series sin x = x sum_k (-x^2)^k/(2k+1)!, cos x = sum_k (-x^2)^k/(2k)!,
// summed in double-float (truncation below 5e-17), then the quadrant q.
__device__ __forceinline__ void df_sincos_quadrant(df x, int q, df* sn, df* cs)
{
    // 1/n! split into float hi + lo parts (odd n for sin, even n for cos)
    const float2 ks[8] = {{1.0f, 0.0f}, {-0.1666666716337204f, 4.967053879312289e-09f},
                          {0.008333333767950535f, -4.34617203337595e-10f},
                          {-0.00019841270113829523f, 2.725596874933456e-12f},
                          {2.7557318844628753e-06f, 3.793571224297229e-14f},
                          {-2.5052107943679403e-08f, -4.4176230446483665e-16f},
                          {1.6059044372074283e-10f, -5.352526511562726e-18f},
                          {-7.647163609812713e-13f, -1.2200710471178288e-20f}};
    const float2 kc[9] = {{1.0f, 0.0f}, {-0.5f, 0.0f}, {0.0416666679084301f, -1.2417634698280722e-09f},
                          {-0.0013888889225199819f, 3.3631094437103215e-11f},
                          {2.4801587642286904e-05f, -3.40699609366682e-13f},
                          {-2.755731998149713e-07f, 7.575112209051195e-15f},
                          {2.0876755879584152e-09f, 1.1082839147459852e-16f},
                          {-1.147074536050896e-11f, -2.372207689231238e-19f},
                          {4.7794772561329454e-14f, 7.62544404448643e-22f}};
    const df y = df_mul(x, x);
    df ps{ks[7].x, ks[7].y};
#pragma unroll
    for (int i = 6; i >= 0; --i) ps = df_add(df_mul(ps, y), df{ks[i].x, ks[i].y});
    df pc{kc[8].x, kc[8].y};
#pragma unroll
    for (int i = 7; i >= 0; --i) pc = df_add(df_mul(pc, y), df{kc[i].x, kc[i].y});
    const df s0 = df_mul(x, ps);
    switch (q & 3) {
        case 0: *sn = s0; *cs = pc; break;
        case 1: *sn = pc; *cs = df_negate(s0); break;
        case 2: *sn = df_negate(s0); *cs = df_negate(pc); break;
        default: *sn = df_negate(pc); *cs = s0; break;
    }
}

// sin and cos of the exact product a*b (a, b doubles, |a*b| up to ~1e12).
// The product is split exactly (FMA two-product) and reduced modulo pi/2 in
// FP64 against a two-term pi/2; the remainder |t| <= pi/4 goes to
// df_sincos_quadrant.
__device__ __forceinline__ void df_sincos_prod(double a, double b, df* sn, df* cs)
{
    const double kPio2Hi = 1.5707963267948966;       // nearest double to pi/2
    const double kPio2Lo = 6.123233995736766e-17;    // pi/2 - kPio2Hi
    const double k2OverPi = 0.6366197723675814;
    const double p = a * b;
    const double e = fma(a, b, -p);
    const double k = rint(p * k2OverPi);
    double t = fma(-k, kPio2Hi, p);
    t = fma(-k, kPio2Lo, t) + e;
    df_sincos_quadrant(df_from(t), (int)((long long)k & 3), sn, cs);
}

// sin and cos of 2 pi F / 2^64 (F a fraction of a turn in 64-bit fixed
// point), with integer arithmetic down to the FP32 pipes: the quadrant is the
// top two bits (rounded), the rest an exact sum of three floats times 2 pi.
__device__ __forceinline__ void df_sincos_turns(unsigned long long F, df* sn, df* cs)
{
    const unsigned long long Fq = F + (1ULL << 61);
    const int quad = (int)(Fq >> 62);
    const long long rem = (long long)(Fq & ((1ULL << 62) - 1)) - (1LL << 61);   // [-2^61, 2^61)
    const float f1 = (float)(int)(rem >> 40) * 5.9604644775390625e-08f;          // 2^-24
    const float f2 = (float)(int)((rem >> 16) & 0xFFFFFF) * 3.552713678800501e-15f;   // 2^-48
    const float f3 = (float)(int)(rem & 0xFFFF) * 5.421010862427522e-20f;        // 2^-64
    float s, e;
    two_sum(f1, f2, s, e);
    const df turns = fast_two_sum(s, e + f3);
    const df x = df_mul(turns, df{6.2831854820251465f, -1.7484555314695172e-07f});   // 2 pi
    df_sincos_quadrant(x, quad, sn, cs);
}

// sin and cos of 2 pi F / 2^64 (F a fraction of a turn in 64-bit fixed
// point) from a table tw[k] = e^{2 pi i k / 8192}, k < 4096, as double-float
// (cos h, cos l, sin h, sin l): table-driven argument reduction.  The
// quadrant is the top two bits (rounded); of the remainder x (|x| <= pi/4)
// the nearest table angle theta_k = 2 pi k / 8192 (k <= 1024) is taken and
// the residual delta = x - theta_k (|delta| <= pi / 8192, from 48 exact bits
// of the fixed-point remainder) enters through its Taylor series:
// sin delta = delta - delta^3/6 and 1 - cos delta = delta^2/2 - delta^4/24,
// whose next terms are below 1e-19.  Then sin(theta + delta) =
// sin theta + (cos theta sin delta - sin theta (1 - cos delta)) and
// cos(theta + delta) = cos theta - (sin theta sin delta + cos theta (1 - cos
// delta)) in double-float; odd symmetry gives negative x.
__device__ __forceinline__ void df_sincos_turns_tab(unsigned long long F, const float4* __restrict__ tw, df* sn,
                                                    df* cs)
{
    const unsigned long long Fq = F + (1ULL << 61);
    const int quad = (int)(Fq >> 62);
    const long long rem = (long long)(Fq & ((1ULL << 62) - 1)) - (1LL << 61);   // [-2^61, 2^61)
    const long long ar = rem < 0 ? -rem : rem;                                      // [0, 2^61]
    const int k = (int)((ar + (1LL << 50)) >> 51);                                 // nearest k / 8192 turn
    const long long r = (ar - ((long long)k << 51)) >> 3;                          // [-2^47, 2^47], 2^-61 turns
    float th, tl;
    two_sum((float)(int)(r >> 24) * 16777216.f, (float)(int)(r & 0xFFFFFF), th, tl);
    const float s61 = 4.336808689942018e-19f;                                      // 2^-61
    const df dl = df_mul(df{th * s61, tl * s61}, df{6.2831854820251465f, -1.7484555314695172e-07f});
    const df d2 = df_mul(dl, dl);
    const df sd = fast_two_sum(dl.h, dl.l - dl.h * d2.h * (1.f / 6.f));          // sin delta
    const df u{0.5f * d2.h, 0.5f * d2.l - d2.h * d2.h * (1.f / 24.f)};            // 1 - cos delta
    const float4 t = tw[k];
    const df ck{t.x, t.y}, sk{t.z, t.w};
    df s0 = df_add(sk, df_add(df_mul(ck, sd), df_negate(df_mul(sk, u))));
    const df c0 = df_add(ck, df_negate(df_add(df_mul(sk, sd), df_mul(ck, u))));
    if (rem < 0) s0 = df_negate(s0);
    switch (quad & 3) {
        case 0: *sn = s0; *cs = c0; break;
        case 1: *sn = c0; *cs = df_negate(s0); break;
        case 2: *sn = df_negate(s0); *cs = df_negate(c0); break;
        default: *sn = df_negate(c0); *cs = s0; break;
    }
}

// sin, cos of 2 pi F / 2^64 (a fraction of a turn in 64-bit fixed point) in
// FP32: the quadrant from the top bits, sincosf of the remainder.
__device__ __forceinline__ void f32_sincos_turns(unsigned long long F, float* sn, float* cs)
{
    const unsigned long long Fq = F + (1ULL << 61);
    const long long rem = (long long)(Fq & ((1ULL << 62) - 1)) - (1LL << 61);
    const float t = (float)(int)(rem >> 32) * 1.4629180792671596e-09f;   // 2 pi 2^-32
    float s0, c0;
    sincosf(t, &s0, &c0);
    switch ((int)(Fq >> 62)) {
        case 0: *sn = s0; *cs = c0; break;
        case 1: *sn = c0; *cs = -s0; break;
        case 2: *sn = -s0; *cs = -c0; break;
        default: *sn = -c0; *cs = s0; break;
    }
}

// Bits [s, s + 63] of the signed 128-bit product X * K, 0 <= s <= 64.
__device__ __forceinline__ unsigned long long mul128_bits(long long X, long long K, int s)
{
    const unsigned long long lo = (unsigned long long)X * (unsigned long long)K;
    const unsigned long long hi = (unsigned long long)__mul64hi(X, K);
    if (s <= 0) return lo;
    if (s >= 64) return hi;
    return (hi << (64 - s)) | (lo >> s);
}

// round(r 2^fr) for finite r >= 0 with r 2^fr < 2^62, from the bits of r
// (integer instructions only).
__device__ __forceinline__ long long fx_from_double(double r, int fr)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(r);
    const int e = (int)((b >> 52) & 0x7ff);
    if (e == 0) return 0;                                   // zero or subnormal
    const long long m = (long long)((b & 0xFFFFFFFFFFFFFULL) | (1ULL << 52));
    const int sh = e - 1075 + fr;                           // r 2^fr = m 2^sh
    if (sh >= 0) return m << sh;
    if (sh <= -54) return 0;
    return (m + (1LL << (-sh - 1))) >> (-sh);
}

}  // namespace nuht
