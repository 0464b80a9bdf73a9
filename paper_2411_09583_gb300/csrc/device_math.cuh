// Device helpers: Bessel recurrences and series (FP64, FP32), FP32 Hankel expansion.
#pragma once

#include <cstdint>

#include "nuht_internal.h"

namespace nuht {

// True when |v| > 2^498 (~1e150): checked on the high word with integer ops.
__device__ __forceinline__ bool too_big(double v)
{
    return (__double2hiint(v) & 0x7fffffff) > 0x5F100000;
}

// Start index of the Miller backward recurrence for J_0..J_ntop(y): even and
// at least max(ntop + 8, y + 20 + 4 sqrt(y)) (gives ~4e-16 absolute accuracy
// for y <= 60, ntop <= 80, checked against an independent evaluator).
__device__ __forceinline__ int miller_start(int ntop, double y)
{
    const float yf = (float)y;
    const float a = yf + 20.f + 4.f * sqrtf(yf);
    int ns = (int)a + 1;
    if (ns < ntop + 8) ns = ntop + 8;
    return ns + (ns & 1);
}

// J_n(x), n >= 0, by the power series (DLMF 10.2.2); used for x < 1.
__device__ __forceinline__ double jn_series(int n, double x)
{
    double h = 0.5 * x;
    double lead = 1.0;
    for (int i = 1; i <= n; ++i) lead *= h / (double)i;
    double q = -h * h, term = lead, sum = lead;
#pragma unroll
    for (int k = 1; k <= 10; ++k) {
        term *= q / ((double)k * (double)(n + k));
        sum += term;
    }
    return sum;
}

// J_n(x) for n >= 0 and 1 <= x (moderate): Miller backward recurrence from a
// start index beyond max(n, x), normalised by J_0 + 2 sum_k J_2k = 1.
__device__ inline double jn_miller(int n, double x)
{
    int ns = miller_start(n, x);
    double inv2x = 2.0 / x;
    double jp1 = 0.0, jc = 1.0;
    double S = 2.0;          // 2 * J_ns (ns even)
    double res = 0.0;
    for (int i = ns; i >= 2; i -= 2) {
        double jm = fma((double)i * inv2x, jc, -jp1);          // J_{i-1}
        double jmm = fma((double)(i - 1) * inv2x, jm, -jc);    // J_{i-2}
        if (i - 1 == n) res = jm;
        if (i - 2 == n) res = jmm;
        S = fma(2.0, jmm, S);
        jp1 = jm;
        jc = jmm;
        if (too_big(jc)) {
            const double sc = 1e-150;
            jc *= sc; jp1 *= sc; S *= sc; res *= sc;
        }
    }
    S -= jc;                 // J_0 was added with weight 2; it counts once
    return res / S;
}

// J_n(x) for x <= a crossover z (local side of a direct block).
__device__ __forceinline__ double jn_small_arg(int n, double x)
{
    if (x < 1.0) return jn_series(n, x);
    return jn_miller(n, x);
}


// ---------------------------------------------------------- FP32 variants
// (for tolerances eps >= 1e-6, where FP32 evaluation error stays far below eps)

// J_n(x), 1 <= x, Miller's recurrence in FP32 (rescaled by 2^-60 past 2^60).
__device__ inline float jn_miller_f32(int n, float x)
{
    const int ns = miller_start(n, (double)x);
    const float inv2x = 2.0f / x;
    float jp1 = 0.f, jc = 1.f, S = 2.f, res = 0.f;
    for (int i = ns; i >= 2; i -= 2) {
        const float jm = fmaf((float)i * inv2x, jc, -jp1);
        const float jmm = fmaf((float)(i - 1) * inv2x, jm, -jc);
        if (i - 1 == n) res = jm;
        if (i - 2 == n) res = jmm;
        S = fmaf(2.f, jmm, S);
        jp1 = jm;
        jc = jmm;
        if (fabsf(jc) > 1.152921504606847e18f) {
            const float sc = 8.673617379884035e-19f;
            jc *= sc; jp1 *= sc; S *= sc; res *= sc;
        }
    }
    return res / (S - jc);
}

// Hankel's expansion in FP32 after an FP64 reduction of the exact product w*r modulo pi/2.
__device__ inline float jn_hankel_f32(const ProbParams& P, double w, double r)
{
    const double p = w * r;
    const double e = fma(w, r, -p);
    const double k = rint(p * 0.6366197723675814);
    double t = fma(-k, 1.5707963267948966, p);
    t = fma(-k, 6.123233995736766e-17, t) + e;
    float s0, c0;
    sincosf((float)t, &s0, &c0);
    float sx, cx;
    switch ((int)((long long)k & 3)) {
        case 0: sx = s0; cx = c0; break;
        case 1: sx = c0; cx = -s0; break;
        case 2: sx = -s0; cx = -c0; break;
        default: sx = -c0; cx = s0; break;
    }
    const float y = (float)(1.0 / p);
    const float u = y * P.z2.x, u2 = u * u;   // z / x < 1, with the coefficients a_q z^-q
    float pp = 0.f, qq = 0.f;
    for (int l = P.M - 1; l >= 0; --l) {
        const float sg = (l & 1) ? -1.f : 1.f;
        pp = fmaf(pp, u2, sg * P.a2[2 * l].x);
        qq = fmaf(qq, u2, sg * P.a2[2 * l + 1].x);
    }
    qq *= u;
    const float cph = (float)P.cphi, sph = (float)P.sphi;
    const float cchi = cx * cph - sx * sph, schi = sx * cph + cx * sph;
    return sqrtf(0.6366197723675814f * y) * (pp * cchi - qq * schi);
}

}  // namespace nuht
