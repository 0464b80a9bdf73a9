// Local blocks (Wimp expansion, Sec. 3.1) and direct blocks (Sec. 4.1).
//
// A local block A(k0:k1, j0:j1) with R = max r of the block is applied as the
// rank-(L+1) product of Sec. 3.1:
//     moments   mu_l = sum_j c_j T_{2l(+1)}(r_j / R),       l = 0..L
//     evaluate  g_k += sum_l C_l(omega_k R) mu_l,
// C_l(x) = delta_l J_{nu/2+l}(x/2) J_{nu/2-l}(x/2) for even nu and
// 2 J_{(nu+1)/2+l}(x/2) J_{(nu-1)/2-l}(x/2) with T_{2l+1} for odd nu (the
// argument x/2 follows the proof of Lemma 3.1; the odd form is Graf's addition
// theorem with both arguments x/2).
//
// Arithmetic: the Chebyshev recurrences, the Miller recurrence and the sums
// run in double-float (df64.cuh, ~48 bits on the FP32 pipes); the moments'
// column sums end in one FP64 atomic per moment, and the rare small-argument
// rows use the FP64 power series.  Mixed precision evaluates the local blocks
// in FP32 (k_local_eval_f32; the moments stay double-float).
//
// Direct blocks are small mixed blocks summed entry by entry with a device
// J_nu: Miller recurrence (or the power series) where omega r <= z, and the
// M-term Hankel expansion, accurate to eps there by the choice of z, where
// omega r > z.  omega r is the exact 128-bit product of the block's
// fixed-point omega and r; at eps >= 1e-6 the entries are FP32 values, summed
// in FP32 slots where the rounding bound allows (direct_sum_mode).
#include <algorithm>
#include <cstdint>

#include "device_math.cuh"
#include "df64.cuh"
#include "nuht_internal.h"

namespace nuht {

namespace {

constexpr int kMomThreads = 128;

__device__ __forceinline__ df df_neg(df a) { return df{-a.h, -a.l}; }
__device__ __forceinline__ df df_scale(df a, float p2) { return df{a.h * p2, a.l * p2}; }

// |v| > 2^60: the double-float Miller recurrence rescales by 2^-60 (exact)
__device__ __forceinline__ bool df_big(df v) { return fabsf(v.h) > 1.152921504606847e18f; }

// (double)i * inv2y as double-float, with inv2y = (ih, il)
__device__ __forceinline__ df df_imul(float fi, float ih, float il)
{
    const float p = fi * ih;
    float e = fmaf(fi, ih, -p);
    e = fmaf(fi, il, e);
    return fast_two_sum(p, e);
}

// Sum of a compensated accumulator over the warp (two-sums through the
// shuffles); the total is in lane 0.
__device__ __forceinline__ acc2 warp_sum_acc(acc2 a)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const float os = __shfl_down_sync(0xffffffffu, a.s, off);
        const float oc = __shfl_down_sync(0xffffffffu, a.c, off);
        float s, e;
        two_sum(a.s, os, s, e);
        a.s = s;
        a.c += oc + e;
    }
    return a;
}

// dst[l] += sum over the CTA's threads of acc[l * nt + thread], l <= L: one
// warp per l, compensated FP32 sums, one conversion and one FP64 atomic per l
// (FP64 runs at 1/64 of the FP32 rate).
__device__ __forceinline__ void reduce_columns_add(const acc2* acc, int nt, int L, Accum dst)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int l = warp; l <= L; l += nw) {
        acc2 a{0.f, 0.f};
        for (int k = lane; k < nt; k += 32) {
            const acc2 v = acc[l * nt + k];
            float s, e;
            two_sum(a.s, v.s, s, e);
            a.s = s;
            a.c += v.c + e;
        }
        a = warp_sum_acc(a);
        if (lane == 0) dst.add(l, acc_value(a));
    }
}

// One CTA per tile of columns of one local block.  Each thread keeps its own
// column of partial moments (compensated double-float accumulators) in shared
// memory, acc[l * blockDim + tid]; the columns are summed at the end
// (reduce_columns_add) and added to the block's moments.  TWO: a second real
// component (coefficients c2b, moments momb, accumulators after the first
// component's) shares each point's Chebyshev recurrence.
template <bool TWO>
__device__ __forceinline__ void local_moments_tile(const ProbParams* __restrict__ probs,
                                                   const LocalBlock* __restrict__ blks, const Tile t,
                                                   const float2* __restrict__ r2, const float2* __restrict__ c2,
                                                   double* __restrict__ mom, acc2* acc,
                                                   const float2* __restrict__ c2b = nullptr,
                                                   double* __restrict__ momb = nullptr)
{
    const LocalBlock B = blks[t.blk];
    const int L = probs[B.prob].L;
    const int odd = probs[B.prob].nu & 1;
    const int nt = blockDim.x, tid = threadIdx.x;
    acc2* accb = acc + (L + 1) * nt;
    for (int l = 0; l <= L; ++l) {
        acc[l * nt + tid] = acc2{0.f, 0.f};
        if (TWO) accb[l * nt + tid] = acc2{0.f, 0.f};
    }
    const df invR{B.iR_h, B.iR_l};
    // two points per step: two independent recurrences (a point beyond the
    // tile enters with c = 0)
    const int64_t jend = t.start + t.count;
    for (int64_t j = t.start + tid; j < jend; j += 2 * nt) {
        const int64_t jb = j + nt < jend ? j + nt : j;
        const float2 ra = r2[j], ca = c2[j], rb = r2[jb];
        const float2 cb = j + nt < jend ? c2[jb] : make_float2(0.f, 0.f);
        float2 da = make_float2(0.f, 0.f), db = da;
        if (TWO) {
            da = c2b[j];
            db = j + nt < jend ? c2b[jb] : make_float2(0.f, 0.f);
        }
        const df ya = df_mul(df{ra.x, ra.y}, invR), yb = df_mul(df{rb.x, rb.y}, invR);   // r_j / R in [0, 1]
        const df cja{ca.x, ca.y}, cjb{cb.x, cb.y}, dja{da.x, da.y}, djb{db.x, db.y};
        const df ua = df_add(df_mul(df{2.f * ya.h, 2.f * ya.l}, ya), df{-1.f, 0.f});   // T_2(y)
        const df ub = df_add(df_mul(df{2.f * yb.h, 2.f * yb.l}, yb), df{-1.f, 0.f});
        const df u2a{2.f * ua.h, 2.f * ua.l}, u2b{2.f * ub.h, 2.f * ub.l};
        // even: T_{2l}(y) = T_l(u); odd: T_{2l+1}(y) with T_1 = y, T_3 = y (2u - 1)
        df t0a = odd ? ya : df{1.f, 0.f}, t0b = odd ? yb : df{1.f, 0.f};
        df t1a = odd ? df_mul(ya, df_add(u2a, df{-1.f, 0.f})) : ua;
        df t1b = odd ? df_mul(yb, df_add(u2b, df{-1.f, 0.f})) : ub;
        acc_fma(acc[tid], cja, t0a);
        acc_fma(acc[tid], cjb, t0b);
        if (TWO) {
            acc_fma(accb[tid], dja, t0a);
            acc_fma(accb[tid], djb, t0b);
        }
        if (L >= 1) {
            acc_fma(acc[nt + tid], cja, t1a);
            acc_fma(acc[nt + tid], cjb, t1b);
            if (TWO) {
                acc_fma(accb[nt + tid], dja, t1a);
                acc_fma(accb[nt + tid], djb, t1b);
            }
        }
        for (int l = 2; l <= L; ++l) {
            const df t2a = cheb_step(u2a, t1a, t0a);
            const df t2b = cheb_step(u2b, t1b, t0b);
            acc2 a = acc[l * nt + tid];
            acc_fma(a, cja, t2a);
            acc_fma(a, cjb, t2b);
            acc[l * nt + tid] = a;
            if (TWO) {
                acc2 a2 = accb[l * nt + tid];
                acc_fma(a2, dja, t2a);
                acc_fma(a2, djb, t2b);
                accb[l * nt + tid] = a2;
            }
            t0a = t1a;
            t1a = t2a;
            t0b = t1b;
            t1b = t2b;
        }
    }
    __syncthreads();
    reduce_columns_add(acc, nt, L, Accum{mom, probs[B.prob].fxs}.at(B.mom_off));
    if (TWO) reduce_columns_add(accb, nt, L, Accum{momb, probs[B.prob].fxs}.at(B.mom_off));
}

__global__ void __launch_bounds__(kMomThreads)
k_local_moments(const ProbParams* __restrict__ probs, const LocalBlock* __restrict__ blks,
                const Tile* __restrict__ tiles, const float2* __restrict__ r2,
                const float2* __restrict__ c2, double* __restrict__ mom)
{
    extern __shared__ acc2 acc[];
    local_moments_tile<false>(probs, blks, tiles[blockIdx.x], r2, c2, mom, acc);
}

// A pair of real components in one pass (one recurrence per point for both).
__global__ void __launch_bounds__(kMomThreads)
k_local_moments2(const ProbParams* __restrict__ probs, const LocalBlock* __restrict__ blks,
                 const Tile* __restrict__ tiles, const float2* __restrict__ r2, const float2* __restrict__ c2,
                 const float2* __restrict__ c2b, double* __restrict__ mom, double* __restrict__ momb)
{
    extern __shared__ acc2 acc[];
    local_moments_tile<true>(probs, blks, tiles[blockIdx.x], r2, c2, mom, acc, c2b, momb);
}

// J_0..J_ntop(y), unnormalised, into this thread's column jb[n * nt + tid]
// (double-float); returns the normalisation S = J_0 + 2 sum_k J_2k of the same
// scale.  Miller's backward recurrence from ns (even), rescaled by 2^-60
// whenever a value passes 2^60.  Needs y >= 1 (growth per step <= 2 ns / y).
// Steps above both the highest order needed and the turning point (n > y)
// run in FP32: there the recurrence damps any perturbation relative to J_n
// (it acts like a change of the arbitrary start values), so only the steps
// that produce the returned values need double-float.
__device__ __forceinline__ int miller_fp32_floor(int ntop, float y)
{
    const int t = (int)(y + 8.f + 2.f * sqrtf(y)) + 1;
    return (t > ntop + 2 ? t : ntop + 2);
}

// FP32 steps of Miller's recurrence from ns down to (above) lo; returns the
// state (J_{i+1}, J_i, S) and the next index i.
__device__ __forceinline__ int miller_fp32_head(int ns, int lo, float ih, float* jp1, float* jc, float* S)
{
    float fp1 = 0.f, fc = 1.f, fS = 2.f;
    int i = ns;
    for (; i - 2 >= lo; i -= 2) {
        const float fm = fmaf((float)i * ih, fc, -fp1);
        const float fmm = fmaf((float)(i - 1) * ih, fm, -fc);
        fS = fmaf(2.f, fmm, fS);
        fp1 = fm;
        fc = fmm;
        if (fabsf(fc) > 1.152921504606847e18f) {
            const float sc = 8.673617379884035e-19f;   // 2^-60
            fc *= sc; fp1 *= sc; fS *= sc;
        }
    }
    *jp1 = fp1;
    *jc = fc;
    *S = fS;
    return i;
}

// One step J_{i-1} = (2i/y) J_i - J_{i+1} of Miller's recurrence in
// double-float, (ih, il) = 2/y: on entry (jh, jl) = J_i and (ph, pl) =
// J_{i+1}, on exit J_{i-1} and J_i.  A compensated multiply-subtract: the
// factor 2i/y and the product stay unevaluated (hi, lo) pairs and only the
// result is renormalised.
__device__ __forceinline__ void miller_step(int i, float ih, float il, float& jh, float& jl, float& ph, float& pl)
{
    const float fi = (float)i;
    const float th = fi * ih;
    const float tl = fmaf(fi, il, fmaf(fi, ih, -th));
    const float P = th * jh;
    const float Pe = fmaf(tl, jh, fmaf(th, jl, fmaf(th, jh, -P)));
    float sm, e;
    two_sum(P, -ph, sm, e);
    const df nj = fast_two_sum(sm, e + (Pe - pl));
    ph = jh;
    pl = jl;
    jh = nj.h;
    jl = nj.l;
}

// The double-float steps start from the FP32 head's state scaled near 1 (an
// exact power of two) and rescale by 2^-20 whenever a value passes 2^20 (the
// check runs every second step, whose growth is below 2^16, so values stay
// below 2^36): products of two stored values times a moment (below 2^33)
// then stay far inside the FP32 range without per-term scaling.  Each step J_{i-1} = (2i/y) J_i - J_{i+1} is one compensated
// multiply-subtract: the factor 2i/y and the product are kept as unevaluated
// (hi, lo) pairs and only the result is renormalised.  S, the normalisation,
// is a compensated FP32 sum.
__device__ __forceinline__ df miller_store_df(df y, int ntop, int ns, float2* jb, int nt, int tid)
{
    const df iy = df_recip(y);
    const float ih = 2.f * iy.h, il = 2.f * iy.l;   // 2 / y
    float f1, f0, fS;
    const int i0 = miller_fp32_head(ns, miller_fp32_floor(ntop, y.h), ih, &f1, &f0, &fS);
    const float s0 = ldexpf(1.f, -ilogbf(f0));
    float jh = f0 * s0, jl = 0.f, ph = f1 * s0, pl = 0.f;
    acc2 S{fS * s0, 0.f};
    if (i0 <= ntop) jb[i0 * nt + tid] = make_float2(jh, jl);
    auto step = [&](int i) { miller_step(i, ih, il, jh, jl, ph, pl); };
    for (int i = i0; i >= 2; i -= 2) {
        step(i);
        if (i - 1 <= ntop) jb[(i - 1) * nt + tid] = make_float2(jh, jl);
        step(i - 1);
        if (i - 2 <= ntop) jb[(i - 2) * nt + tid] = make_float2(jh, jl);
        float s2, e2;
        two_sum(S.s, 2.f * jh, s2, e2);
        S.s = s2;
        S.c += e2 + 2.f * jl;
        if (fabsf(jh) > 1048576.f) {
            const float sc = 9.5367431640625e-07f;   // 2^-20
            jh *= sc; jl *= sc; ph *= sc; pl *= sc; S.s *= sc; S.c *= sc;
            const int top = ntop < i0 ? ntop : i0;
            for (int q = i - 2; q <= top; ++q) {
                const float2 v = jb[q * nt + tid];
                jb[q * nt + tid] = make_float2(v.x * sc, v.y * sc);
            }
        }
    }
    // J_0 was added with weight 2; it counts once
    float s2, e2;
    two_sum(S.s, -jh, s2, e2);
    return fast_two_sum(s2, S.c + e2 - jl);
}

// 1 / k as double-float (k < 2^24, exact in FP32)
__device__ __forceinline__ df df_inv_int(int k) { return df_recip(df{(float)k, 0.f}); }

// J_n(x) for 0 <= x < 1 from the power series (DLMF 10.2.2) in double-float:
// (x/2)^n / n! times sum_k (-x^2/4)^k n! / (k! (n+k)!), summed until a term
// falls below 2^-53 of the sum (at most 9 terms: the ratio of consecutive
// terms is at most 1/(4 k (n+k))).  FP32-pipe arithmetic only (FP64 runs at
// 1/64 of the FP32 rate here); an (x/2)^n / n! below FP32's range gives 0,
// far below any tolerance.
// lead (x/2)^n / n! times the sum, q = -x^2/4
__device__ __forceinline__ df jn_series_sum(int n, df lead, df q)
{
    df term = lead, sum = lead;
    for (int k = 1; k <= 9; ++k) {
        term = df_mul(df_mul(term, q), df_inv_int(k * (n + k)));
        sum = df_add(sum, term);
        if (fabsf(term.h) <= 1.1102230246251565e-16f * fabsf(sum.h)) break;
    }
    return sum;
}

__device__ __forceinline__ df jn_series_df(int n, df x)
{
    const df h{0.5f * x.h, 0.5f * x.l};
    df lead{1.f, 0.f};
    for (int i = 1; i <= n && lead.h != 0.f; ++i) lead = df_mul(df_mul(lead, h), df_inv_int(i));
    return jn_series_sum(n, lead, df_neg(df_mul(h, h)));
}

// The same series in FP32 (mixed precision): six terms reach 1e-9 relative.
__device__ __forceinline__ float jn_series_f32(int n, float x)
{
    const float h = 0.5f * x;
    float lead = 1.f;
    for (int i = 1; i <= n && lead != 0.f; ++i) lead *= h / (float)i;
    const float q = -h * h;
    float term = lead, sum = lead;
    for (int k = 1; k <= 6; ++k) {
        term *= q / (float)(k * (n + k));
        sum += term;
    }
    return sum;
}

// Small arguments (y < 1): J_0..J_ntop(y) directly from the power series, in
// double-float; already normalised (returns 1).
__device__ __forceinline__ df series_store_df(df y, int ntop, float2* jb, int nt, int tid)
{
    const df h{0.5f * y.h, 0.5f * y.l};
    const df q = df_neg(df_mul(h, h));
    df lead{1.f, 0.f};   // (y/2)^n / n!
    for (int n = 0; n <= ntop; ++n) {
        if (n > 0 && lead.h != 0.f) lead = df_mul(df_mul(lead, h), df_inv_int(n));
        const df v = lead.h != 0.f ? jn_series_sum(n, lead, q) : df{0.f, 0.f};
        jb[n * nt + tid] = make_float2(v.h, v.l);
    }
    return df{1.f, 0.f};
}

// nu = 0: sum_l sgn_l J_l(y)^2 mu_l (and the same with mub) accumulated while
// Miller's backward recurrence produces J_l, l <= L, without storing them:
// the steps, the start and the rescaling of miller_store_df; a rescale by
// 2^-20 scales the sums of squares by 2^-40.  Returns S (unnormalised
// values, as miller_store_df).
__device__ __forceinline__ df miller_sum_nu0(df y, int L, int ns, const float2* mu, const float2* mub, bool two,
                                            acc2* sum, acc2* sumb)
{
    const df iy = df_recip(y);
    const float ih = 2.f * iy.h, il = 2.f * iy.l;   // 2 / y
    float f1, f0, fS;
    const int i0 = miller_fp32_head(ns, miller_fp32_floor(L, y.h), ih, &f1, &f0, &fS);
    const float s0 = ldexpf(1.f, -ilogbf(f0));
    float jh = f0 * s0, jl = 0.f, ph = f1 * s0, pl = 0.f;
    acc2 S{fS * s0, 0.f};
    acc2 A{0.f, 0.f}, Ab{0.f, 0.f};
    auto take = [&](int l) {
        if (l <= L) {
            const float p = jh * jh;
            const float e = fmaf(2.f * jh, jl, fmaf(jh, jh, -p));
            acc_fma(A, df{p, e}, df{mu[l].x, mu[l].y});
            if (two) acc_fma(Ab, df{p, e}, df{mub[l].x, mub[l].y});
        }
    };
    auto step = [&](int i) { miller_step(i, ih, il, jh, jl, ph, pl); };
    take(i0);
    for (int i = i0; i >= 2; i -= 2) {
        step(i);
        take(i - 1);
        step(i - 1);
        take(i - 2);
        float s2, e2;
        two_sum(S.s, 2.f * jh, s2, e2);
        S.s = s2;
        S.c += e2 + 2.f * jl;
        if (fabsf(jh) > 1048576.f) {
            const float sc = 9.5367431640625e-07f;    // 2^-20
            const float sc2 = 9.094947017729282e-13f; // 2^-40
            jh *= sc; jl *= sc; ph *= sc; pl *= sc; S.s *= sc; S.c *= sc;
            A.s *= sc2; A.c *= sc2; Ab.s *= sc2; Ab.c *= sc2;
        }
    }
    *sum = A;
    *sumb = Ab;
    float s2, e2;
    two_sum(S.s, -jh, s2, e2);
    return fast_two_sum(s2, S.c + e2 - jl);
}

// nu = 0, y < 1: the same sums from the power series values (normalised).
__device__ __forceinline__ void series_sum_nu0(df y, int L, const float2* mu, const float2* mub, bool two,
                                               acc2* sum, acc2* sumb)
{
    const df h{0.5f * y.h, 0.5f * y.l};
    const df q = df_neg(df_mul(h, h));
    df lead{1.f, 0.f};   // (y/2)^n / n!
    acc2 A{0.f, 0.f}, Ab{0.f, 0.f};
    for (int n = 0; n <= L && lead.h != 0.f; ++n) {
        if (n > 0) lead = df_mul(df_mul(lead, h), df_inv_int(n));
        if (lead.h == 0.f) break;
        const df v = jn_series_sum(n, lead, q);
        const float p = v.h * v.h;
        const float e = fmaf(2.f * v.h, v.l, fmaf(v.h, v.h, -p));
        acc_fma(A, df{p, e}, df{mu[n].x, mu[n].y});
        if (two) acc_fma(Ab, df{p, e}, df{mub[n].x, mub[n].y});
    }
    *sum = A;
    *sumb = Ab;
}

// One thread per row of a local block.  J_0..J_ntop(x/2) by Miller's backward
// recurrence, kept (unnormalised) in this thread's column of shared memory,
// then sum_l C_l mu_l divided by the square of the normalisation.  With momb
// (the moments of a second real component) the same C_l also give
// sum_l C_l mub_l into g_sb.
// coherent: read the moments past L1 (they were just written by other CTAs
// of the same launch, the persistent local kernel)
__device__ __forceinline__ void local_eval_tile(const ProbParams* __restrict__ probs,
                                                const LocalBlock* __restrict__ blks, const Tile t,
                                                const float2* __restrict__ w2, const double* mom,
                                                double* __restrict__ g_s, const double* momb,
                                                double* __restrict__ g_sb, float2* sm2, bool coherent)
{
    const LocalBlock B = blks[t.blk];
    const ProbParams& P = probs[B.prob];
    const int nt = blockDim.x, tid = threadIdx.x;
    const int nu = P.nu, L = P.L;
    const bool two = momb != nullptr;
    float2* mu = sm2;                 // [L + 1] moments of this block, double-float
    float2* mub = sm2 + (P.ntop + 1); // [L + 1] the second component's (two)
    float2* jb = sm2 + (two ? 2 : 1) * (P.ntop + 1);  // [ntop + 1][nt]
    const int hp = (nu & 1) ? (nu + 1) / 2 : nu / 2;   // index paired with +l
    const int hm = (nu & 1) ? (nu - 1) / 2 : nu / 2;   // index paired with -l
    // the moments times the sign and weight of their term: C_l = sgn_l J_{hp+l} J_{|hm-l|},
    // sgn_l = (-1 for an odd negative index hm - l) (2 unless l = 0 and nu is even)
    for (int l = tid; l <= L; l += nt) {
        const int b = hm - l;
        float sgn = (b < 0 && ((-b) & 1)) ? -1.f : 1.f;
        if (l > 0 || (nu & 1)) sgn *= 2.f;
        const double v = coherent ? __ldcg(&mom[B.mom_off + l]) : mom[B.mom_off + l];
        const float h = (float)v;
        mu[l] = make_float2(sgn * h, sgn * (float)(v - (double)h));
        if (two) {
            const double vb = coherent ? __ldcg(&momb[B.mom_off + l]) : momb[B.mom_off + l];
            const float hb = (float)vb;
            mub[l] = make_float2(sgn * hb, sgn * (float)(vb - (double)hb));
        }
    }
    __syncthreads();
    if (tid >= t.count) return;
    const int64_t k = t.start + tid;
    const float2 wk = w2[k];
    const df ydf = df_mul(df{wk.x, wk.y}, df{0.5f * B.R_h, 0.5f * B.R_l});   // y = omega R / 2
    double val, valb = 0.0;
    if (!(ydf.h > 0.f)) {
        // y below the FP32 range: J_n(y) = delta_n0 to far below rounding, so
        // only C_0 survives, and only for nu = 0
        val = (nu == 0) ? (double)mu[0].x + (double)mu[0].y : 0.0;
        if (two) valb = (nu == 0) ? (double)mub[0].x + (double)mub[0].y : 0.0;
    } else {
        const int ntop = hp + L;
        const int ns = miller_start(ntop, (double)ydf.h);
        df S{1.f, 0.f};
        acc2 sum{0.f, 0.f}, sumb{0.f, 0.f};
        if (nu == 0) {
            // C_l = sgn_l J_l^2, summed as the values are made (no column)
            if (ydf.h >= 1.f)
                S = miller_sum_nu0(ydf, L, ns, mu, mub, two, &sum, &sumb);
            else
                series_sum_nu0(ydf, L, mu, mub, two, &sum, &sumb);
        } else if (ydf.h >= 1.f) {
            S = miller_store_df(ydf, ntop, ns, jb, nt, tid);
        } else {
            S = series_store_df(ydf, ntop, jb, nt, tid);
        }
        // The stored values stay below 2^36 and the signed moments below 2^33
        // (inputs scaled below 2, at most 2^31 points), so the products
        // J_a J_b mu_l (each an unevaluated (hi, lo) pair) and their sums stay
        // inside the FP32 range; S^2 is divided out at the end.
        if (nu != 0) {
            for (int l = 0; l <= L; ++l) {
                const int b = hm - l;
                const float2 va = jb[(hp + l) * nt + tid];
                const float2 vb = jb[(b >= 0 ? b : -b) * nt + tid];
                const float p = va.x * vb.x;
                const float e = fmaf(va.y, vb.x, fmaf(va.x, vb.y, fmaf(va.x, vb.x, -p)));
                acc_fma(sum, df{p, e}, df{mu[l].x, mu[l].y});
                if (two) acc_fma(sumb, df{p, e}, df{mub[l].x, mub[l].y});
            }
        }
        const df iS = df_recip(S);
        val = df_to(df_mul(df_mul(fast_two_sum(sum.s, sum.c), iS), iS));
        if (two) valb = df_to(df_mul(df_mul(fast_two_sum(sumb.s, sumb.c), iS), iS));
    }
    Accum{g_s, P.fxs}.add(k, (double)P.sgn * val);
    if (two) Accum{g_sb, P.fxs}.add(k, (double)P.sgn * valb);
}

__global__ void k_local_eval(const ProbParams* __restrict__ probs, const LocalBlock* __restrict__ blks,
                             const Tile* __restrict__ tiles, const float2* __restrict__ w2,
                             const double* __restrict__ mom, double* __restrict__ g_s,
                             const double* __restrict__ momb, double* __restrict__ g_sb)
{
    extern __shared__ float2 sm2[];
    local_eval_tile(probs, blks, tiles[blockIdx.x], w2, mom, g_s, momb, g_sb, sm2, false);
}

// Persistent local stage: one launch of resident CTAs takes work items from a
// device queue (q[0], an atomic counter): first every moment tile (of each
// component), then every evaluation tile.  An evaluation tile of block b
// waits until all of b's moment tiles are done (q[2 + b] counts them): the
// items it waits for were taken from the queue before it by CTAs that are
// running and wait on nothing, so the wait always ends; it is still bounded
// by wait_limit polls, after which the CTA records NUHT_ERR_TIMEOUT in
// *status, skips the tile and goes on, so the launch always finishes.
// stall (testing aid) asks block 0 for one moment tile more than it has.
__global__ void __launch_bounds__(kMomThreads)
k_local_persistent(const ProbParams* __restrict__ probs, const LocalBlock* __restrict__ blks,
                   const Tile* __restrict__ tmom, int n_tmom, const Tile* __restrict__ teval, int n_teval,
                   const int32_t* __restrict__ mom_pre, const float2* __restrict__ r2,
                   const float2* __restrict__ c2, const float2* __restrict__ c2b, const float2* __restrict__ w2,
                   double* mom, double* momb, double* __restrict__ g_s, double* __restrict__ g_sb, int* q,
                   int* status, int wait_limit, int stall)
{
    extern __shared__ float4 smq[];
    __shared__ int item, give_up;
    const int ncomp = momb ? 2 : 1;
    const int nmom = ncomp * n_tmom, total = nmom + n_teval;
    int* done = q + 2;
    for (;;) {
        if (threadIdx.x == 0) item = atomicAdd(&q[0], 1);
        __syncthreads();
        const int it = item;
        if (it >= total) break;
        if (it < nmom) {
            const int comp = it >= n_tmom ? 1 : 0;
            const Tile t = tmom[it - comp * n_tmom];
            local_moments_tile<false>(probs, blks, t, r2, comp ? c2b : c2, comp ? momb : mom, (acc2*)smq);
            __threadfence();   // the moments' atomics before the count
            __syncthreads();
            if (threadIdx.x == 0) atomicAdd(&done[t.blk], 1);
        } else {
            const Tile t = teval[it - nmom];
            if (threadIdx.x == 0) {
                const int need = ncomp * (mom_pre[t.blk + 1] - mom_pre[t.blk]) + (stall && t.blk == 0 ? 1 : 0);
                int polls = 0;
                give_up = 0;
                while (*(volatile int*)&done[t.blk] < need) {
                    if (++polls > wait_limit) {
                        atomicCAS(status, 0, NUHT_ERR_TIMEOUT);
                        give_up = 1;
                        break;
                    }
                    __nanosleep(128);
                }
                __threadfence();
            }
            __syncthreads();
            if (!give_up) local_eval_tile(probs, blks, t, w2, mom, g_s, momb, g_sb, (float2*)smq, true);
        }
        __syncthreads();   // item and the shared buffers are reused by the next item
    }
}

// Mixed precision (eps >= 1e-6): k_local_eval in FP32.  J_0..J_ntop(y) by
// Miller's recurrence in FP32 (rescaled by 2^-60 when a value passes 2^60,
// the stored ones with it), normalised by S = J_0 + 2 sum_k J_2k, then
// sum_l C_l mu_l with FP32 products.  The recurrence and the products round
// at ~1e-6 relative, and |C_l| <= 2 with sum over a row's local blocks of
// |mu_l| <= ||c||_1 (disjoint columns): a few 1e-6 ||c||_1, inside
// 10 eps ||c||_1.  y below 1e-7 keeps J_n = delta_n0 (J_1(y) < 5e-8); above
// it two steps grow a value by at most (2 ns / y)^2 < 2^60, so with the rescale
// at 2^60 nothing passes 2^121.
__global__ void k_local_eval_f32(const ProbParams* __restrict__ probs, const LocalBlock* __restrict__ blks,
                                 const Tile* __restrict__ tiles, const float2* __restrict__ w2,
                                 const double* __restrict__ mom, double* __restrict__ g_s,
                                 const double* __restrict__ momb, double* __restrict__ g_sb)
{
    extern __shared__ float smf[];
    const Tile t = tiles[blockIdx.x];
    const LocalBlock B = blks[t.blk];
    const ProbParams& P = probs[B.prob];
    const int nt = blockDim.x, tid = threadIdx.x;
    const int nu = P.nu, L = P.L;
    const bool two = momb != nullptr;
    float* mu = smf;                   // [L + 1]
    float* mub = smf + (P.ntop + 1);   // [L + 1] the second component's (two)
    float* jb = smf + (two ? 2 : 1) * (P.ntop + 1);    // [ntop + 1][nt]
    for (int l = tid; l <= L; l += nt) {
        mu[l] = (float)mom[B.mom_off + l];
        if (two) mub[l] = (float)momb[B.mom_off + l];
    }
    __syncthreads();
    if (tid >= t.count) return;
    const int64_t k = t.start + tid;
    const float y = w2[k].x * (0.5f * B.R_h);   // omega R / 2
    const int hp = (nu & 1) ? (nu + 1) / 2 : nu / 2;
    const int hm = (nu & 1) ? (nu - 1) / 2 : nu / 2;
    const int ntop = hp + L;
    float val = 0.f, valb = 0.f;
    if (!(y >= 1e-7f)) {
        if (nu == 0) {
            val = mu[0];
            if (two) valb = mub[0];
        }
    } else {
        const int ns = miller_start(ntop, (double)y);
        const float inv2y = 2.f / y;
        float jp1 = 0.f, jc = 1.f, S = 2.f;
        if (ns <= ntop) jb[ns * nt + tid] = jc;
        for (int i = ns; i >= 2; i -= 2) {
            const float jm = fmaf((float)i * inv2y, jc, -jp1);
            const float jmm = fmaf((float)(i - 1) * inv2y, jm, -jc);
            if (i - 1 <= ntop) jb[(i - 1) * nt + tid] = jm;
            if (i - 2 <= ntop) jb[(i - 2) * nt + tid] = jmm;
            S = fmaf(2.f, jmm, S);
            jp1 = jm;
            jc = jmm;
            if (fabsf(jc) > 1.152921504606847e18f) {
                const float sc = 8.673617379884035e-19f;   // 2^-60
                jc *= sc; jp1 *= sc; S *= sc;
                for (int q = i - 2; q <= ntop; ++q) jb[q * nt + tid] *= sc;
            }
        }
        const float iS = 1.f / (S - jc);   // J_0 was added with weight 2; it counts once
        for (int l = 0; l <= L; ++l) {
            const int b = hm - l;
            const float va = jb[(hp + l) * nt + tid] * iS;
            const float vb = jb[(b >= 0 ? b : -b) * nt + tid] * iS;
            float sgn = (b < 0 && ((-b) & 1)) ? -1.f : 1.f;
            if (l > 0 || (nu & 1)) sgn *= 2.f;
            const float cl = va * vb * sgn;
            val = fmaf(cl, mu[l], val);
            if (two) valb = fmaf(cl, mub[l], valb);
        }
    }
    Accum{g_s, P.fxs}.add(k, (double)(P.sgn < 0 ? -val : val));
    if (two) Accum{g_sb, P.fxs}.add(k, (double)(P.sgn < 0 ? -valb : valb));
}

// J_n(x) for 1 <= x by Miller's recurrence in double-float (no storage).
__device__ __forceinline__ double jn_miller_df(int n, double x)
{
    const int ns = miller_start(n, x);
    const double inv2x = 2.0 / x;
    const float ih = (float)inv2x, il = (float)(inv2x - (double)ih);
    float f1, f0, fS;
    const int i0 = miller_fp32_head(ns, miller_fp32_floor(n, (float)x), ih, &f1, &f0, &fS);
    df jp1{f1, 0.f}, jc{f0, 0.f}, S{fS, 0.f}, res{0.f, 0.f};
    for (int i = i0; i >= 2; i -= 2) {
        const df jm = df_add(df_mul(df_imul((float)i, ih, il), jc), df_neg(jp1));
        const df jmm = df_add(df_mul(df_imul((float)(i - 1), ih, il), jm), df_neg(jc));
        if (i - 1 == n) res = jm;
        if (i - 2 == n) res = jmm;
        S = df_add(S, df{2.f * jmm.h, 2.f * jmm.l});
        jp1 = jm;
        jc = jmm;
        if (df_big(jc)) {
            const float sc = 8.673617379884035e-19f;   // 2^-60
            jc = df_scale(jc, sc); jp1 = df_scale(jp1, sc); S = df_scale(S, sc); res = df_scale(res, sc);
        }
    }
    S = df_add(S, df_neg(jc));
    return df_to(res) / df_to(S);
}

// Hankel's expansion (Sec. 3.2, M pairs) at the exact product x = w r in
// double-float: the phase x mod pi/2 is reduced in FP64 (df_sincos_prod),
// 1/x, the two series in 1/x^2 and the amplitude sqrt(2/(pi x)) in double-float.
__device__ __forceinline__ double jn_hankel_df(const ProbParams& P, double w, double r)
{
    const double p = w * r;
    const double e = fma(w, r, -p);
    const float ph = (float)p;
    const df x = fast_two_sum(ph, (float)(p - (double)ph) + (float)e);
    const df y = df_recip(x);
    // the series in u = z / x (< 1) with the coefficients a_q z^-q
    const df u = df_mul(y, df{P.z2.x, P.z2.y});
    const df u2 = df_mul(u, u);
    df pp{0.f, 0.f}, qq{0.f, 0.f};
    for (int l = P.M - 1; l >= 0; --l) {
        const float2 a0 = P.a2[2 * l], a1 = P.a2[2 * l + 1];
        const bool neg = l & 1;
        pp = df_add(df_mul(pp, u2), neg ? df{-a0.x, -a0.y} : df{a0.x, a0.y});
        qq = df_add(df_mul(qq, u2), neg ? df{-a1.x, -a1.y} : df{a1.x, a1.y});
    }
    qq = df_mul(qq, u);
    df sx, cx;
    df_sincos_prod(w, r, &sx, &cx);
    const df cph{P.cphi2.x, P.cphi2.y}, sph{P.sphi2.x, P.sphi2.y};
    const df cchi = df_add(df_mul(cx, cph), df_negate(df_mul(sx, sph)));   // cos(x + phi)
    const df schi = df_add(df_mul(sx, cph), df_mul(cx, sph));              // sin(x + phi)
    const df amp = df_sqrt(df_mul(df{0.6366197466850281f, 2.5682552973194106e-08f}, y));   // sqrt(2 / (pi x))
    return df_to(df_mul(amp, df_add(df_mul(pp, cchi), df_negate(df_mul(qq, schi)))));
}

// Direct entries in a fixed-point frame per direct block: Om = omega 2^fw and
// R = r 2^fr are integers below 2^62, so P = Om R = omega r 2^(fw + fr) is
// exact in 128 bits.  x = omega r comes from its top bits as double-float and
// the phase omega r / (2 pi) in turns from bits of P * round(2^64 / (2 pi)),
// all with integer instructions (FP64 runs at 1/64 of the FP32 rate here).
struct DirFx {
    int fr, fw;
};

// (hi 2^64 + lo) 2^-s as double-float (relative 2^-48); 0 for 0.
__device__ __forceinline__ df df_from_u128(unsigned long long hi, unsigned long long lo, int s)
{
    if (hi == 0 && lo == 0) return df{0.f, 0.f};
    const int lz = hi ? __clzll((long long)hi) : 64 + __clzll((long long)lo);
    unsigned long long t;
    if (lz == 0) t = hi;
    else if (lz < 64) t = (hi << lz) | (lo >> (64 - lz));
    else t = lo << (lz - 64);
    const int e = 64 - lz - s;   // value = t 2^e
    const float h = ldexpf((float)(unsigned)(t >> 40), e + 40);
    const float l = ldexpf((float)(unsigned)((t >> 16) & 0xFFFFFF), e + 16);
    return fast_two_sum(h, l);
}

// The fraction of a turn of P 2^-s / (2 pi) in 64-bit fixed point, 64 <= s <= 127.
__device__ __forceinline__ unsigned long long turns_u128(unsigned long long Ph, unsigned long long Pl, int s)
{
    const unsigned long long C = 2935890503282001226ULL;   // round(2^64 / (2 pi))
    const unsigned long long a_lo = Ph * C, a_hi = __umul64hi(Ph, C);
    const unsigned long long b_hi = __umul64hi(Pl, C);
    const int t = s - 64;
    const unsigned long long A = t == 0 ? a_lo : (a_hi << (64 - t)) | (a_lo >> t);
    return A + (b_hi >> t);
}

// jn_hankel_df with x = omega r given as double-float and its phase in turns.
__device__ __forceinline__ df jn_hankel_dfx(const ProbParams& P, df x, unsigned long long turns)
{
    const df y = df_recip(x);
    const df u = df_mul(y, df{P.z2.x, P.z2.y});
    const df u2 = df_mul(u, u);
    df pp{0.f, 0.f}, qq{0.f, 0.f};
    for (int l = P.M - 1; l >= 0; --l) {
        const float2 a0 = P.a2[2 * l], a1 = P.a2[2 * l + 1];
        const bool neg = l & 1;
        pp = df_add(df_mul(pp, u2), neg ? df{-a0.x, -a0.y} : df{a0.x, a0.y});
        qq = df_add(df_mul(qq, u2), neg ? df{-a1.x, -a1.y} : df{a1.x, a1.y});
    }
    qq = df_mul(qq, u);
    df sx, cx;
    df_sincos_turns_tab(turns, P.tw2, &sx, &cx);
    const df cph{P.cphi2.x, P.cphi2.y}, sph{P.sphi2.x, P.sphi2.y};
    const df cchi = df_add(df_mul(cx, cph), df_negate(df_mul(sx, sph)));   // cos(x + phi)
    const df schi = df_add(df_mul(sx, cph), df_mul(cx, sph));              // sin(x + phi)
    const df amp = df_sqrt(df_mul(df{0.6366197466850281f, 2.5682552973194106e-08f}, y));   // sqrt(2 / (pi x))
    return df_mul(amp, df_add(df_mul(pp, cchi), df_negate(df_mul(qq, schi))));
}

// jn_miller_df with x >= 1 given as double-float (no FP64 divisions).
__device__ __forceinline__ df jn_miller_dfx(int n, df x)
{
    const float xf = x.h;
    const float a = xf + 20.f + 4.f * sqrtf(xf);
    int ns = (int)a + 1;
    if (ns < n + 8) ns = n + 8;
    ns += ns & 1;
    const df i2 = df_recip(df{0.5f * x.h, 0.5f * x.l});   // 2 / x
    const float ih = i2.h, il = i2.l;
    float f1, f0, fS;
    const int i0 = miller_fp32_head(ns, miller_fp32_floor(n, xf), ih, &f1, &f0, &fS);
    // compensated steps from the head's state (as miller_store_df), keeping J_n
    float jh = f0, jl = 0.f, ph = f1, pl = 0.f;
    acc2 S{fS, 0.f};
    df res{0.f, 0.f};
    for (int i = i0; i >= 2; i -= 2) {
        miller_step(i, ih, il, jh, jl, ph, pl);
        if (i - 1 == n) res = df{jh, jl};
        miller_step(i - 1, ih, il, jh, jl, ph, pl);
        if (i - 2 == n) res = df{jh, jl};
        float s2, e2;
        two_sum(S.s, 2.f * jh, s2, e2);
        S.s = s2;
        S.c += e2 + 2.f * jl;
        if (fabsf(jh) > 1.152921504606847e18f) {
            const float sc = 8.673617379884035e-19f;   // 2^-60
            jh *= sc; jl *= sc; ph *= sc; pl *= sc; S.s *= sc; S.c *= sc; res = df_scale(res, sc);
        }
    }
    float s2, e2;
    two_sum(S.s, -jh, s2, e2);   // J_0 was added with weight 2; it counts once
    return df_mul(res, df_recip(fast_two_sum(s2, S.c + e2 - jl)));
}

// J_nu at the exact product w*r: asymptotic side (Hankel in double-float, or
// FP32 when lowp) or local side (series; Miller in double-float, or FP32 when lowp).
__device__ __forceinline__ double direct_entry(const ProbParams& P, double w, double r, bool asy, bool lowp)
{
    if (asy) return lowp ? (double)jn_hankel_f32(P, w, r) : jn_hankel_df(P, w, r);
    const double x = w * r;
    if (x < 1.0) return lowp ? (double)jn_series_f32(P.nu, (float)x) : df_to(jn_series_df(P.nu, df_from(x)));
    return lowp ? (double)jn_miller_f32(P.nu, (float)x) : jn_miller_df(P.nu, x);
}

// jn_hankel_f32 with x = omega r in FP32 and its phase in turns.
__device__ __forceinline__ float jn_hankel_f32x(const ProbParams& P, float x, unsigned long long turns)
{
    float sx, cx;
    f32_sincos_turns(turns, &sx, &cx);
    const float y = 1.f / x;
    const float u = y * P.z2.x, u2 = u * u;   // z / x < 1, with the coefficients a_q z^-q
    float pp = 0.f, qq = 0.f;
    for (int l = P.M - 1; l >= 0; --l) {
        const float sg = (l & 1) ? -1.f : 1.f;
        pp = fmaf(pp, u2, sg * P.a2[2 * l].x);
        qq = fmaf(qq, u2, sg * P.a2[2 * l + 1].x);
    }
    qq *= u;
    const float cph = P.cphi2.x, sph = P.sphi2.x;
    const float cchi = cx * cph - sx * sph, schi = sx * cph + cx * sph;
    return sqrtf(0.6366197723675814f * y) * (pp * cchi - qq * schi);
}

// jn_miller_f32 with the start index from FP32 x (no FP64).
__device__ __forceinline__ float jn_miller_f32x(int n, float x)
{
    const float a = x + 20.f + 4.f * sqrtf(x);
    int ns = (int)a + 1;
    if (ns < n + 8) ns = n + 8;
    ns += ns & 1;
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
            const float sc = 8.673617379884035e-19f;   // 2^-60
            jc *= sc; jp1 *= sc; S *= sc; res *= sc;
        }
    }
    return res / (S - jc);
}

// direct_entry in the block's fixed-point frame; the series for x < 1 as in
// direct_entry.
__device__ __forceinline__ df direct_entry_df(const ProbParams& P, DirFx F, double w, double r, bool asy,
                                              bool lowp)
{
    const int s = F.fr + F.fw;
    // the phase in turns needs s <= 127; x alone (local side) any s >= 64
    if (s < 64 || (asy && s > 127)) return df_from(direct_entry(P, w, r, asy, lowp));
    const unsigned long long Om = (unsigned long long)fx_from_double(w, F.fw);
    const unsigned long long R = (unsigned long long)fx_from_double(r, F.fr);
    const unsigned long long Pl = Om * R, Ph = __umul64hi(Om, R);
    const df x = df_from_u128(Ph, Pl, s);
    if (asy) return lowp ? df{jn_hankel_f32x(P, x.h, turns_u128(Ph, Pl, s)), 0.f}
                         : jn_hankel_dfx(P, x, turns_u128(Ph, Pl, s));
    if (x.h < 1.f) return lowp ? df{jn_series_f32(P.nu, x.h), 0.f} : jn_series_df(P.nu, x);
    return lowp ? df{jn_miller_f32x(P.nu, x.h), 0.f} : jn_miller_dfx(P.nu, x);
}

__device__ __forceinline__ double direct_entry_fx(const ProbParams& P, DirFx F, double w, double r, bool asy,
                                                  bool lowp)
{
    return df_to(direct_entry_df(P, F, w, r, asy, lowp));
}

// direct_entry_fx for lowp as an FP32 value (no FP64 beyond the rare series).
__device__ __forceinline__ float direct_entry_f32x(const ProbParams& P, DirFx F, double w, double r, bool asy)
{
    const int s = F.fr + F.fw;
    if (s < 64 || (asy && s > 127)) return (float)direct_entry(P, w, r, asy, true);
    const unsigned long long Om = (unsigned long long)fx_from_double(w, F.fw);
    const unsigned long long R = (unsigned long long)fx_from_double(r, F.fr);
    const unsigned long long Pl = Om * R, Ph = __umul64hi(Om, R);
    const df x = df_from_u128(Ph, Pl, s);
    if (asy) return jn_hankel_f32x(P, x.h, turns_u128(Ph, Pl, s));
    if (x.h < 1.f) return jn_series_f32(P.nu, x.h);
    return jn_miller_f32x(P.nu, x.h);
}

// The fixed-point frame of a direct block: r < 2^(62 - fr), omega < 2^(62 - fw).
__device__ __forceinline__ DirFx direct_frame(const double* __restrict__ r_s, const double* __restrict__ w_s,
                                              const DirectBlock& B)
{
    int er, ew;
    frexp(r_s[B.j1], &er);
    frexp(w_s[B.k1], &ew);
    return DirFx{62 - er, 62 - ew};
}

// Division of an entry index by the block's column count with one wide
// multiply: m = ceil(2^32 / d) gives floor(e m / 2^32) = floor(e / d) exactly
// whenever e d < 2^32 (direct blocks hold at most a few thousand entries).
struct ColDiv {
    unsigned long long m;
    __device__ __forceinline__ explicit ColDiv(int d) : m(((1ull << 32) + (unsigned)d - 1) / (unsigned)d) {}
    __device__ __forceinline__ int operator()(int e) const { return (int)(((unsigned long long)(unsigned)e * m) >> 32); }
};

// Splits the entries of a direct block into a local list (omega r <= z, from
// the front) and an asymptotic list (from the back) in shared memory, so that
// warps run one branch each.  The split uses the FP32 parts of omega and r
// (either branch is accurate to eps near the crossover) and one counter update
// per warp and list.  Returns the number of local entries.  blockDim is a
// multiple of 32.
__device__ __forceinline__ int direct_partition(const ProbParams& P, const DirectBlock& B, int cols, int area,
                                                const float2* __restrict__ r2, const float2* __restrict__ w2,
                                                int* list, int* cnt, bool colmajor = false)
{
    // entry e is (row e / cols, column e % cols), or with colmajor (row e % rows,
    // column e / rows)
    const int rows = area / cols;
    if (threadIdx.x == 0) { cnt[0] = 0; cnt[1] = 0; }
    __syncthreads();
    const float zf = (float)P.z;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int area_pad = (area + 31) & ~31;
    const ColDiv div(colmajor ? rows : cols);
    for (int e = threadIdx.x; e < area_pad; e += blockDim.x) {
        const bool valid = e < area;
        bool asy = false;
        if (valid) {
            int rr, cc;
            if (colmajor) {
                cc = div(e);
                rr = e - cc * rows;
            } else {
                rr = div(e);
                cc = e - rr * cols;
            }
            asy = w2[B.k0 + rr].x * r2[B.j0 + cc].x > zf;
        }
        const unsigned ma = __ballot_sync(0xffffffffu, valid && asy);
        const unsigned ml = __ballot_sync(0xffffffffu, valid && !asy);
        int ba = 0, bl = 0;
        if (lane == 0) {
            if (ma) ba = atomicAdd(&cnt[1], __popc(ma));
            if (ml) bl = atomicAdd(&cnt[0], __popc(ml));
        }
        ba = __shfl_sync(0xffffffffu, ba, 0);
        bl = __shfl_sync(0xffffffffu, bl, 0);
        if (valid) {
            if (asy) list[area - 1 - (ba + __popc(ma & lt))] = e;
            else list[bl + __popc(ml & lt)] = e;
        }
    }
    __syncthreads();
    return cnt[0];
}

// One CTA per direct block (area <= min_size): entries in parallel after the
// branch split, row sums in shared memory, then one atomic add per row.
// mode 0: double-float entries, FP64 row sums.  mode 1 (eps >= 1e-6): FP32
// entries, FP64 row sums.  mode 2: FP32 entries whose products with the FP32
// parts of c accumulate in FP32 atomics, each row spread over S = kDirSlots
// slots (fewer when S rows > kDirSlotFloats) by list position, the slots of a
// row then summed by a warp in compensated FP32 (direct_sum_mode picks it when
// its rounding bound fits the tolerance).  With g_sb set, every entry is also applied to a second
// coefficient vector (c_sb, c2b) into g_sb: the entries are evaluated once for
// both (the two real components of complex c, or two vectors).
constexpr int kDirSlots = 32;
constexpr int kDirSlotFloats = 4096;

__global__ void k_direct(const ProbParams* __restrict__ probs, const DirectBlock* __restrict__ blks,
                         const double* __restrict__ r_s, const double* __restrict__ w_s,
                         const float2* __restrict__ r2, const float2* __restrict__ w2,
                         const double* __restrict__ c_s, const float2* __restrict__ c2, double* __restrict__ g_s,
                         const double* __restrict__ c_sb, const float2* __restrict__ c2b, double* __restrict__ g_sb,
                         int mode, int det)
{
    // per vector: [rows] FP64 row sums or [rows][S] FP32 slots (mode 2); none in
    // the deterministic mode (never mode 2), where every entry's product goes
    // straight into the exact fixed-point sums of g
    extern __shared__ double rowacc[];
    __shared__ int cnt[2];
    const bool two = g_sb != nullptr;
    const DirectBlock B = blks[blockIdx.x];
    const ProbParams& P = probs[B.prob];
    const int rows = B.k1 - B.k0 + 1, cols = B.j1 - B.j0 + 1;
    const ColDiv cdiv(cols);
    const int area = rows * cols;
    int S = kDirSlots;
    while (S > 1 && S * rows > kDirSlotFloats) S >>= 1;
    const int accd = det ? 0 : (mode == 2 ? kDirSlotFloats / 2 : rows);   // doubles per vector
    double* rowaccb = rowacc + accd;
    float* rowf = (float*)rowacc;
    float* rowfb = (float*)rowaccb;
    int* list = (int*)(rowacc + (two ? 2 : 1) * accd);
    if (mode == 2) {
        for (int i = threadIdx.x; i < S * rows; i += blockDim.x) {
            rowf[i] = 0.f;
            if (two) rowfb[i] = 0.f;
        }
    } else {
        for (int i = threadIdx.x; i < accd; i += blockDim.x) {
            rowacc[i] = 0.0;
            if (two) rowaccb[i] = 0.0;
        }
    }
    const int nloc = direct_partition(P, B, cols, area, r2, w2, list, cnt);
    const DirFx F = direct_frame(r_s, w_s, B);
    if (mode == 2) {
        for (int t = threadIdx.x; t < area; t += blockDim.x) {
            const int e = list[t];
            const int rr = cdiv(e), cc = e - rr * cols;
            const float v = direct_entry_f32x(P, F, w_s[B.k0 + rr], r_s[B.j0 + cc], t >= nloc);
            const int slot = rr * S + (t & (S - 1));
            atomicAdd(&rowf[slot], v * c2[B.j0 + cc].x);
            if (two) atomicAdd(&rowfb[slot], v * c2b[B.j0 + cc].x);
        }
        __syncthreads();
        // a row's S <= 32 slots summed by one warp, compensated FP32 sums
        // through the shuffles (no FP64 adds: FP64 runs at 1/64 of the rate)
        const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        for (int i = threadIdx.x >> 5; i < rows; i += nw) {
            const acc2 a = warp_sum_acc(acc2{lane < S ? rowf[i * S + lane] : 0.f, 0.f});
            if (lane == 0) atomicAdd(&g_s[B.k0 + i], (double)P.sgn * acc_value(a));
            if (two) {
                const acc2 ab = warp_sum_acc(acc2{lane < S ? rowfb[i * S + lane] : 0.f, 0.f});
                if (lane == 0) atomicAdd(&g_sb[B.k0 + i], (double)P.sgn * acc_value(ab));
            }
        }
        return;
    }
    if (det) {
        for (int t = threadIdx.x; t < area; t += blockDim.x) {
            const int e = list[t];
            const int rr = cdiv(e), cc = e - rr * cols;
            const double v = direct_entry_fx(P, F, w_s[B.k0 + rr], r_s[B.j0 + cc], t >= nloc, mode == 1);
            fx_add(reinterpret_cast<Fx128*>(g_s) + B.k0 + rr, (double)P.sgn * (v * c_s[B.j0 + cc]), P.fxs);
            if (two) fx_add(reinterpret_cast<Fx128*>(g_sb) + B.k0 + rr, (double)P.sgn * (v * c_sb[B.j0 + cc]), P.fxs);
        }
        return;
    }
    // A warp's 32 list positions hold runs of entries of one row (the list keeps
    // each warp's chunk of the partition in row order): the products are summed
    // over each run by a segmented scan through the shuffles, and one lane per
    // run adds the run's sum to the row, instead of one shared-memory FP64
    // atomic (a compare-and-swap loop, serialised within a run) per entry.
    const int lane = threadIdx.x & 31;
    const int area_pad = (area + 31) & ~31;
    // Entries and products in double-float (the FP32 pipes), the run sums too;
    // one conversion to FP64 per run.
    for (int t = threadIdx.x; t < area_pad; t += blockDim.x) {
        int rr = -1;
        df p{0.f, 0.f}, pb{0.f, 0.f};
        if (t < area) {
            const int e = list[t];
            rr = cdiv(e);
            const int cc = e - rr * cols;
            const df v = direct_entry_df(P, F, w_s[B.k0 + rr], r_s[B.j0 + cc], t >= nloc, mode == 1);
            const float2 cv = c2[B.j0 + cc];
            p = df_mul(v, df{cv.x, cv.y});
            if (two) {
                const float2 cvb = c2b[B.j0 + cc];
                pb = df_mul(v, df{cvb.x, cvb.y});
            }
        }
        const int rprev = __shfl_up_sync(0xffffffffu, rr, 1);
        const int rnext = __shfl_down_sync(0xffffffffu, rr, 1);
        const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || rprev != rr);
        const int seg0 = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));   // first lane of this run
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const df q{__shfl_up_sync(0xffffffffu, p.h, off), __shfl_up_sync(0xffffffffu, p.l, off)};
            df qb{0.f, 0.f};
            if (two) qb = df{__shfl_up_sync(0xffffffffu, pb.h, off), __shfl_up_sync(0xffffffffu, pb.l, off)};
            if (lane - off >= seg0) {
                p = df_add(p, q);
                if (two) pb = df_add(pb, qb);
            }
        }
        if (rr >= 0 && (lane == 31 || rnext != rr)) {
            atomicAdd(&rowacc[rr], df_to(p));
            if (two) atomicAdd(&rowaccb[rr], df_to(pb));
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < rows; i += blockDim.x) {
        atomicAdd(&g_s[B.k0 + i], (double)P.sgn * rowacc[i]);
        if (two) atomicAdd(&g_sb[B.k0 + i], (double)P.sgn * rowaccb[i]);
    }
}

// ------------------------------------------------------------------ adjoint
// Transposed local block A_blk^T = T C^T: adjoint moments
//   nu_l = sum_{k in block} g_k C_l(omega_k R)          (rows, Miller per row)
// then c_j += sum_l T_{2l(+1)}(r_j / R) nu_l              (columns).
//
// One CTA per tile of rows, in passes of blockDim rows.  Phase 1: each thread
// runs the Miller recurrence of one row into its column of jb (as in
// k_local_eval) and leaves g_k / S^2 and its power-of-two scale in shared
// memory.  Phase 2: warp w takes l = w, w + nwarps, ... and sums
// C_l(row) g_row / S_row^2 over the pass's rows straight from jb (compensated
// FP32 sums, one FP64 atomic per moment and pass).  No per-thread moment
// accumulators: the CTA holds as little shared memory as k_local_eval.  TWO:
// a second real component's g (g_sb) summed into momb with the same C_l.
constexpr int kAdjRowsPerLane = kMomThreads / 32;

template <bool TWO>
__global__ void __launch_bounds__(kMomThreads)
k_local_adj_moments(const ProbParams* __restrict__ probs, const LocalBlock* __restrict__ blks,
                    const Tile* __restrict__ tiles, const float2* __restrict__ w2,
                    const double* __restrict__ g_s, double* __restrict__ mom,
                    const double* __restrict__ g_sb, double* __restrict__ momb)
{
    extern __shared__ float2 sm2[];
    const Tile t = tiles[blockIdx.x];
    const LocalBlock B = blks[t.blk];
    const ProbParams& P = probs[B.prob];
    const int nt = blockDim.x, tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const int nu = P.nu, L = P.L;
    const int hp = (nu & 1) ? (nu + 1) / 2 : nu / 2;   // index paired with +l
    const int hm = (nu & 1) ? (nu - 1) / 2 : nu / 2;   // index paired with -l
    const int ntop = hp + L;
    float2* jb = sm2;                                  // [ntop + 1][nt]
    float2* gsm = sm2 + (size_t)(P.ntop + 1) * nt;     // [nt] g_k / S^2 per row
    float* p2m = (float*)(gsm + nt);                   // [nt] scale per row
    float2* gsmb = (float2*)(p2m + nt);                // [nt] second g_k / S^2 (TWO)
    for (int base = 0; base < t.count; base += nt) {
        const int cnt = t.count - base < nt ? t.count - base : nt;
        if (tid < cnt) {
            const int64_t k = t.start + base + tid;
            const double gk = (double)P.sgn * g_s[k];
            const double gkb = TWO ? (double)P.sgn * g_sb[k] : 0.0;
            const float2 wk = w2[k];
            const df ydf = df_mul(df{wk.x, wk.y}, df{0.5f * B.R_h, 0.5f * B.R_l});   // y = omega R / 2
            if (!(ydf.h > 0.f)) {
                // y below the FP32 range: J_n(y) = delta_n0 to far below rounding
                for (int q = 0; q <= ntop; ++q) jb[q * nt + tid] = make_float2(q == 0 ? 1.f : 0.f, 0.f);
                const df g = df_from(gk);
                gsm[tid] = make_float2(g.h, g.l);
                if (TWO) {
                    const df gb = df_from(gkb);
                    gsmb[tid] = make_float2(gb.h, gb.l);
                }
                p2m[tid] = 1.f;
            } else {
                const int ns = miller_start(ntop, (double)ydf.h);
                df S = (ydf.h >= 1.f) ? miller_store_df(ydf, ntop, ns, jb, nt, tid)
                                      : series_store_df(ydf, ntop, jb, nt, tid);
                // a power of two near 1/S keeps products of two values in FP32 range
                const float p2 = exp2f(-(float)ilogbf(S.h));
                S = df_scale(S, p2);
                const df iS = df_recip(S);
                const df gs = df_mul(df_mul(df_from(gk), iS), iS);   // g_k / S^2
                gsm[tid] = make_float2(gs.h, gs.l);
                if (TWO) {
                    const df gsb = df_mul(df_mul(df_from(gkb), iS), iS);
                    gsmb[tid] = make_float2(gsb.h, gsb.l);
                }
                p2m[tid] = p2;
            }
        }
        __syncthreads();
        float pr[kAdjRowsPerLane];
        df gr[kAdjRowsPerLane], grb[TWO ? kAdjRowsPerLane : 1];
#pragma unroll
        for (int i = 0; i < kAdjRowsPerLane; ++i) {
            const int kk = lane + 32 * i;
            pr[i] = kk < cnt ? p2m[kk] : 0.f;
            const float2 g = kk < cnt ? gsm[kk] : make_float2(0.f, 0.f);
            gr[i] = df{g.x, g.y};
            if (TWO) {
                const float2 gb = kk < cnt ? gsmb[kk] : make_float2(0.f, 0.f);
                grb[TWO ? i : 0] = df{gb.x, gb.y};
            }
        }
        for (int l = warp; l <= L; l += nw) {
            const int b = hm - l, bi = b >= 0 ? b : -b;
            float sgn = (b < 0 && (bi & 1)) ? -1.f : 1.f;
            if (l > 0 || (nu & 1)) sgn *= 2.f;
            acc2 a{0.f, 0.f}, ab{0.f, 0.f};
#pragma unroll
            for (int i = 0; i < kAdjRowsPerLane; ++i) {
                const int kk = lane + 32 * i;
                if (kk < cnt) {
                    const float2 va = jb[(hp + l) * nt + kk];
                    const float2 vb = jb[bi * nt + kk];
                    const float p = pr[i], ps = p * sgn;
                    const df cl = df_mul(df{va.x * p, va.y * p}, df{vb.x * ps, vb.y * ps});
                    acc_fma(a, cl, gr[i]);
                    if (TWO) acc_fma(ab, cl, grb[TWO ? i : 0]);
                }
            }
            a = warp_sum_acc(a);
            if (lane == 0) Accum{mom, P.fxs}.add(B.mom_off + l, acc_value(a));
            if (TWO) {
                ab = warp_sum_acc(ab);
                if (lane == 0) Accum{momb, P.fxs}.add(B.mom_off + l, acc_value(ab));
            }
        }
        __syncthreads();   // jb and gsm are rewritten by the next pass
    }
}

__global__ void __launch_bounds__(kMomThreads)
k_local_adj_eval(const ProbParams* __restrict__ probs, const LocalBlock* __restrict__ blks,
                 const Tile* __restrict__ tiles, const float2* __restrict__ r2,
                 const double* __restrict__ mom, double* __restrict__ c_s)
{
    extern __shared__ float2 mu2[];
    const Tile t = tiles[blockIdx.x];
    const LocalBlock B = blks[t.blk];
    const int L = probs[B.prob].L;
    const int odd = probs[B.prob].nu & 1;
    const int nt = blockDim.x, tid = threadIdx.x;
    for (int l = tid; l <= L; l += nt) {
        const double v = mom[B.mom_off + l];
        const float h = (float)v;
        mu2[l] = make_float2(h, (float)(v - (double)h));
    }
    __syncthreads();
    const df invR{B.iR_h, B.iR_l};
    for (int64_t j = t.start + tid; j < t.start + t.count; j += nt) {
        // the same arithmetic as k_local_moments (the transpose of the same operator)
        const float2 rj = r2[j];
        const df y = df_mul(df{rj.x, rj.y}, invR);
        const df u = df_add(df_mul(df{2.f * y.h, 2.f * y.l}, y), df{-1.f, 0.f});
        const df u2{2.f * u.h, 2.f * u.l};
        df t0 = odd ? y : df{1.f, 0.f};
        df t1 = odd ? df_mul(y, df_add(u2, df{-1.f, 0.f})) : u;
        acc2 sum{0.f, 0.f};
        acc_fma(sum, t0, df{mu2[0].x, mu2[0].y});
        if (L >= 1) acc_fma(sum, t1, df{mu2[1].x, mu2[1].y});
        for (int l = 2; l <= L; ++l) {
            const df t2 = cheb_step(u2, t1, t0);
            acc_fma(sum, t2, df{mu2[l].x, mu2[l].y});
            t0 = t1;
            t1 = t2;
        }
        Accum{c_s, probs[B.prob].fxs}.add(j, acc_value(sum));
    }
}

// Transposed direct block: column sums (entries split by branch as in
// k_direct), one atomic add per column.
__global__ void k_direct_adj(const ProbParams* __restrict__ probs, const DirectBlock* __restrict__ blks,
                             const double* __restrict__ r_s, const double* __restrict__ w_s,
                             const float2* __restrict__ r2, const float2* __restrict__ w2,
                             const double* __restrict__ g_s, double* __restrict__ c_s, int lowp, int det)
{
    // [cols] FP64 column sums; none in the deterministic mode, where every
    // entry's product goes straight into the exact fixed-point sums of c
    extern __shared__ double colacc[];
    __shared__ int cnt[2];
    const DirectBlock B = blks[blockIdx.x];
    const ProbParams& P = probs[B.prob];
    const int rows = B.k1 - B.k0 + 1, cols = B.j1 - B.j0 + 1;
    const ColDiv rdiv(rows);
    const int area = rows * cols;
    const int accd = det ? 0 : cols;
    int* list = (int*)(colacc + accd);
    for (int i = threadIdx.x; i < accd; i += blockDim.x) colacc[i] = 0.0;
    // entries in column-major order, so that a warp's list positions hold runs
    // of one column (as the forward's hold runs of one row)
    const int nloc = direct_partition(P, B, cols, area, r2, w2, list, cnt, true);
    const DirFx F = direct_frame(r_s, w_s, B);
    if (det) {
        for (int t = threadIdx.x; t < area; t += blockDim.x) {
            const int e = list[t];
            const int cc = rdiv(e), rr = e - cc * rows;
            const double v = direct_entry_fx(P, F, w_s[B.k0 + rr], r_s[B.j0 + cc], t >= nloc, lowp != 0);
            fx_add(reinterpret_cast<Fx128*>(c_s) + B.j0 + cc, (double)P.sgn * (v * g_s[B.k0 + rr]), P.fxs);
        }
        return;
    }
    // run sums by a segmented scan through the shuffles, one shared-memory
    // atomic per run (see k_direct)
    const int lane = threadIdx.x & 31;
    const int area_pad = (area + 31) & ~31;
    for (int t = threadIdx.x; t < area_pad; t += blockDim.x) {
        int cc = -1;
        double p = 0.0;
        if (t < area) {
            const int e = list[t];
            cc = rdiv(e);
            const int rr = e - cc * rows;
            p = direct_entry_fx(P, F, w_s[B.k0 + rr], r_s[B.j0 + cc], t >= nloc, lowp != 0) * g_s[B.k0 + rr];
        }
        const int cprev = __shfl_up_sync(0xffffffffu, cc, 1);
        const int cnext = __shfl_down_sync(0xffffffffu, cc, 1);
        const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || cprev != cc);
        const int seg0 = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const double q = __shfl_up_sync(0xffffffffu, p, off);
            if (lane - off >= seg0) p += q;
        }
        if (cc >= 0 && (lane == 31 || cnext != cc)) atomicAdd(&colacc[cc], p);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < cols; i += blockDim.x)
        atomicAdd(&c_s[B.j0 + i], (double)P.sgn * colacc[i]);
}

// ------------------------------------------------------------ vector groups
// The G real components of one call (vectors, or the parts of complex c)
// share the local and direct blocks' Bessel work: the basis T_{2l(+1)}(r_j/R)
// of a point and the Miller sweep of a row are formed once for all G, and a
// direct entry is evaluated once.  The moments are then the dense product of
// Sec. 3.1's factorisation applied to G columns at once,
//     mu[v][l] = sum_j T_{2l(+1)}(r_j / R) c_v[j]    ((L+1) x n_b by n_b x G per block),
// and a row's evaluation is sum_l C_l(omega_k R) mu[v][l] for every v.
// Component v's data sit at v times a stride (c_stride, mom_stride, g_stride)
// from the first's.

// One CTA per moment tile, in passes of blockDim points.  Each thread forms
// one point's basis into Tb[l][p] and stages its G coefficients in Cs[v][p]
// (double-float).  The (L+1) G outputs o = l G + v are then split over the
// threads: item it = o S + sub sums the pass's points p = sub (mod S) into a
// compensated accumulator that stays in registers across the passes (S = 1,
// 2, 4 or 8 lanes per output, so that small products still use the whole
// CTA); the S partial sums meet by shuffles, one atomic add per output and tile.
constexpr int kMomGroupOut = 8;   // items per thread

__global__ void __launch_bounds__(kMomThreads)
k_local_moments_group(const ProbParams* __restrict__ probs, const LocalBlock* __restrict__ blks,
                      const Tile* __restrict__ tiles, const float2* __restrict__ r2,
                      const float2* __restrict__ c2, int64_t c_stride, int G, double* __restrict__ mom,
                      int64_t mom_stride)
{
    extern __shared__ float2 smg[];
    const Tile t = tiles[blockIdx.x];
    const LocalBlock B = blks[t.blk];
    const ProbParams& P = probs[B.prob];
    const int L = P.L, odd = P.nu & 1;
    const int nt = blockDim.x, tid = threadIdx.x;
    const int O = (L + 1) * G;
    int S = 1;
    while (S < 8 && O * S < 2 * nt) S <<= 1;
    const int ps = nt + S;                 // row stride of Tb and Cs
    float2* Tb = smg;                      // [L + 1][ps]
    float2* Cs = smg + (L + 1) * ps;       // [G][ps]
    const int items = O * S;
    const int nout = (items + nt - 1) / nt;   // <= kMomGroupOut (checked by the launcher)
    const int sub = tid & (S - 1);
    int toff[kMomGroupOut], coff[kMomGroupOut];
    acc2 a[kMomGroupOut];
#pragma unroll
    for (int i = 0; i < kMomGroupOut; ++i) {
        const int it = tid + i * nt;
        const int o = it < items ? it / S : 0;
        const int l = o / G;
        toff[i] = l * ps;
        coff[i] = (o - l * G) * ps;
        a[i] = acc2{0.f, 0.f};
    }
    const df invR{B.iR_h, B.iR_l};
    const int64_t jend = t.start + t.count;
    for (int64_t j0 = t.start; j0 < jend; j0 += nt) {
        const int np = (int)(jend - j0 < nt ? jend - j0 : nt);
        __syncthreads();   // the previous pass's reads are done
        if (tid < np) {
            const int64_t j = j0 + tid;
            const float2 rj = r2[j];
            const df y = df_mul(df{rj.x, rj.y}, invR);                          // r_j / R in [0, 1]
            const df u = df_add(df_mul(df{2.f * y.h, 2.f * y.l}, y), df{-1.f, 0.f});   // T_2(y)
            const df u2{2.f * u.h, 2.f * u.l};
            // even: T_{2l}(y) = T_l(u); odd: T_{2l+1}(y) with T_1 = y, T_3 = y (2u - 1)
            df t0 = odd ? y : df{1.f, 0.f};
            df t1 = odd ? df_mul(y, df_add(u2, df{-1.f, 0.f})) : u;
            Tb[tid] = make_float2(t0.h, t0.l);
            if (L >= 1) Tb[ps + tid] = make_float2(t1.h, t1.l);
            for (int l = 2; l <= L; ++l) {
                const df t2 = cheb_step(u2, t1, t0);
                Tb[l * ps + tid] = make_float2(t2.h, t2.l);
                t0 = t1;
                t1 = t2;
            }
            for (int v = 0; v < G; ++v) Cs[v * ps + tid] = c2[v * c_stride + j];
        }
        __syncthreads();
        for (int p = sub; p < np; p += S) {
#pragma unroll
            for (int i = 0; i < kMomGroupOut; ++i) {
                if (i < nout) {
                    const float2 tv = Tb[toff[i] + p], cv = Cs[coff[i] + p];
                    acc_fma(a[i], df{cv.x, cv.y}, df{tv.x, tv.y});
                }
            }
        }
    }
    const Accum dst{mom, P.fxs};
#pragma unroll
    for (int i = 0; i < kMomGroupOut; ++i) {
        if (i >= nout) break;   // uniform over the CTA
        acc2 v = a[i];
        for (int off = S >> 1; off > 0; off >>= 1) {
            const float os = __shfl_xor_sync(0xffffffffu, v.s, off);
            const float oc = __shfl_xor_sync(0xffffffffu, v.c, off);
            float s2, q2;
            two_sum(v.s, os, s2, q2);
            v.s = s2;
            v.c += oc + q2;
        }
        const int it = tid + i * nt;
        if (it < items && sub == 0) {
            const int o = it / S, l = o / G;
            dst.add((o - l * G) * mom_stride + B.mom_off + l, acc_value(v));
        }
    }
}

// One thread per row of a local block, as k_local_eval: Miller's recurrence
// fills this thread's column of jb, then each C_l is formed once and applied
// to the moments of all G <= GM components (mu[l][v], double-float in shared
// memory, read by broadcast) with GM compensated sums in registers.
template <int GM>
__global__ void k_local_eval_group(const ProbParams* __restrict__ probs, const LocalBlock* __restrict__ blks,
                                   const Tile* __restrict__ tiles, const float2* __restrict__ w2,
                                   const double* __restrict__ mom, int64_t mom_stride, int G,
                                   double* __restrict__ g_s, int64_t g_stride)
{
    extern __shared__ float2 sme[];
    const Tile t = tiles[blockIdx.x];
    const LocalBlock B = blks[t.blk];
    const ProbParams& P = probs[B.prob];
    const int nt = blockDim.x, tid = threadIdx.x;
    const int nu = P.nu, L = P.L;
    float2* mu = sme;                          // [L + 1][GM]
    float2* jb = sme + (P.ntop + 1) * GM;      // [ntop + 1][nt]
    for (int i = tid; i < (L + 1) * GM; i += nt) {
        const int l = i / GM, v = i - l * GM;
        const double x = v < G ? mom[v * mom_stride + B.mom_off + l] : 0.0;
        const float h = (float)x;
        mu[i] = make_float2(h, (float)(x - (double)h));
    }
    __syncthreads();
    if (tid >= t.count) return;
    const int64_t k = t.start + tid;
    const float2 wk = w2[k];
    const df ydf = df_mul(df{wk.x, wk.y}, df{0.5f * B.R_h, 0.5f * B.R_l});   // y = omega R / 2
    const Accum dst{g_s, P.fxs};
    if (!(ydf.h > 0.f)) {
        // y below the FP32 range: only C_0 survives, and only for nu = 0
        for (int v = 0; v < G; ++v)
            dst.add(v * g_stride + k, nu == 0 ? (double)P.sgn * ((double)mu[v].x + (double)mu[v].y) : 0.0);
        return;
    }
    {
        const int hp = (nu & 1) ? (nu + 1) / 2 : nu / 2;   // index paired with +l
        const int hm = (nu & 1) ? (nu - 1) / 2 : nu / 2;   // index paired with -l
        const int ntop = hp + L;
        const int ns = miller_start(ntop, (double)ydf.h);
        df S;
        if (ydf.h >= 1.f) S = miller_store_df(ydf, ntop, ns, jb, nt, tid);
        else S = series_store_df(ydf, ntop, jb, nt, tid);
        const float p2 = exp2f(-(float)ilogbf(S.h));
        S = df_scale(S, p2);
        acc2 sum[GM];
#pragma unroll
        for (int v = 0; v < GM; ++v) sum[v] = acc2{0.f, 0.f};
        for (int l = 0; l <= L; ++l) {
            df cl;
            if (nu == 0) {
                // C_l = (2 - delta_l0) (-1)^l J_l^2
                const float2 v = jb[l * nt + tid];
                const float xh = v.x * p2, xl = v.y * p2;
                const float p = xh * xh;
                float e = fmaf(xh, xh, -p);
                e = fmaf(2.f * xh, xl, e);
                const df sq = fast_two_sum(p, e);
                const float sgn = l == 0 ? 1.f : ((l & 1) ? -2.f : 2.f);
                cl = df{sgn * sq.h, sgn * sq.l};
            } else {
                const int b = hm - l;
                const float2 va = jb[(hp + l) * nt + tid];
                const float2 vb = jb[(b >= 0 ? b : -b) * nt + tid];
                float sgn = (b < 0 && ((-b) & 1)) ? -1.f : 1.f;
                if (l > 0 || (nu & 1)) sgn *= 2.f;
                cl = df_mul(df{va.x * p2, va.y * p2}, df{vb.x * p2 * sgn, vb.y * p2 * sgn});
            }
            const float2* ml = mu + l * GM;
#pragma unroll
            for (int v = 0; v < GM; ++v)
                if (v < G) acc_fma(sum[v], cl, df{ml[v].x, ml[v].y});
        }
        const df iS = df_recip(S);
        const df iS2 = df_mul(iS, iS);
#pragma unroll
        for (int v = 0; v < GM; ++v)
            if (v < G)
                dst.add(v * g_stride + k, (double)P.sgn * df_to(df_mul(fast_two_sum(sum[v].s, sum[v].c), iS2)));
    }
}

// One CTA per direct block for a group of G components: the entries are
// evaluated once (after the branch split of k_direct) into shared memory,
// column-major as double-float values; then each (row, component) pair sums
// its row against the component's coefficients (compensated double-float),
// one atomic add per row and component.  Consecutive threads take
// consecutive rows of one component: conflict-free entry reads, one
// coefficient address per warp.
__global__ void k_direct_group(const ProbParams* __restrict__ probs, const DirectBlock* __restrict__ blks,
                               const double* __restrict__ r_s, const double* __restrict__ w_s,
                               const float2* __restrict__ r2, const float2* __restrict__ w2,
                               const float2* __restrict__ c2, int64_t c_stride, int G, double* __restrict__ g_s,
                               int64_t g_stride, int lowp)
{
    extern __shared__ float2 dsm[];
    __shared__ int cnt[2];
    const DirectBlock B = blks[blockIdx.x];
    const ProbParams& P = probs[B.prob];
    const int rows = B.k1 - B.k0 + 1, cols = B.j1 - B.j0 + 1;
    const ColDiv cdiv(cols);
    const int area = rows * cols;
    float2* E = dsm;                        // [cols][rows]
    int* list = (int*)(dsm + area);         // [area]
    const int nloc = direct_partition(P, B, cols, area, r2, w2, list, cnt);
    const DirFx F = direct_frame(r_s, w_s, B);
    for (int t = threadIdx.x; t < area; t += blockDim.x) {
        const int e = list[t];
        const int rr = cdiv(e), cc = e - rr * cols;
        const double v = direct_entry_fx(P, F, w_s[B.k0 + rr], r_s[B.j0 + cc], t >= nloc, lowp != 0);
        const float h = (float)v;
        E[cc * rows + rr] = make_float2(h, (float)(v - (double)h));
    }
    __syncthreads();
    const Accum dst{g_s, P.fxs};
    for (int o = threadIdx.x; o < rows * G; o += blockDim.x) {
        const int v = o / rows, rr = o - v * rows;
        const float2* cv = c2 + v * c_stride + B.j0;
        acc2 s{0.f, 0.f};
        for (int cc = 0; cc < cols; ++cc) {
            const float2 ev = E[cc * rows + rr], cf = cv[cc];
            acc_fma(s, df{ev.x, ev.y}, df{cf.x, cf.y});
        }
        dst.add(v * g_stride + B.k0 + rr, (double)P.sgn * acc_value(s));
    }
}

// Adjoint local blocks for a group of G <= GM components: each row's Miller
// sweep (phase 1) and each C_l(row) (phase 2) are formed once for all members;
// the adjoint moments are the dense product nu[v][l] = sum_rows C_l(row)
// g_v(row) / S(row)^2, G compensated sums per warp and l.
template <int GM>
__global__ void __launch_bounds__(kMomThreads)
k_local_adj_moments_group(const ProbParams* __restrict__ probs, const LocalBlock* __restrict__ blks,
                          const Tile* __restrict__ tiles, const float2* __restrict__ w2,
                          const double* __restrict__ g_s, int64_t g_stride, int G, double* __restrict__ mom,
                          int64_t mom_stride)
{
    extern __shared__ float2 sm2[];
    const Tile t = tiles[blockIdx.x];
    const LocalBlock B = blks[t.blk];
    const ProbParams& P = probs[B.prob];
    const int nt = blockDim.x, tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const int nu = P.nu, L = P.L;
    const int hp = (nu & 1) ? (nu + 1) / 2 : nu / 2;   // index paired with +l
    const int hm = (nu & 1) ? (nu - 1) / 2 : nu / 2;   // index paired with -l
    const int ntop = hp + L;
    float2* jb = sm2;                                  // [ntop + 1][nt]
    float2* gsm = sm2 + (size_t)(P.ntop + 1) * nt;     // [GM][nt] g_v,k / S^2 per row
    float* p2m = (float*)(gsm + GM * nt);              // [nt] scale per row
    for (int base = 0; base < t.count; base += nt) {
        const int cnt = t.count - base < nt ? t.count - base : nt;
        if (tid < cnt) {
            const int64_t k = t.start + base + tid;
            const float2 wk = w2[k];
            const df ydf = df_mul(df{wk.x, wk.y}, df{0.5f * B.R_h, 0.5f * B.R_l});   // y = omega R / 2
            df iS2{1.f, 0.f};
            float p2 = 1.f;
            if (!(ydf.h > 0.f)) {
                // y below the FP32 range: J_n(y) = delta_n0 to far below rounding
                for (int q = 0; q <= ntop; ++q) jb[q * nt + tid] = make_float2(q == 0 ? 1.f : 0.f, 0.f);
            } else {
                const int ns = miller_start(ntop, (double)ydf.h);
                df S = (ydf.h >= 1.f) ? miller_store_df(ydf, ntop, ns, jb, nt, tid)
                                      : series_store_df(ydf, ntop, jb, nt, tid);
                p2 = exp2f(-(float)ilogbf(S.h));
                S = df_scale(S, p2);
                const df iS = df_recip(S);
                iS2 = df_mul(iS, iS);
            }
            p2m[tid] = p2;
            for (int v = 0; v < GM; ++v) {
                const df gs = v < G ? df_mul(df_from((double)P.sgn * g_s[v * g_stride + k]), iS2) : df{0.f, 0.f};
                gsm[v * nt + tid] = make_float2(gs.h, gs.l);
            }
        }
        __syncthreads();
        for (int l = warp; l <= L; l += nw) {
            const int b = hm - l, bi = b >= 0 ? b : -b;
            float sgn = (b < 0 && (bi & 1)) ? -1.f : 1.f;
            if (l > 0 || (nu & 1)) sgn *= 2.f;
            acc2 a[GM];
#pragma unroll
            for (int v = 0; v < GM; ++v) a[v] = acc2{0.f, 0.f};
            for (int kk = lane; kk < cnt; kk += 32) {
                const float2 va = jb[(hp + l) * nt + kk];
                const float2 vb = jb[bi * nt + kk];
                const float p = p2m[kk], ps = p * sgn;
                const df cl = df_mul(df{va.x * p, va.y * p}, df{vb.x * ps, vb.y * ps});
#pragma unroll
                for (int v = 0; v < GM; ++v) {
                    if (v < G) {
                        const float2 g = gsm[v * nt + kk];
                        acc_fma(a[v], cl, df{g.x, g.y});
                    }
                }
            }
            const Accum dst{mom, P.fxs};
#pragma unroll
            for (int v = 0; v < GM; ++v) {
                if (v < G) {
                    const acc2 sv = warp_sum_acc(a[v]);
                    if (lane == 0) dst.add(v * mom_stride + B.mom_off + l, acc_value(sv));
                }
            }
        }
        __syncthreads();   // jb and gsm are rewritten by the next pass
    }
}

// Adjoint local evaluation for a group: each point's basis T_{2l(+1)}(r_j/R)
// once, applied to the G members' adjoint moments (mu[l][v] in shared
// memory), G compensated sums per point.
template <int GM>
__global__ void __launch_bounds__(kMomThreads)
k_local_adj_eval_group(const ProbParams* __restrict__ probs, const LocalBlock* __restrict__ blks,
                       const Tile* __restrict__ tiles, const float2* __restrict__ r2,
                       const double* __restrict__ mom, int64_t mom_stride, int G, double* __restrict__ c_s,
                       int64_t c_stride)
{
    extern __shared__ float2 mu2[];   // [L + 1][GM]
    const Tile t = tiles[blockIdx.x];
    const LocalBlock B = blks[t.blk];
    const int L = probs[B.prob].L;
    const int odd = probs[B.prob].nu & 1;
    const int nt = blockDim.x, tid = threadIdx.x;
    for (int i = tid; i < (L + 1) * GM; i += nt) {
        const int l = i / GM, v = i - l * GM;
        const double x = v < G ? mom[v * mom_stride + B.mom_off + l] : 0.0;
        const float h = (float)x;
        mu2[i] = make_float2(h, (float)(x - (double)h));
    }
    __syncthreads();
    const df invR{B.iR_h, B.iR_l};
    const Accum dst{c_s, probs[B.prob].fxs};
    for (int64_t j = t.start + tid; j < t.start + t.count; j += nt) {
        const float2 rj = r2[j];
        const df y = df_mul(df{rj.x, rj.y}, invR);
        const df u = df_add(df_mul(df{2.f * y.h, 2.f * y.l}, y), df{-1.f, 0.f});
        const df u2{2.f * u.h, 2.f * u.l};
        df t0 = odd ? y : df{1.f, 0.f};
        df t1 = odd ? df_mul(y, df_add(u2, df{-1.f, 0.f})) : u;
        acc2 sum[GM];
#pragma unroll
        for (int v = 0; v < GM; ++v) sum[v] = acc2{0.f, 0.f};
        for (int l = 0; l <= L; ++l) {
            df tl;
            if (l == 0) tl = t0;
            else if (l == 1) tl = t1;
            else {
                tl = cheb_step(u2, t1, t0);
                t0 = t1;
                t1 = tl;
            }
            const float2* ml = mu2 + l * GM;
#pragma unroll
            for (int v = 0; v < GM; ++v)
                if (v < G) acc_fma(sum[v], tl, df{ml[v].x, ml[v].y});
        }
#pragma unroll
        for (int v = 0; v < GM; ++v)
            if (v < G) dst.add(v * c_stride + j, acc_value(sum[v]));
    }
}

}  // namespace

int local_adj_threads(int ntop_max)
{
    // (ntop + 1) double-float values plus 12 bytes of row data per thread
    int t = (int)(200 * 1024 / (8 * (ntop_max + 1) + 12));
    t = (t / 32) * 32;
    if (t > kMomThreads) t = kMomThreads;
    if (t < 32) t = 32;
    return t;
}

cudaError_t launch_local_adj_moments(const ProbParams* probs, const LocalBlock* blks, const Tile* tiles,
                                     int ntiles, int ntop_max, int threads, const float2* w2,
                                     const double* g_s, double* mom, const double* g_sb, double* momb,
                                     cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    if (threads < 32 || threads > kMomThreads || (threads & 31)) return cudaErrorInvalidValue;
    if ((g_sb == nullptr) != (momb == nullptr)) return cudaErrorInvalidValue;
    const bool two = g_sb != nullptr;
    size_t smem = sizeof(float2) * (size_t)(ntop_max + 1) * threads + (sizeof(float2) + sizeof(float)) * threads +
                  (two ? sizeof(float2) * threads : 0);
    auto kern = two ? k_local_adj_moments<true> : k_local_adj_moments<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<ntiles, threads, smem, s>>>(probs, blks, tiles, w2, g_s, mom, g_sb, momb);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_local_adj_eval(const ProbParams* probs, const LocalBlock* blks, const Tile* tiles,
                                  int ntiles, int lmax, const float2* r2, const double* mom, double* c_s,
                                  cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    size_t smem = sizeof(float2) * (size_t)(lmax + 1);
    k_local_adj_eval<<<ntiles, kMomThreads, smem, s>>>(probs, blks, tiles, r2, mom, c_s);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_direct_adj(const ProbParams* probs, const DirectBlock* blks, int nblk, int max_cols,
                              int max_area, int lowp, const double* r_s, const double* w_s, const float2* r2,
                              const float2* w2, const double* g_s, double* c_s, int det, cudaStream_t s)
{
    if (nblk <= 0) return cudaSuccess;
    size_t smem = sizeof(double) * (det ? 1 : (size_t)(max_cols > 0 ? max_cols : 1)) +
                  sizeof(int) * (size_t)max_area;
    cudaError_t e = cudaFuncSetAttribute(k_direct_adj, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_direct_adj<<<nblk, 256, smem, s>>>(probs, blks, r_s, w_s, r2, w2, g_s, c_s, lowp, det);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_local_moments(const ProbParams* probs, const LocalBlock* blks, const Tile* tiles,
                                 int ntiles, int lmax, const float2* r2, const float2* c2,
                                 double* mom, cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    const int threads = local_moment_threads(lmax);
    size_t smem = sizeof(acc2) * (size_t)(lmax + 1) * threads;
    cudaError_t e = cudaFuncSetAttribute(k_local_moments, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_local_moments<<<ntiles, threads, smem, s>>>(probs, blks, tiles, r2, c2, mom);
    count_launches(1);
    return cudaGetLastError();
}

// The pair kernel when its 2 (lmax + 1) accumulators per thread fit the
// one-component kernel's threads in ~200 KB of shared memory; else
// cudaErrorInvalidValue (the caller runs two one-component launches).
cudaError_t launch_local_moments2(const ProbParams* probs, const LocalBlock* blks, const Tile* tiles,
                                  int ntiles, int lmax, const float2* r2, const float2* c2, const float2* c2b,
                                  double* mom, double* momb, cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    const int threads = local_moment_threads(lmax);
    const size_t smem = 2 * sizeof(acc2) * (size_t)(lmax + 1) * threads;
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_local_moments2, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_local_moments2<<<ntiles, threads, smem, s>>>(probs, blks, tiles, r2, c2, c2b, mom, momb);
    count_launches(1);
    return cudaGetLastError();
}

bool local_moments2_fits(int lmax)
{
    return 2 * sizeof(acc2) * (size_t)(lmax + 1) * local_moment_threads(lmax) <= 200 * 1024;
}

int local_moment_threads(int lmax)
{
    // (lmax + 1) 8-byte accumulators per thread must fit in ~200 KB of shared memory
    int t = (int)(200 * 1024 / (8 * (lmax + 1)));
    t = (t / 32) * 32;
    if (t > kMomThreads) t = kMomThreads;
    if (t < 32) t = 32;
    return t;
}

int local_eval_threads(int ntop_max)
{
    // (ntop + 1) doubles per thread must fit in ~200 KB of shared memory
    int t = (int)(200 * 1024 / (8 * (ntop_max + 1)));
    t = (t / 32) * 32;
    if (t > 128) t = 128;
    if (t < 32) t = 32;
    return t;
}

cudaError_t launch_local_eval(const ProbParams* probs, const LocalBlock* blks, const Tile* tiles,
                                   int ntiles, int ntop_max, bool column, int threads, const float2* w2,
                                   const double* mom, double* g_s, const double* momb, double* g_sb,
                                   cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    const size_t nmu = momb ? 2 : 1;
    // rows of order 0 keep no Bessel column (their sums are formed during the sweep)
    const size_t col = column ? (size_t)(ntop_max + 1) * threads : 0;
    size_t smem = sizeof(float2) * (col + nmu * (size_t)(ntop_max + 1));
    cudaError_t e = cudaFuncSetAttribute(k_local_eval, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_local_eval<<<ntiles, threads, smem, s>>>(probs, blks, tiles, w2, mom, g_s, momb, g_sb);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_local_persistent(const ProbParams* probs, const LocalBlock* blks, const Tile* tmom, int n_tmom,
                                    const Tile* teval, int n_teval, const int32_t* mom_pre, int lmax, int ntop_max,
                                    int threads, const float2* r2, const float2* c2, const float2* c2b,
                                    const float2* w2, double* mom, double* momb, double* g_s, double* g_sb, int* q,
                                    int nloc, int* status, int wait_limit, int stall, cudaStream_t s)
{
    if (n_tmom + n_teval <= 0) return cudaSuccess;
    if (threads < 32 || threads > kMomThreads || (threads & 31)) return cudaErrorInvalidValue;
    const size_t nmu = momb ? 2 : 1;
    const size_t sm_mom = sizeof(acc2) * (size_t)(lmax + 1) * threads;
    const size_t sm_eval = sizeof(float2) * ((size_t)(ntop_max + 1) * threads + nmu * (size_t)(ntop_max + 1));
    const size_t smem = sm_mom > sm_eval ? sm_mom : sm_eval;
    cudaError_t e = cudaFuncSetAttribute(k_local_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_local_persistent, threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const int items = (momb ? 2 : 1) * n_tmom + n_teval;
    int grid = sms * per_sm;
    if (grid > items) grid = items;
    e = cudaMemsetAsync(q, 0, sizeof(int) * (size_t)(nloc + 2), s);
    if (e != cudaSuccess) return e;
    k_local_persistent<<<grid, threads, smem, s>>>(probs, blks, tmom, n_tmom, teval, n_teval, mom_pre, r2, c2, c2b,
                                                   w2, mom, momb, g_s, g_sb, q, status, wait_limit, stall);
    count_launches(1);
    return cudaGetLastError();
}

// The direct kernel's mode for tolerance eps and the tallest and widest direct
// blocks.  In mode 2 a slot's chain of FP32 additions holds at most
// 3 cols / 32 + 4 terms when S = 32 (a row's entries fill at most cols / 32 + 2
// warp chunks of the lists, each adding at most one entry to a slot per list),
// and at most cols <= 127 terms when a block has more than 128 rows (S < 32):
// the rounding of one output's direct sums is below that count times
// 2^-24 sum |J c| (a row's direct blocks have disjoint columns), and mode 2 is
// used when that is at most 2 eps ||c||_1, a fifth of the tolerance.
int direct_sum_mode(double eps, int max_rows, int max_cols)
{
    if (eps < 1e-6) return 0;
    const int c = max_cols > 0 ? max_cols : 1;
    double chain = 3.0 * c / kDirSlots + 4.0;
    if (max_rows > kDirSlotFloats / kDirSlots) chain = std::max(chain, (double)std::min(c, 127));
    return chain * 5.9604644775390625e-08 <= 2.0 * eps ? 2 : 1;
}

cudaError_t launch_local_eval_f32(const ProbParams* probs, const LocalBlock* blks, const Tile* tiles,
                                  int ntiles, int ntop_max, int threads, const float2* w2, const double* mom,
                                  double* g_s, const double* momb, double* g_sb, cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    const size_t nmu = momb ? 2 : 1;
    size_t smem = sizeof(float) * ((size_t)(ntop_max + 1) * threads + nmu * (size_t)(ntop_max + 1));
    cudaError_t e = cudaFuncSetAttribute(k_local_eval_f32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_local_eval_f32<<<ntiles, threads, smem, s>>>(probs, blks, tiles, w2, mom, g_s, momb, g_sb);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_direct(const ProbParams* probs, const DirectBlock* blks, int nblk, int max_rows,
                          int max_area, int mode, const double* r_s, const double* w_s, const float2* r2,
                          const float2* w2, const double* c_s, const float2* c2, double* g_s,
                          const double* c_sb, const float2* c2b, double* g_sb, int det, cudaStream_t s)
{
    if (nblk <= 0) return cudaSuccess;
    if (det && mode == 2) mode = 1;   // no FP32 slot sums in the deterministic mode
    const size_t acc = det ? 1 : (g_sb ? 2 : 1) *
                       (mode == 2 ? (size_t)kDirSlotFloats / 2 : (size_t)(max_rows > 0 ? max_rows : 1));
    size_t smem = sizeof(double) * acc + sizeof(int) * (size_t)max_area;
    cudaError_t e = cudaFuncSetAttribute(k_direct, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_direct<<<nblk, 256, smem, s>>>(probs, blks, r_s, w_s, r2, w2, c_s, c2, g_s, c_sb, c2b, g_sb, mode, det);
    count_launches(1);
    return cudaGetLastError();
}

int local_group_fits(int lmax, int ntop_max, int eval_threads, int G)
{
    constexpr size_t kSmemMax = 200 * 1024;
    const size_t mom_smem = sizeof(float2) * (size_t)(lmax + 1 + G) * (kMomThreads + 8);
    const size_t eval_smem = sizeof(float2) * (size_t)(ntop_max + 1) * (eval_threads + kGroupMax);
    return G >= 1 && G <= kGroupMax && (lmax + 1) * G <= kMomGroupOut * kMomThreads && mom_smem <= kSmemMax &&
           eval_smem <= kSmemMax;
}

cudaError_t launch_local_moments_group(const ProbParams* probs, const LocalBlock* blks, const Tile* tiles,
                                       int ntiles, int lmax, const float2* r2, const float2* c2,
                                       int64_t c_stride, int G, double* mom, int64_t mom_stride, cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    if (G < 1 || G > kGroupMax || (lmax + 1) * G > kMomGroupOut * kMomThreads) return cudaErrorInvalidValue;
    const size_t smem = sizeof(float2) * (size_t)(lmax + 1 + G) * (kMomThreads + 8);
    cudaError_t e = cudaFuncSetAttribute(k_local_moments_group, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_local_moments_group<<<ntiles, kMomThreads, smem, s>>>(probs, blks, tiles, r2, c2, c_stride, G, mom,
                                                            mom_stride);
    count_launches(1);
    return cudaGetLastError();
}

template <int GM>
static cudaError_t eval_group_as(const ProbParams* probs, const LocalBlock* blks, const Tile* tiles, int ntiles,
                                 int ntop_max, int threads, const float2* w2, const double* mom,
                                 int64_t mom_stride, int G, double* g_s, int64_t g_stride, cudaStream_t s)
{
    const size_t smem = sizeof(float2) * (size_t)(ntop_max + 1) * (threads + GM);
    cudaError_t e = cudaFuncSetAttribute(k_local_eval_group<GM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_local_eval_group<GM><<<ntiles, threads, smem, s>>>(probs, blks, tiles, w2, mom, mom_stride, G, g_s,
                                                          g_stride);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_local_eval_group(const ProbParams* probs, const LocalBlock* blks, const Tile* tiles,
                                    int ntiles, int ntop_max, int threads, const float2* w2, const double* mom,
                                    int64_t mom_stride, int G, double* g_s, int64_t g_stride, cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    if (G < 1 || G > kGroupMax) return cudaErrorInvalidValue;
    if (G <= 4)
        return eval_group_as<4>(probs, blks, tiles, ntiles, ntop_max, threads, w2, mom, mom_stride, G, g_s,
                                g_stride, s);
    if (G <= 8)
        return eval_group_as<8>(probs, blks, tiles, ntiles, ntop_max, threads, w2, mom, mom_stride, G, g_s,
                                g_stride, s);
    return eval_group_as<16>(probs, blks, tiles, ntiles, ntop_max, threads, w2, mom, mom_stride, G, g_s,
                             g_stride, s);
}

cudaError_t launch_direct_group(const ProbParams* probs, const DirectBlock* blks, int nblk, int max_area,
                                int lowp, const double* r_s, const double* w_s, const float2* r2, const float2* w2,
                                const float2* c2, int64_t c_stride, int G, double* g_s, int64_t g_stride,
                                cudaStream_t s)
{
    if (nblk <= 0) return cudaSuccess;
    if (G < 1 || G > kGroupMax) return cudaErrorInvalidValue;
    const size_t smem = (sizeof(float2) + sizeof(int)) * (size_t)(max_area > 0 ? max_area : 1);
    cudaError_t e = cudaFuncSetAttribute(k_direct_group, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_direct_group<<<nblk, 128, smem, s>>>(probs, blks, r_s, w_s, r2, w2, c2, c_stride, G, g_s, g_stride, lowp);
    count_launches(1);
    return cudaGetLastError();
}

template <int GM>
static cudaError_t adj_group_as(const ProbParams* probs, const LocalBlock* blks, const Tile* teval, int n_teval,
                                const Tile* tmom, int n_tmom, int lmax, int ntop_max, int threads, const float2* w2,
                                const float2* r2, const double* g_s, int64_t g_stride, int G, double* mom,
                                int64_t mom_stride, double* c_s, int64_t c_stride, bool moments, cudaStream_t s)
{
    if (moments) {
        if (n_teval <= 0) return cudaSuccess;
        const size_t smem = sizeof(float2) * (size_t)(ntop_max + 1 + GM) * threads + sizeof(float) * threads;
        cudaError_t e = cudaFuncSetAttribute(k_local_adj_moments_group<GM>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_local_adj_moments_group<GM><<<n_teval, threads, smem, s>>>(probs, blks, teval, w2, g_s, g_stride, G, mom,
                                                                     mom_stride);
    } else {
        if (n_tmom <= 0) return cudaSuccess;
        const size_t smem = sizeof(float2) * (size_t)(lmax + 1) * GM;
        cudaError_t e = cudaFuncSetAttribute(k_local_adj_eval_group<GM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        k_local_adj_eval_group<GM><<<n_tmom, kMomThreads, smem, s>>>(probs, blks, tmom, r2, mom, mom_stride, G, c_s,
                                                                     c_stride);
    }
    count_launches(1);
    return cudaGetLastError();
}

int local_adj_group_threads(int ntop_max)
{
    // (ntop + 1 + 16) double-float values plus a scale per thread within ~200 KB
    int t = (int)(200 * 1024 / (8 * (ntop_max + 1 + kGroupMax) + 4));
    t = (t / 32) * 32;
    if (t > kMomThreads) t = kMomThreads;
    if (t < 32) t = 32;
    return t;
}

cudaError_t launch_local_adj_group(const ProbParams* probs, const LocalBlock* blks, const Tile* teval, int n_teval,
                                   const Tile* tmom, int n_tmom, int lmax, int ntop_max, int threads,
                                   const float2* w2, const float2* r2, const double* g_s, int64_t g_stride, int G,
                                   double* mom, int64_t mom_stride, double* c_s, int64_t c_stride, bool moments,
                                   cudaStream_t s)
{
    if (G < 1 || G > kGroupMax) return cudaErrorInvalidValue;
    if (G <= 4)
        return adj_group_as<4>(probs, blks, teval, n_teval, tmom, n_tmom, lmax, ntop_max, threads, w2, r2, g_s,
                               g_stride, G, mom, mom_stride, c_s, c_stride, moments, s);
    if (G <= 8)
        return adj_group_as<8>(probs, blks, teval, n_teval, tmom, n_tmom, lmax, ntop_max, threads, w2, r2, g_s,
                               g_stride, G, mom, mom_stride, c_s, c_stride, moments, s);
    return adj_group_as<16>(probs, blks, teval, n_teval, tmom, n_tmom, lmax, ntop_max, threads, w2, r2, g_s,
                            g_stride, G, mom, mom_stride, c_s, c_stride, moments, s);
}

}  // namespace nuht
