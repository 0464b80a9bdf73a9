// Asymptotic blocks: Hankel's expansion applied with 2M type-3 NUFFTs
// (Sec. 3.2).  For a block with points r_j in [r_lo, r_hi] and frequencies
// omega_k in [w_lo, w_hi], rho = r_lo, and q = 0..2M-1:
//
//   F_q(omega_k) = sum_j c_j (r_j/rho)^(-q-1/2) e^{i omega_k r_j}
//   g_k += sqrt(2/pi) Re( e^{i phi} sum_q a_q(nu) i^q (omega_k rho)^(-q-1/2) F_q(omega_k) )
//
// which is the M-pair form of Sec. 3.2 (the pair (2l, 2l+1) with the Re / -Im
// split is i^q), rescaled by rho so that no weight exceeds one.
//
// Type-3 NUFFT (exponential-of-semicircle kernel psi(t) = exp(beta (sqrt(1-t^2) - 1)),
// width w, upsampling sigma = 2), with r_c, X the centre / half-width of the
// points and w_c, S those of the frequencies:
//   x_j = r_j - r_c, s_k = omega_k - w_c,
//   h = pi / (sigma S),  alpha = w h / 2,
//   b_l = sum_j [c_j W_q(r_j) e^{i w_c x_j}] psi((l h - x_j)/alpha),  |l| <= N1   (spread)
//   Q_t = sum_l b_l / psi^(alpha2 l) e^{2 pi i l t / nf2},  alpha2 = w pi / nf2   (FFT)
//   P(s) = sum_t psi((s h - 2 pi t / nf2)/alpha2) Q_t                             (interpolate)
//   F_q(omega_k) = e^{i omega_k r_c} (4 / w^2) P(s_k) / psi^(alpha s_k)
// where psi^(xi) = int psi(t) cos(xi t) dt.  The two 1/psi^ factors undo the
// smoothing of the two spreading steps (Poisson summation); 4 / w^2 collects
// the grid spacings h and 2 pi / nf2 against alpha and alpha2.
//
// Arithmetic: a point's or frequency's grid cell, kernel coordinate and phase
// come from 64-bit fixed-point products with per-block constants (integer
// instructions); kernel taps, weighted values, the per-bin moments and sums
// and the FFT run in double-float (df64.cuh, ~48 bits, on the FP32 pipes);
// the spreading grids accumulate in FP64 atomics.  The FFT output is stored
// split into (hi, lo) floats so that the interpolation reads it as
// double-float without FP64 work.  Mixed precision (the _f32 kernels and the
// LOWP FFT instances) keeps the fixed-point positions and phases and runs the
// taps, sums and butterflies in FP32.
#include <cstdint>

#include "device_math.cuh"
#include "df64.cuh"
#include "nuht_internal.h"

namespace nuht {

int device_sm_count();

namespace {

constexpr int kWinCells = 64;   // grid cells an interpolation tile stages in shared memory
constexpr int kInterpTileThreads = 256;   // most frequencies per interpolation tile (one thread each)
constexpr int kAdjInterpThreads = 128;    // points per pass of an adjoint interpolation tile

// ------------------------------------------------------------------ spread
// A point r_j of a block covers the w grid cells l0 + i, i < w, with
// l0 = ceil((r_j - r_c)/h - w/2), and tap i of the ES kernel is the
// polynomial piece psi_i(v), v = 2 (l0 - (r_j - r_c)/h + w/2) - 1 in [-1, 1].

// floor(X K / 2^s) for the signed 128-bit product, 1 <= s <= 127 (the
// result fits in 64 bits).
__device__ __forceinline__ long long mul128_shr(long long X, long long K, int s)
{
    const unsigned long long lo = (unsigned long long)X * (unsigned long long)K;
    const long long hi = __mul64hi(X, K);
    if (s >= 64) return hi >> (s - 64);
    return (long long)(((unsigned long long)hi << (64 - s)) | (lo >> s));
}

// v 2^40 (|v| <= 1) as double-float, exactly.
__device__ __forceinline__ df df_from_sv(long long sv)
{
    float s2, e2;
    two_sum((float)(int)(sv >> 20) * 9.5367431640625e-07f, (float)(int)(sv & 0xFFFFF) * 9.094947017729282e-13f,
            s2, e2);
    return df{s2, e2};
}

// The cell l0 and kernel coordinate v (double-float) of r_j in the block's
// fixed-point frame (integer instructions, exact to 2^-41 cells), and its
// offset X = R_j - R_c for the phase.
__device__ __forceinline__ int spread_cell_fx(const AsyBlock& B, int w, double rj, long long* Xo, df* v)
{
    const long long X = fx_from_double(rj, B.fr) - B.Rc_fx;
    *Xo = X;
    const long long A = mul128_shr(X, B.KH, B.sA) - ((long long)w << 40);   // (x/h - w/2) 2^41
    const long long l0 = (A + ((1LL << 41) - 1)) >> 41;                     // ceil
    *v = df_from_sv(((l0 << 41) - A) - (1LL << 40));                       // v 2^40, v in [-1, 1)
    return (int)l0;
}

// c_j (r_j/rho)^(-1/2) e^{i w_c x_j} as double-float (re, im), x_j = r_j - r_c,
// and the ratio (r_j/rho)^(-1) that steps the weight from q to q + 1; r_j and
// c_j come as double-float pairs, the phase w_c x_j / (2 pi) from the
// fixed-point offset.
__device__ __forceinline__ void spread_weight_fx(const AsyBlock& B, const float4* __restrict__ tw, long long X,
                                                 float2 r2, float2 c2, df* wr, df* wi, df* rat)
{
    df sn, cs;
    df_sincos_turns_tab(mul128_bits(X, B.KW, B.sW), tw, &sn, &cs);
    *rat = df_mul(df{B.rho_h, B.rho_l}, df_recip(df{r2.x, r2.y}));
    const df w0 = df_mul(df{c2.x, c2.y}, df_sqrt(*rat));
    *wr = df_mul(w0, cs);
    *wi = df_mul(w0, sn);
}

// A signed 64-bit integer as double-float (relative error 2^-48): three
// exact 21-bit parts.
__device__ __forceinline__ df df_from_i64(long long x)
{
    const int a = (int)(x >> 42);
    const int b = (int)((x >> 21) & 0x1FFFFF);
    const int c = (int)(x & 0x1FFFFF);
    float s, e;
    two_sum((float)a * 4398046511104.f, (float)b * 2097152.f, s, e);   // 2^42, 2^21
    return fast_two_sum(s, e + (float)c);
}

// FFT-grid cell t0 = ceil(s hd - w/2) of a frequency omega_k and its kernel
// coordinate as sv = v 2^40 (v in [-1, 1)), in the block's fixed-point
// frequency frame (integer instructions, exact to 2^-40 cells); Om and
// S = Om - Wc_fx for the phase and the deconvolution argument.
__device__ __forceinline__ int interp_cell_sv(const AsyBlock& B, int w, double wk, long long* Om, long long* Sw,
                                              long long* svo)
{
    const long long O = fx_from_double(wk, B.fw);
    const long long S = O - B.Wc_fx;
    *Om = O;
    *Sw = S;
    const long long A = mul128_shr(S, B.KD, B.sD) - ((long long)w << 39);   // (s hd - w/2) 2^40
    const long long t0 = (A + ((1LL << 40) - 1)) >> 40;                     // ceil
    *svo = 2 * ((t0 << 40) - A) - (1LL << 40);
    return (int)t0;
}

// psi^(xi) for xi >= 0 given as double-float, double-float throughout: with
// t = xi times the table's pieces per unit, piece floor(t) (clamped to the
// table) and v = 2 (t - piece) - 1 in [-1, 1], the compensated Horner sum of
// that piece's polynomial.
__device__ __forceinline__ df psihat_of(const Tables& T, df xi)
{
    const df t = df_mul(xi, df{T.ph_scale2.x, T.ph_scale2.y});
    int piece = (int)t.h;
    if ((float)piece == t.h && t.l < 0.f && piece > 0) --piece;
    if (piece > T.ph_pieces - 1) piece = T.ph_pieces - 1;
    const df u = df_add(t, df{-(float)piece, 0.f});
    const df v = df_add(df{2.f * u.h, 2.f * u.l}, df{-1.f, 0.f});
    return horner_comp(T.ph2 + piece * (T.ph_deg + 1), T.ph_deg, v.h, v.l, T.ph_comp);
}

// psi^(xi) for xi = alpha s (s from the fixed-point offset S).
__device__ __forceinline__ df psihat_fx(const Tables& T, const AsyBlock& B, long long S)
{
    const float sc = ldexpf(1.f, -B.fw);
    const df s = df_from_i64(S < 0 ? -S : S);
    return psihat_of(T, df_mul(df{B.alpha_h, B.alpha_l}, df{s.h * sc, s.l * sc}));
}

constexpr int kSpreadSub = 8;       // point sub-ranges per moment, combined by shuffles
constexpr int kMomMinPerBin = 16;   // tiles with at least this many points per bin use moments
constexpr int kMaxTileBins = 32;

// Row strides of the moment path's shared arrays: = 2 mod 4 elements, so
// that the eight point rows a quarter-warp reads (16-byte loads of float2
// pairs, or 8-byte loads of float pairs) fall in distinct banks.
__host__ __device__ __forceinline__ int mom_stride(int n) { return ((n + 1) & ~1) + (((n + 1) & 2) ? 0 : 2); }

struct MomLayout {
    int ndf, nf;     // degree pairs accumulated in double-float / in FP32
    int sud, suf;    // row strides of the basis: double-float part (float2), FP32 part (float)
    int sx;          // row stride of the weighted values (float2)
    int dpad;        // rows of the moment matrix (2 ndf + 2 nf)
};

__host__ __device__ __forceinline__ MomLayout mom_layout(int nb, int dcs, int Q2)
{
    MomLayout L;
    L.ndf = (dcs + 1) >> 1;
    L.nf = (nb - dcs + 1) >> 1;
    L.sud = mom_stride(2 * L.ndf);
    L.suf = L.nf > 0 ? mom_stride(2 * L.nf) : 0;
    L.sx = mom_stride(Q2);
    L.dpad = 2 * (L.ndf + L.nf);
    return L;
}

// Degree of row e of the moment matrix (pairs of double-float degrees
// 0..2 ndf - 1, then pairs of FP32 degrees from dcs); -1 for padding.
__device__ __forceinline__ int mom_degree(int e, int ndf, int dcs, int nb)
{
    const int d = e < 2 * ndf ? e : dcs + (e - 2 * ndf);
    return (e < 2 * ndf ? d < dcs : d < nb) ? d : -1;
}

// Dense tile: all points of one bin (same l0) share the cells, so
//   grid[l0 + i][q'] += sum_d A[i][d] M[d][q'],  M[d][q'] = sum_{p in bin} T_d(v_p) x_q'(p),
// where psi_i(v) = sum_d A[i][d] T_d(v) is tap i in the Chebyshev basis and
// x_q'(p) runs over (re, im) of the 2M weighted values.  The moments are a
// small dense contraction over the bin's points (register-blocked, 2 degrees
// x 4 values per thread, the point range split over 8 lanes); degrees >=
// tab.dcs, whose coefficients are tiny, accumulate in plain FP32, the rest
// in double-float.
//
// Shared by the spreading of points (forward) and of frequencies (adjoint):
// target(j, &v, xq) gives target j's cell and kernel coordinate v and writes
// its 2M weighted values as double-float (re, im) pairs xq[2q], xq[2q + 1];
// cell(c) is the grid index of cell c, or -1 for a cell outside the grid.
// Members (forward spreading of V real components): target writes member 0's
// values; values(vm, xq) rewrites this thread's point's values for member vm,
// whose grid sits moff accumulator elements after member 0's.  The basis,
// the cells and the bins are formed once for all members.
template <class Target, class Values, class Cell, class Acc>
__device__ __forceinline__ void spread_moments(int Q, int qs, const Tile& t, const Tables& tab, Target&& target,
                                               Values&& values, int V, int64_t moff, Cell&& cell, Acc gb,
                                               float2* sm)
{
    const int nt = blockDim.x, tid = threadIdx.x, cnt = t.count;
    const int w = tab.w, nb = tab.nb, dcs = tab.dcs;
    const int Q2 = 2 * Q;
    const MomLayout L = mom_layout(nb, dcs, Q2);
    const int nq = Q2 >> 2;
    float2* Ud = sm;                                  // [nt][sud]  T_d(v_p), d < dcs
    float2* X = Ud + nt * L.sud;                      // [nt][sx]   x_q'(p)
    float2* Mb = X + nt * L.sx;                       // [dpad][Q2] moments of the current bin
    float2* Ach = Mb + L.dpad * Q2;                   // [w][dpad]  Chebyshev coefficients, row order of Mb
    float* Uf = (float*)(Ach + w * L.dpad);           // [nt][suf]  T_d(v_p), d >= dcs
    int* l0s = (int*)(Uf + nt * L.suf);               // [nt]
    __shared__ int bstart[kMaxTileBins + 3];
    for (int i = tid; i < w * L.dpad; i += nt) {
        const int r = i / L.dpad, e = i - r * L.dpad;
        const int d = mom_degree(e, L.ndf, dcs, nb);
        Ach[i] = d >= 0 ? tab.ch2[r * (tab.deg + 1) + d] : make_float2(0.f, 0.f);
    }
    if (tid < cnt) {
        df vd;
        l0s[tid] = target(t.start + tid, &vd, X + tid * L.sx);
        // Chebyshev basis by T_{d+1} = 2 v T_d - T_{d-1}
        float2* ud = Ud + tid * L.sud;
        float* uf = Uf + tid * L.suf;
        const float vh = vd.h, vl = vd.l;
        df tm{1.f, 0.f}, tc{vh, vl};
        ud[0] = make_float2(1.f, 0.f);
        ud[1] = make_float2(vh, vl);                 // dcs >= 2
        const df v2{2.f * vh, 2.f * vl};
        int d = 2;
        for (; d < dcs; ++d) {
            const df tn = cheb_step(v2, tc, tm);
            ud[d] = make_float2(tn.h, tn.l);
            tm = tc;
            tc = tn;
        }
        for (int e = dcs; e < L.sud; ++e) ud[e] = make_float2(0.f, 0.f);
        float fm = tm.h, fc = tc.h;
        for (; d < nb; ++d) {
            const float fn = fmaf(2.f * vh, fc, -fm);
            uf[d - dcs] = fn;
            fm = fc;
            fc = fn;
        }
        for (int e = nb - dcs; e < L.suf; ++e) uf[e] = 0.f;
    }
    __syncthreads();
    const int lfirst = l0s[0];
    const int nbins = l0s[cnt - 1] - lfirst + 1;
    // first point of each bin (the tile's points are sorted, so bins are runs)
    for (int b = tid; b <= nbins; b += nt) {
        const int key = lfirst + b;
        int lo = 0, hi = cnt;
        while (lo < hi) { const int mid = (lo + hi) >> 1; if (l0s[mid] < key) lo = mid + 1; else hi = mid; }
        bstart[b] = lo;
    }
    __syncthreads();
    const int npairs = L.ndf + L.nf;
    const int nitems = npairs * nq * kSpreadSub;
    const int nqA = min(nq, (qs + 1) >> 1);        // quads holding a term q < qs
    const int nA = L.ndf * nqA, nB = L.ndf * (nq - nqA);
    const int nitems_pad = (nitems + 31) & ~31;
    for (int vm = 0; vm < V; ++vm) {
    if (vm > 0) {
        if (tid < cnt) values(vm, X + tid * L.sx);
        __syncthreads();
    }
    const Acc gv = gb.at(vm * moff);
    for (int b = 0; b < nbins; ++b) {
        const int p0 = bstart[b], p1 = bstart[b + 1];
        if (p0 == p1) continue;
        for (int it = tid; it < nitems_pad; it += nt) {
            const bool live = it < nitems;
            const int sub = it & (kSpreadSub - 1);
            const int o = live ? it / kSpreadSub : 0;
            // outputs (degree pair dp, value quad qq) ordered by cost so that warps
            // are uniform: double-float degrees with a quad holding a term q < qs,
            // then double-float degrees with quads of small terms, then FP32 degrees
            int dp, qq;
            if (o < nA) {
                dp = o / nqA;
                qq = o - dp * nqA;
            } else if (o < nA + nB) {
                const int ob = o - nA;
                dp = ob / (nq - nqA);
                qq = nqA + (ob - dp * (nq - nqA));
            } else {
                const int ob = o - nA - nB;
                dp = L.ndf + ob / nq;
                qq = ob - (dp - L.ndf) * nq;
            }
            const bool lowd = dp >= L.ndf;       // FP32-tier degrees
            const bool lowq = o >= nA && !lowd;  // double-float degrees, small Hankel terms only
            acc2 A[2][4];
#pragma unroll
            for (int e = 0; e < 2; ++e)
#pragma unroll
                for (int f = 0; f < 4; ++f) A[e][f] = acc2{0.f, 0.f};
            if (live && !lowd && lowq) {
                const float2* up = Ud + 2 * dp;
#pragma unroll 2
                for (int p = p0 + sub; p < p1; p += kSpreadSub) {
                    const float4 uu = *(const float4*)(up + p * L.sud);
                    const float4 xa = *(const float4*)(X + p * L.sx + 4 * qq);
                    const float4 xb = *(const float4*)(X + p * L.sx + 4 * qq + 2);
                    const float xs[4] = {xa.x, xa.z, xb.x, xb.z};
#pragma unroll
                    for (int f = 0; f < 4; ++f) {
                        A[0][f].s = fmaf(uu.x, xs[f], A[0][f].s);
                        A[1][f].s = fmaf(uu.z, xs[f], A[1][f].s);
                    }
                }
            } else if (live && !lowd) {
                const float2* up = Ud + 2 * dp;
#pragma unroll 2
                for (int p = p0 + sub; p < p1; p += kSpreadSub) {
                    const float4 uu = *(const float4*)(up + p * L.sud);
                    const float4 xa = *(const float4*)(X + p * L.sx + 4 * qq);
                    const float4 xb = *(const float4*)(X + p * L.sx + 4 * qq + 2);
                    const df xs[4] = {{xa.x, xa.y}, {xa.z, xa.w}, {xb.x, xb.y}, {xb.z, xb.w}};
#pragma unroll
                    for (int f = 0; f < 4; ++f) {
                        acc_fma(A[0][f], df{uu.x, uu.y}, xs[f]);
                        acc_fma(A[1][f], df{uu.z, uu.w}, xs[f]);
                    }
                }
            } else if (live) {
                const float* up = Uf + 2 * (dp - L.ndf);
#pragma unroll 2
                for (int p = p0 + sub; p < p1; p += kSpreadSub) {
                    const float2 uu = *(const float2*)(up + p * L.suf);
                    const float4 xa = *(const float4*)(X + p * L.sx + 4 * qq);
                    const float4 xb = *(const float4*)(X + p * L.sx + 4 * qq + 2);
                    const float xs[4] = {xa.x, xa.z, xb.x, xb.z};
#pragma unroll
                    for (int f = 0; f < 4; ++f) {
                        A[0][f].s = fmaf(uu.x, xs[f], A[0][f].s);
                        A[1][f].s = fmaf(uu.y, xs[f], A[1][f].s);
                    }
                }
            }
            // combine the kSpreadSub partial sums (adjacent lanes)
#pragma unroll
            for (int e = 0; e < 2; ++e)
#pragma unroll
                for (int f = 0; f < 4; ++f) {
                    acc2 a = A[e][f];
#pragma unroll
                    for (int off = kSpreadSub >> 1; off > 0; off >>= 1) {
                        const float os = __shfl_xor_sync(0xffffffffu, a.s, off);
                        const float oc = __shfl_xor_sync(0xffffffffu, a.c, off);
                        float s2, q2;
                        two_sum(a.s, os, s2, q2);
                        a.s = s2;
                        a.c += oc + q2;
                    }
                    if (live && sub == 0) {
                        const df m = fast_two_sum(a.s, a.c);
                        Mb[(2 * dp + e) * Q2 + 4 * qq + f] = make_float2(m.h, m.l);
                    }
                }
        }
        __syncthreads();
        // grid[l0 + i][q'] += sum_d A[i][d] M[d][q']
        const int l0 = lfirst + b;
        for (int o = tid; o < w * Q2; o += nt) {
            const int i = o / Q2, qv = o - i * Q2;
            const int64_t idx = cell(l0 + i);
            if (idx < 0) continue;
            acc2 s{0.f, 0.f};
            const float2* ar = Ach + i * L.dpad;
            float sf = 0.f;
            int e = 0;
            if ((qv >> 1) < qs) {
                for (; e < 2 * L.ndf; ++e) {
                    const float2 a2 = ar[e], m2 = Mb[e * Q2 + qv];
                    acc_fma(s, df{a2.x, a2.y}, df{m2.x, m2.y});
                }
            }
            for (; e < L.dpad; ++e) sf = fmaf(ar[e].x, Mb[e * Q2 + qv].x, sf);
            const double val = acc_value(s) + (double)sf;
            if (val != 0.0) gv.add(2 * ((int64_t)idx * Q + (qv >> 1)) + (qv & 1), val);
        }
        __syncthreads();
    }
    }
}

// Shared memory (bytes) of the moment path for nt points and Q = 2M.
__host__ __device__ __forceinline__ size_t spread_moments_smem(int nt, int Q, int w, int nb, int dcs)
{
    const MomLayout L = mom_layout(nb, dcs, 2 * Q);
    return sizeof(float2) * ((size_t)nt * L.sud + (size_t)nt * L.sx + (size_t)L.dpad * 2 * Q +
                             (size_t)w * L.dpad) +
           sizeof(float) * (size_t)nt * L.suf + sizeof(int) * (size_t)nt;
}

// q-folded dense tile.  Within the bin of cell L, r_p = R_L - (h/2) v_p with
// R_L = r_c + h (L + (w - 1)/2), so the weights are (rho/r_p)^q = s^q (1 - eta v_p)^-q,
// s = rho / R_L, eta = h / (2 R_L): a smooth function of v_p.  Its Chebyshev
// form sum_k beta_qk T_k(v) (from the Taylor series sum_j C(q+j-1, j) (eta v)^j
// and v^j = sum_k MC(j, k) T_k(v)) and T_d T_k = (T_{d+k} + T_{|d-k|}) / 2 give
//   M[d][q] = sum_p T_d(v_p) (rho/r_p)^q y_p = sum_k beta_qk (N[d+k] + N[|d-k|]) / 2,
//   N[e] = sum_p T_e(v_p) y_p,   y_p = c_p (r_p/rho)^(-1/2) e^{i w_c x_p},
// so each point adds to 2 (nb + K - 1) moments N instead of nb x 2M moments M.
// K terms are kept where the Taylor tail is below tab.fold_tol; N is
// double-float for degrees below dcs plus those reached with a beta above
// tab.fold_df_tol, plain FP32 above.  M then feeds the same grid update as
// the plain moment path.  Tiles whose bins are too wide for their radius
// (eta too large for kFoldMax terms) take the plain moment path.
constexpr int kFoldMax = 8;          // Chebyshev terms of the weights' dependence on v within a bin
constexpr int kBetaStride = kFoldMax + 1;   // row stride of beta (float2): odd, so the q rows an
                                            // M item's half-warp reads fall in distinct banks
constexpr int kFoldDfMax = 4;        // extra double-float degrees of N the fold may need
constexpr int kFoldGroupBytes = 8192;

// Constants of the fold's weight expansion: 1/(j + 1) as double-float and
// MC(j, k) = 2^(1-j) C(j, (j-k)/2) (halved for k = 0; zero unless j >= k and
// j - k is even), the Chebyshev coefficients of v^j -- exact small floats.
struct FoldConsts {
    float2 inv[kFoldMax];
    float mc[kFoldMax][kFoldMax];
};
constexpr FoldConsts make_fold_consts()
{
    FoldConsts c{};
    for (int j = 0; j < kFoldMax; ++j) {
        const double v = 1.0 / (j + 1);
        const float h = (float)v;
        c.inv[j] = float2{h, (float)(v - (double)h)};
        for (int k = 0; k < kFoldMax; ++k) {
            double m = 0.0;
            if (k <= j && ((j - k) & 1) == 0) {
                const int i = (j - k) / 2;
                double binom = 1.0;
                for (int t = 0; t < i; ++t) binom = binom * (j - t) / (t + 1);
                m = binom * 2.0;
                for (int t = 0; t < j; ++t) m *= 0.5;
                if (k == 0) m *= 0.5;
            }
            c.mc[j][k] = (float)m;
        }
    }
    return c;
}
__constant__ FoldConsts kFoldC = make_fold_consts();

// a f for a double-float a and a float f
__device__ __forceinline__ df df_mul_f(df a, float f)
{
    const float p = a.h * f;
    return fast_two_sum(p, fmaf(a.l, f, fmaf(a.h, f, -p)));
}

struct FoldPlan {
    int K;      // terms k < K of the weights' Chebyshev form
    int E;      // moments N[e], e < E (even)
    int Edf;    // N[e] in double-float for e < Edf (even)
};

// The fold's sizes for a tile whose first bin is cell lfirst; false when it
// does not apply (plain moment path).  Bounds with q = Q - 1, the largest,
// in FP32 (a bound, evaluated by one thread while the tile waits: FP64 here
// would stall the CTA).
__device__ bool fold_plan(const AsyBlock& B, const Tables& tab, int Q, int lfirst, FoldPlan* fp)
{
    const float R = (float)B.rc + (float)B.h * ((float)lfirst + 0.5f * (float)(tab.w - 1));
    if (!(R > 0.f)) return false;
    const float eta = (float)B.h / (2.f * R);
    const int qm = Q - 1;
    float t[kFoldMax + 1], tail[kFoldMax + 1];
    t[0] = 1.f;
#pragma unroll
    for (int j = 0; j < kFoldMax; ++j) t[j + 1] = t[j] * eta * (float)(qm + j) * (1.f / (float)(j + 1));
    const float ratio = eta * (float)(qm + kFoldMax) * (1.f / (float)(kFoldMax + 1));
    if (!(ratio < 0.5f)) return false;
    tail[kFoldMax] = 2.f * t[kFoldMax];   // geometric tail, ratio < 1/2
#pragma unroll
    for (int k = kFoldMax - 1; k >= 0; --k) tail[k] = tail[k + 1] + t[k];
    // 1.01: room for the FP32 rounding of the bound itself
    int K = 1;
    while (K <= kFoldMax && 1.01f * tail[K] > tab.fold_tol) ++K;
    if (K > kFoldMax) return false;
    int kd = 0;
    while (kd + 1 < K && 1.01f * tail[kd + 1] > tab.fold_df_tol) ++kd;
    if (kd > kFoldDfMax) return false;
    fp->K = K;
    fp->E = (tab.nb + K - 1 + 1) & ~1;
    const int edf = (tab.dcs + kd + 1) & ~1;
    fp->Edf = edf < fp->E ? edf : fp->E;
    return true;
}

__host__ __device__ __forceinline__ int fold_group_bins(int dpad, int Q2)
{
    int g = kFoldGroupBytes / (int)(sizeof(float2) * dpad * Q2);
    if (g < 1) g = 1;
    return g < kMaxTileBins ? g : kMaxTileBins;
}

__host__ __device__ __forceinline__ int fold_emax(int nb) { return (nb + kFoldMax - 1 + 1) & ~1; }
__host__ __device__ __forceinline__ int fold_edf_max(int nb, int dcs)
{
    const int e = (dcs + kFoldDfMax + 1) & ~1, em = fold_emax(nb);
    return e < em ? e : em;
}

// Shared memory (bytes) of the folded path for nt points and Q = 2M (its largest layout).
__host__ __device__ __forceinline__ size_t spread_fold_smem(int nt, int Q, int w, int nb, int dcs)
{
    const MomLayout L = mom_layout(nb, dcs, 2 * Q);
    const int G = fold_group_bins(L.dpad, 2 * Q);
    const int em = fold_emax(nb), edm = fold_edf_max(nb, dcs);
    const int sud = mom_stride(edm), suf = mom_stride(em - 2);
    return sizeof(float4) * ((size_t)nt + (size_t)G * em) +
           sizeof(float2) * ((size_t)nt * sud + (size_t)G * L.dpad * (2 * Q + 1) + (size_t)G * Q * kBetaStride +
                             (size_t)w * L.dpad) +
           sizeof(float) * (size_t)nt * suf + sizeof(int) * (size_t)nt;
}

// Members (MULTI): V real components with coefficients c2 + vm c_stride,
// grids moff accumulator elements apart; the points' cells, bases and phase
// factors and the bins are formed once for all members.
template <bool MULTI, class Acc>
__device__ void spread_fold(const AsyBlock& B, int Q, int qs, const Tile& t, const Tables& tab, FoldPlan F,
                            const double* __restrict__ r_s, const float2* __restrict__ r2,
                            const float2* __restrict__ c2, int64_t c_stride, int V, int64_t moff, Acc gb,
                            float4* sm4)
{
    const int nt = blockDim.x, tid = threadIdx.x, cnt = t.count;
    const int w = tab.w, nb = tab.nb, dcs = tab.dcs;
    const int Q2 = 2 * Q, K = F.K, E = F.E, Edf = F.Edf;
    const MomLayout L = mom_layout(nb, dcs, Q2);
    const int G = fold_group_bins(L.dpad, Q2);
    const int sud = mom_stride(Edf), suf = mom_stride(E - Edf);
    float4* Y = sm4;                                  // [nt] y_p as (re.h, re.l, im.h, im.l)
    float4* N = Y + nt;                               // [G][E] N[e] of a group of bins
    float2* Ud = (float2*)(N + G * E);                // [nt][sud] T_e(v_p), e < Edf
    // M rows padded to Q2 + 1 (odd) float2: the items of a half-warp (4 degrees
    // x 4 q pairs) store to distinct banks
    const int Q2s = Q2 + 1;
    float2* Mb = Ud + nt * sud;                       // [G][dpad][Q2s] M of a group of bins
    float2* beta = Mb + G * L.dpad * Q2s;             // [G][Q][kBetaStride] beta_qk
    float2* Ach = beta + G * Q * kBetaStride;         // [w][dpad] Chebyshev coefficients of the taps
    float* Uf = (float*)(Ach + w * L.dpad);           // [nt][suf] T_e(v_p), Edf <= e < E
    int* l0s = (int*)(Uf + nt * suf);                 // [nt]
    __shared__ int bstart[kMaxTileBins + 3];
    for (int i = tid; i < w * L.dpad; i += nt) {
        const int r = i / L.dpad, e = i - r * L.dpad;
        const int d = mom_degree(e, L.ndf, dcs, nb);
        Ach[i] = d >= 0 ? tab.ch2[r * (tab.deg + 1) + d] : make_float2(0.f, 0.f);
    }
    // this thread's point: (r_j/rho)^(-1/2) e^{i w_c x_j} (the weight without c_j)
    df yr{0.f, 0.f}, yi{0.f, 0.f};
    const int64_t j = t.start + tid;
    if (tid < cnt) {
        long long X;
        df vd;
        l0s[tid] = spread_cell_fx(B, w, r_s[j], &X, &vd);
        float2* ud = Ud + tid * sud;
        float* uf = Uf + tid * suf;
        const float vh = vd.h, vl = vd.l;
        df tm{1.f, 0.f}, tc{vh, vl};
        ud[0] = make_float2(1.f, 0.f);
        ud[1] = make_float2(vh, vl);                 // Edf >= 2
        const df v2{2.f * vh, 2.f * vl};
        int d = 2;
        for (; d < Edf; ++d) {
            const df tn = cheb_step(v2, tc, tm);
            ud[d] = make_float2(tn.h, tn.l);
            tm = tc;
            tc = tn;
        }
        float fm = tm.h, fc = tc.h;
        for (; d < E; ++d) {
            const float fn = fmaf(2.f * vh, fc, -fm);
            uf[d - Edf] = fn;
            fm = fc;
            fc = fn;
        }
        df rat;
        spread_weight_fx(B, tab.tw2, X, r2[j], MULTI ? make_float2(1.f, 0.f) : c2[j], &yr, &yi, &rat);
        if (!MULTI) Y[tid] = make_float4(yr.h, yr.l, yi.h, yi.l);
    }
    __syncthreads();
    const int lfirst = l0s[0];
    const int nbins = l0s[cnt - 1] - lfirst + 1;
    for (int b = tid; b <= nbins; b += nt) {
        const int key = lfirst + b;
        int lo = 0, hi = cnt;
        while (lo < hi) { const int mid = (lo + hi) >> 1; if (l0s[mid] < key) lo = mid + 1; else hi = mid; }
        bstart[b] = lo;
    }
    __syncthreads();
    const int nf1 = 2 * B.N1 + 1;
    const int npd = Edf >> 1, npf = (E - Edf) >> 1;
    const df rho{B.rho_h, B.rho_l};
    for (int vm = 0; vm < (MULTI ? V : 1); ++vm) {
    if (MULTI) {
        if (tid < cnt) {
            const float2 cv = c2[vm * c_stride + j];
            const df wr = df_mul(df{cv.x, cv.y}, yr), wi = df_mul(df{cv.x, cv.y}, yi);
            Y[tid] = make_float4(wr.h, wr.l, wi.h, wi.l);
        }
        __syncthreads();
    }
    const Acc gv = gb.at(vm * moff);
    for (int g0 = 0; g0 < nbins; g0 += G) {
        const int gn = nbins - g0 < G ? nbins - g0 : G;
        // (a) N of the group's bins: items (bin, degree pair) split over
        // kSpreadSub lanes each, double-float items first
        const int nitems = gn * (npd + npf) * kSpreadSub;
        const int nitems_pad = (nitems + 31) & ~31;
        for (int it = tid; it < nitems_pad; it += nt) {
            const bool live = it < nitems;
            const int sub = it & (kSpreadSub - 1);
            const int o = live ? it / kSpreadSub : 0;
            int b, pr;
            bool dfi;
            if (o < gn * npd) {
                b = o / npd;
                pr = o - b * npd;
                dfi = true;
            } else {
                const int o2 = o - gn * npd;
                b = o2 / npf;
                pr = o2 - b * npf;
                dfi = false;
            }
            const int p0 = bstart[g0 + b], p1 = bstart[g0 + b + 1];
            acc2 a00{0.f, 0.f}, a01{0.f, 0.f}, a10{0.f, 0.f}, a11{0.f, 0.f};
            if (live && dfi) {
                const float2* up = Ud + 2 * pr;
#pragma unroll 2
                for (int p = p0 + sub; p < p1; p += kSpreadSub) {
                    const float4 uu = *(const float4*)(up + p * sud);
                    const float4 yv = Y[p];
                    const df u0{uu.x, uu.y}, u1{uu.z, uu.w}, yr{yv.x, yv.y}, yi{yv.z, yv.w};
                    acc_fma(a00, u0, yr);
                    acc_fma(a01, u0, yi);
                    acc_fma(a10, u1, yr);
                    acc_fma(a11, u1, yi);
                }
            } else if (live) {
                const float* up = Uf + 2 * pr;
#pragma unroll 4
                for (int p = p0 + sub; p < p1; p += kSpreadSub) {
                    const float2 uu = *(const float2*)(up + p * suf);
                    const float4 yv = Y[p];
                    a00.s = fmaf(uu.x, yv.x, a00.s);
                    a01.s = fmaf(uu.x, yv.z, a01.s);
                    a10.s = fmaf(uu.y, yv.x, a10.s);
                    a11.s = fmaf(uu.y, yv.z, a11.s);
                }
            }
            acc2* accs[4] = {&a00, &a01, &a10, &a11};
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                acc2 a = *accs[f];
#pragma unroll
                for (int off = kSpreadSub >> 1; off > 0; off >>= 1) {
                    const float os = __shfl_xor_sync(0xffffffffu, a.s, off);
                    const float oc = __shfl_xor_sync(0xffffffffu, a.c, off);
                    float s2, q2;
                    two_sum(a.s, os, s2, q2);
                    a.s = s2;
                    a.c += oc + q2;
                }
                *accs[f] = a;
            }
            if (live && sub == 0) {
                const int e0 = dfi ? 2 * pr : Edf + 2 * pr;
                const df n00 = fast_two_sum(a00.s, a00.c), n01 = fast_two_sum(a01.s, a01.c);
                const df n10 = fast_two_sum(a10.s, a10.c), n11 = fast_two_sum(a11.s, a11.c);
                N[b * E + e0] = make_float4(n00.h, n00.l, n01.h, n01.l);
                N[b * E + e0 + 1] = make_float4(n10.h, n10.l, n11.h, n11.l);
            }
        }
        // beta_qk = s^q sum_{j >= k, j = k mod 2} t_j MC(j, k), t_j = C(q+j-1, j) eta^j,
        // MC(j, k) = 2^(1-j) C(j, (j-k)/2) (halved for k = 0); on the last
        // threads, which have the fewest items of (a)
        for (int sl = nt - 1 - tid; sl < gn * Q; sl += nt) {
            const int b = sl / Q, q = sl - b * Q;
            const double R = B.rc + B.h * ((lfirst + g0 + b) + 0.5 * (w - 1));
            const df iR = df_recip(df_from(R));
            const df s = df_mul(rho, iR);
            const df eta = df_mul(df_from(0.5 * B.h), iR);
            df tj[kFoldMax];
            tj[0] = df{1.f, 0.f};
            for (int j = 0; j + 1 < K; ++j) {
                // t_{j+1} = t_j eta (q + j) / (j + 1)
                const float2 iv = kFoldC.inv[j];
                tj[j + 1] = df_mul(df_mul(tj[j], eta), df_mul_f(df{iv.x, iv.y}, (float)(q + j)));
            }
            // s^q by repeated squaring
            df sq{1.f, 0.f}, sp = s;
            for (int e = q; e > 0; e >>= 1) {
                if (e & 1) sq = df_mul(sq, sp);
                if (e > 1) sp = df_mul(sp, sp);
            }
            float2* bt = beta + (b * Q + q) * kBetaStride;
            for (int k = 0; k < K; ++k) {
                df acc{0.f, 0.f};
                for (int j = k; j < K; j += 2) acc = df_add(acc, df_mul_f(tj[j], kFoldC.mc[j][k]));
                const df bk = df_mul(sq, acc);
                bt[k] = make_float2(bk.h, bk.l);
            }
        }
        __syncthreads();
        // (b) M[d][q] = sum_k beta_qk (N[d+k] + N[|d-k|]) / 2 into the row order of Mb;
        // each item forms two consecutive q, so one sum N[d+k] + N[|d-k|]
        // (an unevaluated (hi, lo) pair) serves both
        for (int o = tid; o < gn * L.dpad * (Q >> 1); o += nt) {
            const int b = o / (L.dpad * (Q >> 1)), rem = o - b * (L.dpad * (Q >> 1));
            const int e = rem / (Q >> 1), q0 = 2 * (rem - e * (Q >> 1));
            const int d = mom_degree(e, L.ndf, dcs, nb);
            float2 mr0 = make_float2(0.f, 0.f), mi0 = mr0, mr1 = mr0, mi1 = mr0;
            if (d >= 0) {
                const float2* bt0 = beta + (b * Q + q0) * kBetaStride;
                const float2* bt1 = bt0 + kBetaStride;
                const float4* Nb = N + b * E;
                const float4 n0 = Nb[d];
                const bool dfe = e < 2 * L.ndf;
                if (dfe && q0 < qs) {
                    const bool df1 = q0 + 1 < qs;
                    acc2 ar0{0.f, 0.f}, ai0{0.f, 0.f}, ar1{0.f, 0.f}, ai1{0.f, 0.f};
                    const float2 b00 = bt0[0], b10 = bt1[0];
                    acc_fma(ar0, df{b00.x, b00.y}, df{n0.x, n0.y});
                    acc_fma(ai0, df{b00.x, b00.y}, df{n0.z, n0.w});
                    if (df1) {
                        acc_fma(ar1, df{b10.x, b10.y}, df{n0.x, n0.y});
                        acc_fma(ai1, df{b10.x, b10.y}, df{n0.z, n0.w});
                    } else {
                        ar1.s = b10.x * n0.x;
                        ai1.s = b10.x * n0.z;
                    }
                    for (int k = 1; k < K; ++k) {
                        const float4 n1 = Nb[d + k], n2 = Nb[d >= k ? d - k : k - d];
                        float sr, er, si, ei;
                        two_sum(n1.x, n2.x, sr, er);
                        two_sum(n1.z, n2.z, si, ei);
                        const df Sr{sr, er + (n1.y + n2.y)}, Si{si, ei + (n1.w + n2.w)};
                        const float2 bk0 = bt0[k], bk1 = bt1[k];
                        acc_fma(ar0, df{0.5f * bk0.x, 0.5f * bk0.y}, Sr);
                        acc_fma(ai0, df{0.5f * bk0.x, 0.5f * bk0.y}, Si);
                        if (df1) {
                            acc_fma(ar1, df{0.5f * bk1.x, 0.5f * bk1.y}, Sr);
                            acc_fma(ai1, df{0.5f * bk1.x, 0.5f * bk1.y}, Si);
                        } else {
                            ar1.s = fmaf(0.5f * bk1.x, sr, ar1.s);
                            ai1.s = fmaf(0.5f * bk1.x, si, ai1.s);
                        }
                    }
                    df v = fast_two_sum(ar0.s, ar0.c);
                    mr0 = make_float2(v.h, v.l);
                    v = fast_two_sum(ai0.s, ai0.c);
                    mi0 = make_float2(v.h, v.l);
                    if (df1) {
                        v = fast_two_sum(ar1.s, ar1.c);
                        mr1 = make_float2(v.h, v.l);
                        v = fast_two_sum(ai1.s, ai1.c);
                        mi1 = make_float2(v.h, v.l);
                    } else {
                        mr1 = make_float2(ar1.s, 0.f);
                        mi1 = make_float2(ai1.s, 0.f);
                    }
                } else {
                    const float b00 = bt0[0].x, b10 = bt1[0].x;
                    float fr0 = b00 * n0.x, fi0 = b00 * n0.z, fr1 = b10 * n0.x, fi1 = b10 * n0.z;
                    for (int k = 1; k < K; ++k) {
                        const float4 n1 = Nb[d + k], n2 = Nb[d >= k ? d - k : k - d];
                        const float sr = n1.x + n2.x, si = n1.z + n2.z;
                        const float h0 = 0.5f * bt0[k].x, h1 = 0.5f * bt1[k].x;
                        fr0 = fmaf(h0, sr, fr0);
                        fi0 = fmaf(h0, si, fi0);
                        fr1 = fmaf(h1, sr, fr1);
                        fi1 = fmaf(h1, si, fi1);
                    }
                    mr0 = make_float2(fr0, 0.f);
                    mi0 = make_float2(fi0, 0.f);
                    mr1 = make_float2(fr1, 0.f);
                    mi1 = make_float2(fi1, 0.f);
                }
            }
            float2* mo = Mb + (b * L.dpad + e) * Q2s + 2 * q0;
            mo[0] = mr0;
            mo[1] = mi0;
            mo[2] = mr1;
            mo[3] = mi1;
        }
        __syncthreads();
        // (c) grid[lfirst + g0 + c][q'] += sum_b sum_d A[c - b][d] M_b[d][q'] over
        // the group's bins b with 0 <= c - b < w
        const int ncell = gn + w - 1;
        for (int o = tid; o < ncell * Q2; o += nt) {
            const int c = o / Q2, qv = o - c * Q2;
            const int idx = lfirst + g0 + c + B.N1;
            if (idx < 0 || idx >= nf1) continue;
            const int b_lo = c - w + 1 > 0 ? c - w + 1 : 0;
            const int b_hi = c < gn - 1 ? c : gn - 1;
            const bool dq = (qv >> 1) < qs;
            acc2 sacc{0.f, 0.f};
            for (int b = b_lo; b <= b_hi; ++b) {
                const float2* ar = Ach + (c - b) * L.dpad;
                const float2* mb = Mb + b * L.dpad * Q2s + qv;
                float sf = 0.f;
                int e = 0;
                if (dq) {
                    for (; e < 2 * L.ndf; ++e) {
                        const float2 a2 = ar[e], m2 = mb[e * Q2s];
                        acc_fma(sacc, df{a2.x, a2.y}, df{m2.x, m2.y});
                    }
                }
                for (; e < L.dpad; ++e) sf = fmaf(ar[e].x, mb[e * Q2s].x, sf);
                float s2, e2;
                two_sum(sacc.s, sf, s2, e2);
                sacc.s = s2;
                sacc.c += e2;
            }
            const double val = acc_value(sacc);
            if (val != 0.0) gv.add(2 * ((int64_t)idx * Q + (qv >> 1)) + (qv & 1), val);
        }
        // no barrier here: (c) reads Ach and Mb only, the next group's (a)
        // and beta write N and beta, and its (b) writes Mb after a barrier
    }
    }
}

// Sparse tile (points spread over many cells): each thread prepares one point
// (cell l0, w kernel taps, the 2M weighted, pre-phased values), then each
// (cell, q) output of the tile's window is owned by one thread, which sums
// over the points whose taps cover that cell and adds the sum to the block's
// global grid.  Members as in spread_fold: the taps and phase factors are
// formed once, the weighted values and the sums per member.
template <bool MULTI, class Acc>
__device__ void spread_taps(const AsyBlock& B, int Q, const Tile& t, const Tables& tab,
                            const double* __restrict__ r_s, const float2* __restrict__ r2,
                            const float2* __restrict__ c2, int64_t c_stride, int V, int64_t moff, Acc gb,
                            float4* smem4)
{
    const int w = tab.w, deg = tab.deg, nt = blockDim.x, tid = threadIdx.x;
    const int ncoef = w * (deg + 1);
    float4* aval = smem4;                                   // [nt][Q]: (re.h, re.l, im.h, im.l)
    float2* coef = (float2*)(aval + nt * Q);                // [w][deg+1]
    float2* taps = coef + ncoef;                            // [nt][w]
    int* l0s = (int*)(taps + nt * w);                       // [nt]
    for (int i = tid; i < ncoef; i += nt) coef[i] = tab.es2[i];
    __syncthreads();
    const int cnt = t.count;
    const int64_t j = t.start + tid;
    df yr{0.f, 0.f}, yi{0.f, 0.f}, rat{0.f, 0.f};   // this point's weight without c_j, and its ratio
    if (tid < cnt) {
        long long X;
        df vd;
        l0s[tid] = spread_cell_fx(B, w, r_s[j], &X, &vd);
        const float vh = vd.h, vl = vd.l;
        for (int i = 0; i < w; ++i) {
            const df tp = horner_comp(coef + i * (deg + 1), deg, vh, vl, tab.deg_comp);
            taps[tid * w + i] = make_float2(tp.h, tp.l);
        }
        spread_weight_fx(B, tab.tw2, X, r2[j], MULTI ? make_float2(1.f, 0.f) : c2[j], &yr, &yi, &rat);
        if (!MULTI) {
            for (int q = 0; q < Q; ++q) {
                aval[tid * Q + q] = make_float4(yr.h, yr.l, yi.h, yi.l);
                yr = df_mul(yr, rat);
                yi = df_mul(yi, rat);
            }
        }
    }
    __syncthreads();
    const int lfirst = l0s[0];
    const int span = l0s[cnt - 1] - lfirst + w;
    const int nf1 = 2 * B.N1 + 1;
    // Outputs (cell, q), q fastest.  For a tile whose span of cells is close
    // to the kernel width every thread walks all the tile's points in
    // lockstep (one row of taps / values per step: broadcast or contiguous
    // reads) and skips points whose taps miss its cell; otherwise it
    // binary-searches the few points that reach its cell.  Each output is
    // split between kSub lanes (halves of the point range) combined by a
    // shuffle, so that more threads than outputs can work.
    constexpr int kSub = 2;
    const bool dense = span <= 2 * w;
    const int nout = span * Q;
    const int lane = tid & 31;
    const int sub = lane & (kSub - 1);
    const unsigned gmask = 0x3u << (lane & ~(kSub - 1));
    const int half = (cnt + 1) >> 1;
    for (int vm = 0; vm < (MULTI ? V : 1); ++vm) {
    if (MULTI) {
        if (tid < cnt) {
            const float2 cv = c2[vm * c_stride + j];
            df wr = df_mul(df{cv.x, cv.y}, yr), wi = df_mul(df{cv.x, cv.y}, yi);
            for (int q = 0; q < Q; ++q) {
                aval[tid * Q + q] = make_float4(wr.h, wr.l, wi.h, wi.l);
                wr = df_mul(wr, rat);
                wi = df_mul(wi, rat);
            }
        }
        __syncthreads();
    }
    const Acc gv = gb.at(vm * moff);
    for (int base = tid - sub; base < nout * kSub; base += nt) {
        const int item = (base + sub) / kSub;   // same item for both lanes of a pair
        const bool live = item < nout;
        const int c = live ? item / Q : 0, q = live ? item - c * Q : 0;
        const int cell = lfirst + c;
        int p_lo, p_hi;
        if (dense) {
            p_lo = sub * half;
            p_hi = sub ? cnt : half;
        } else {
            int lo = 0, hi = cnt;
            const int key = cell - w + 1;
            while (lo < hi) { int mid = (lo + hi) >> 1; if (l0s[mid] < key) lo = mid + 1; else hi = mid; }
            const int plo = lo;
            hi = cnt;
            while (lo < hi) { int mid = (lo + hi) >> 1; if (l0s[mid] <= cell) lo = mid + 1; else hi = mid; }
            const int mid2 = (plo + lo + 1) >> 1;
            p_lo = sub ? mid2 : plo;
            p_hi = sub ? lo : mid2;
        }
        if (!live) p_hi = p_lo;
        acc2 ar{0.f, 0.f}, ai{0.f, 0.f};
        for (int p = p_lo; p < p_hi; ++p) {
            const int i = cell - l0s[p];
            if (i >= 0 && i < w) {
                const float2 k2 = taps[p * w + i];
                const float4 av = aval[p * Q + q];
                const df k{k2.x, k2.y};
                acc_fma(ar, k, df{av.x, av.y});
                acc_fma(ai, k, df{av.z, av.w});
            }
        }
        double vr = acc_value(ar), vi = acc_value(ai);
        vr += __shfl_down_sync(gmask, vr, 1, kSub);
        vi += __shfl_down_sync(gmask, vi, 1, kSub);
        const int idx = cell + B.N1;
        if (live && sub == 0 && idx >= 0 && idx < nf1 && (vr != 0.0 || vi != 0.0)) {
            gv.add(2 * ((int64_t)idx * Q + q), vr);
            gv.add(2 * ((int64_t)idx * Q + q) + 1, vi);
        }
    }
    if (MULTI) __syncthreads();   // aval is rewritten for the next member
    }
}

// One CTA per tile of consecutive (sorted) points of one block; the tile
// takes the moment path when its points are dense in the grid's bins.
// Path of a spreading tile, packed: bits 0-1 the path (0 taps, 1 plain
// moments, 2 q-folded moments), bits 2-5 the fold's K, bits 6-11 its E,
// bits 12-17 its Edf.  The path depends only on the sorted points and the
// block, so it is decided once per plan (k_spread_modes).
__device__ __forceinline__ FoldPlan fold_unpack(int mode)
{
    return FoldPlan{(mode >> 2) & 15, (mode >> 6) & 63, (mode >> 12) & 63};
}

__global__ void k_spread_modes(const ProbParams* __restrict__ probs, const AsyBlock* __restrict__ blks,
                               const Tile* __restrict__ tiles, int ntiles, Tables tab,
                               const double* __restrict__ r_s, int32_t* __restrict__ modes)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ntiles; i += gridDim.x * blockDim.x) {
        const Tile t = tiles[i];
        int mode = 0;
        if (t.count > 0) {
            const AsyBlock B = blks[t.blk];
            long long X;
            df vd;
            const int lfirst = spread_cell_fx(B, tab.w, r_s[t.start], &X, &vd);
            const int nbins = spread_cell_fx(B, tab.w, r_s[t.start + t.count - 1], &X, &vd) - lfirst + 1;
            if (nbins <= kMaxTileBins && t.count >= kMomMinPerBin * nbins) {
                mode = 1;
                FoldPlan fp;
                if (fold_plan(B, tab, probs[B.prob].Q, lfirst, &fp))
                    mode = 2 | (fp.K << 2) | (fp.E << 6) | (fp.Edf << 12);
            }
        }
        modes[i] = mode;
    }
}

// One instance per accumulation mode (DET: the deterministic mode's exact
// fixed-point sums), so that the FP64 path carries no code of the other.
// Members: V real components (coefficients c2 + vm c_stride, grids grid_b +
// vm gb_stride) spread by the same CTAs, which form each point's cell, basis
// or taps and phase factor once.  MULTI: the instance for V > 1 (V = 1 runs
// the instance without the member loop's registers and barriers).
template <bool DET, bool MULTI>
__global__ void k_asy_spread(const ProbParams* __restrict__ probs, const AsyBlock* __restrict__ blks,
                             const Tile* __restrict__ tiles, const int32_t* __restrict__ modes, Tables tab,
                             const double* __restrict__ r_s, const float2* __restrict__ r2,
                             const float2* __restrict__ c2, int64_t c_stride, int V,
                             double2* __restrict__ grid_b, int64_t gb_stride)
{
    extern __shared__ float4 smem4[];
    const Tile t = tiles[blockIdx.x];
    if (t.count <= 0) return;
    const int mode = modes[blockIdx.x];
    const AsyBlock B = blks[t.blk];
    const int Q = probs[B.prob].Q;
    using Acc = typename AccumOf<DET>::type;
    const Acc gb = Acc{(double*)grid_b, probs[B.prob].fxs}.at(2 * B.b_off);
    const int64_t moff = 2 * gb_stride;
    if ((mode & 3) == 2)
        spread_fold<MULTI>(B, Q, probs[B.prob].qs, t, tab, fold_unpack(mode), r_s, r2, c2, c_stride, V, moff, gb,
                           smem4);
    else if (mode & 3) {
        // c_j (r_j/rho)^(-q-1/2) e^{i w_c x_j} onto the 2 N1 + 1 modes
        const int nf1 = 2 * B.N1 + 1;
        df yr{0.f, 0.f}, yi{0.f, 0.f}, rat{0.f, 0.f};   // this thread's point's weight without c_j
        int64_t jt = 0;
        auto put = [&](float2* xq, float2 cv) {
            df wr = df_mul(df{cv.x, cv.y}, yr), wi = df_mul(df{cv.x, cv.y}, yi);
            for (int q = 0; q < Q; ++q) {
                xq[2 * q] = make_float2(wr.h, wr.l);
                xq[2 * q + 1] = make_float2(wi.h, wi.l);
                wr = df_mul(wr, rat);
                wi = df_mul(wi, rat);
            }
        };
        spread_moments(Q, probs[B.prob].qs, t, tab,
            [&](int64_t j, df* v, float2* xq) {
                long long Xp;
                const int l0 = spread_cell_fx(B, tab.w, r_s[j], &Xp, v);
                spread_weight_fx(B, tab.tw2, Xp, r2[j], make_float2(1.f, 0.f), &yr, &yi, &rat);
                jt = j;
                put(xq, c2[j]);
                return l0;
            },
            [&](int vm, float2* xq) { put(xq, c2[vm * c_stride + jt]); }, MULTI ? V : 1, moff,
            [&](int c) -> int64_t { const int x = c + B.N1; return (x >= 0 && x < nf1) ? x : -1; },
            gb, (float2*)smem4);
    }
    else
        spread_taps<MULTI>(B, Q, t, tab, r_s, r2, c2, c_stride, V, moff, gb, smem4);
}

// -------------------------------------------------------------------- FFT
// Complex double-float values are float4 (re.h, re.l, im.h, im.l); the FFTs
// run in double-float on the FP32 pipes (FP64 is 1/64 of the FP32 rate).
__device__ __forceinline__ float4 cdf(df re, df im) { return make_float4(re.h, re.l, im.h, im.l); }

__device__ __forceinline__ float4 cdf_mul(float4 a, float4 b)
{
    const df ar{a.x, a.y}, ai{a.z, a.w}, br{b.x, b.y}, bi{b.z, b.w};
    return cdf(df_add(df_mul(ar, br), df_negate(df_mul(ai, bi))), df_add(df_mul(ar, bi), df_mul(ai, br)));
}

__device__ __forceinline__ float4 cdf_scale(float4 a, df s)
{
    return cdf(df_mul(df{a.x, a.y}, s), df_mul(df{a.z, a.w}, s));
}

// u + v w and u - v w
__device__ __forceinline__ void cdf_butterfly(float4& u, float4& v, float4 w)
{
    const float4 vw = cdf_mul(v, w);
    const df ur{u.x, u.y}, ui{u.z, u.w}, vr{vw.x, vw.y}, vi{vw.z, vw.w};
    u = cdf(df_add(ur, vr), df_add(ui, vi));
    v = cdf(df_add(ur, df_negate(vr)), df_add(ui, df_negate(vi)));
}

// The same on the FP32 parts (x, z) alone (mixed-precision FFTs): the low
// parts of the results are zero.
__device__ __forceinline__ float4 cf_mul(float4 a, float4 b)
{
    return make_float4(a.x * b.x - a.z * b.z, 0.f, a.x * b.z + a.z * b.x, 0.f);
}

__device__ __forceinline__ void cf_butterfly(float4& u, float4& v, float4 w)
{
    const float4 vw = cf_mul(v, w);
    const float ur = u.x, ui = u.z;
    u = make_float4(ur + vw.x, 0.f, ui + vw.z, 0.f);
    v = make_float4(ur - vw.x, 0.f, ui - vw.z, 0.f);
}

// A finite double as double-float from its bits (integer and FP32
// instructions only; FP64 runs at 1/64 of the FP32 rate): the top 24 bits of
// the significand exactly, the next 29 rounded; zero and subnormals give 0.
__device__ __forceinline__ df df_from_bits(double x)
{
    const long long b = __double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7ff);
    if (e == 0) return df{0.f, 0.f};
    const long long m = (b & 0xFFFFFFFFFFFFFLL) | (1LL << 52);   // x = +-m 2^(e - 1075)
    float h = ldexpf((float)(int)(m >> 29), e - 1075 + 29);
    float l = ldexpf((float)(int)(m & 0x1FFFFFFF), e - 1075);
    if (b < 0) {
        h = -h;
        l = -l;
    }
    return fast_two_sum(h, l);
}

// FP64 complex as double-float
__device__ __forceinline__ float4 cdf_from(double2 v)
{
    return cdf(df_from_bits(v.x), df_from_bits(v.y));
}

// nlines independent FFTs (e^{+2 pi i k n / N}) of N = 2^logN points stored
// one after the other in shared memory, each in bit-reversed order, sharing
// every butterfly stage.  tw2[k] = e^{2 pi i k / 2^tw_log2} as double-float.
// LOWP: the butterflies in FP32 on the values' FP32 parts (mixed precision).
// The decimation-in-time stages run two at a time (radix 4): a thread loads
// the four values a group of stages st, st + 1 combines (offsets 0, len,
// 2 len, 3 len), applies both stages' butterflies in registers and stores them
// back, so each value crosses shared memory once per two stages and the CTA
// synchronises half as often.  An odd stage count starts with one radix-2
// stage (twiddle 1).
template <bool LOWP>
__device__ __forceinline__ void fft_bfly(float4& u, float4& v, float4 w)
{
    if (LOWP) cf_butterfly(u, v, w);
    else cdf_butterfly(u, v, w);
}

template <bool LOWP>
__device__ void smem_fft_lines(float4* X, int logN, int nlines, const float4* __restrict__ tw2, int tw_log2)
{
    const int N = 1 << logN;
    int st = 0;
    if (logN & 1) {
        const int half = N >> 1;
        const float4 one = tw2[0];
        for (int b = threadIdx.x; b < nlines * half; b += blockDim.x) {
            const int i0 = 2 * b;   // stage 0: pairs (2b, 2b + 1), twiddle 1
            float4 u = X[i0], v = X[i0 + 1];
            fft_bfly<LOWP>(u, v, one);
            X[i0] = u;
            X[i0 + 1] = v;
        }
        __syncthreads();
        st = 1;
    }
    const int quarter = N >> 2;
    for (; st < logN; st += 2) {
        const int len = 1 << st;
        const int sh1 = tw_log2 - (st + 1), sh2 = tw_log2 - (st + 2);
        for (int b = threadIdx.x; b < nlines * quarter; b += blockDim.x) {
            const int line = b >> (logN - 2);
            const int bb = b & (quarter - 1);
            const int pos = bb & (len - 1);
            const int i0 = line * N + ((bb >> st) << (st + 2)) + pos;
            float4 a = X[i0], c1 = X[i0 + len], c2 = X[i0 + 2 * len], c3 = X[i0 + 3 * len];
            const float4 t1 = tw2[pos << sh1];
            fft_bfly<LOWP>(a, c1, t1);                       // stage st: (0, len), (2 len, 3 len)
            fft_bfly<LOWP>(c2, c3, t1);
            fft_bfly<LOWP>(a, c2, tw2[pos << sh2]);          // stage st + 1: (0, 2 len), (len, 3 len)
            fft_bfly<LOWP>(c1, c3, tw2[(pos + len) << sh2]);
            X[i0] = a;
            X[i0 + len] = c1;
            X[i0 + 2 * len] = c2;
            X[i0 + 3 * len] = c3;
        }
        __syncthreads();
    }
}

// The mixed-precision FFT on FP32 complex values (float2: re, im) in shared
// memory: the stages of smem_fft_lines on half the bytes per value, with the
// twiddles' FP32 parts.
__device__ __forceinline__ void cf2_bfly(float2& u, float2& v, float4 w)
{
    const float vr = v.x * w.x - v.y * w.z, vi = fmaf(v.x, w.z, v.y * w.x);
    const float ur = u.x, ui = u.y;
    u = make_float2(ur + vr, ui + vi);
    v = make_float2(ur - vr, ui - vi);
}

__device__ void smem_fft_lines_f32(float2* X, int logN, int nlines, const float4* __restrict__ tw2, int tw_log2)
{
    const int N = 1 << logN;
    int st = 0;
    if (logN & 1) {
        const int half = N >> 1;
        for (int b = threadIdx.x; b < nlines * half; b += blockDim.x) {
            const int i0 = 2 * b;
            const float2 u = X[i0], v = X[i0 + 1];
            X[i0] = make_float2(u.x + v.x, u.y + v.y);
            X[i0 + 1] = make_float2(u.x - v.x, u.y - v.y);
        }
        __syncthreads();
        st = 1;
    }
    const int quarter = N >> 2;
    for (; st < logN; st += 2) {
        const int len = 1 << st;
        const int sh1 = tw_log2 - (st + 1), sh2 = tw_log2 - (st + 2);
        for (int b = threadIdx.x; b < nlines * quarter; b += blockDim.x) {
            const int line = b >> (logN - 2);
            const int bb = b & (quarter - 1);
            const int pos = bb & (len - 1);
            const int i0 = line * N + ((bb >> st) << (st + 2)) + pos;
            float2 a = X[i0], c1 = X[i0 + len], c2 = X[i0 + 2 * len], c3 = X[i0 + 3 * len];
            const float4 t1 = tw2[pos << sh1];
            cf2_bfly(a, c1, t1);
            cf2_bfly(c2, c3, t1);
            cf2_bfly(a, c2, tw2[pos << sh2]);
            cf2_bfly(c1, c3, tw2[(pos + len) << sh2]);
            X[i0] = a;
            X[i0 + len] = c1;
            X[i0 + 2 * len] = c2;
            X[i0 + 3 * len] = c3;
        }
        __syncthreads();
    }
}

__device__ __forceinline__ float2 cf2_of(float4 v) { return make_float2(v.x, v.z); }
__device__ __forceinline__ float4 cf4_of(float2 v) { return make_float4(v.x, 0.f, v.y, 0.f); }

// e^{2 pi i m / N} for 0 <= m < N = 2^logN as double-float: the table entry for
// the top bits of m / N times the rotation by the rest, an angle below
// 2 pi / 2^tw_log2, from its Taylor series (five terms, truncation < 1e-19).
__device__ __forceinline__ float4 cdf_twiddle(const Tables& tab, int logN, long long m)
{
    const int sh = logN - tab.tw_log2;
    const int hi = sh > 0 ? (int)(m >> sh) : (int)(m << -sh);   // table index, < 2^tw_log2
    const int half = 1 << (tab.tw_log2 - 1);
    float4 t = tab.tw2[hi & (half - 1)];
    if (hi >= half) t = make_float4(-t.x, -t.y, -t.z, -t.w);
    const int lo = sh > 0 ? (int)(m & ((1LL << sh) - 1)) : 0;
    if (lo == 0) return t;
    // angle 2 pi lo / N: lo / N is exact in FP32 (lo < 2^sh <= 2^11, N a power of two)
    const df twopi{6.2831854820251465f, -1.7484555314695172e-07f};
    const df a = df_mul(twopi, df{ldexpf((float)lo, -logN), 0.f});
    const df a2 = df_mul(a, a);
    // sin a = a (1 - a^2/6 (1 - a^2/20 (1 - a^2/42))), cos a = 1 - a^2/2 (1 - a^2/12 (1 - a^2/30))
    df sn = df_add(df{1.f, 0.f}, df_negate(df_mul(a2, df{1.f / 42.f, 0.f})));
    sn = df_add(df{1.f, 0.f}, df_negate(df_mul(df_mul(a2, df{0.05f, -7.450580707946131e-10f}), sn)));
    sn = df_add(df{1.f, 0.f}, df_negate(df_mul(df_mul(a2, df{0.1666666716337204f, -4.967053879312289e-09f}), sn)));
    sn = df_mul(a, sn);
    df cs = df_add(df{1.f, 0.f}, df_negate(df_mul(a2, df{0.03333333507180214f, -1.7384682293e-09f})));
    cs = df_add(df{1.f, 0.f}, df_negate(df_mul(df_mul(a2, df{0.0833333358168602f, -2.4835269e-09f}), cs)));
    cs = df_add(df{1.f, 0.f}, df_negate(df_mul(df_mul(a2, df{0.5f, 0.f}), cs)));
    return cdf_mul(t, cdf(cs, sn));
}

// Split of a two-pass FFT of 2^LN points into lines: N2 = 2^ceil(LN/2)
// points per pass-A line, N1 = 2^floor(LN/2) per pass-B line; each CTA takes
// as many lines as fit kFftLineBatch points.
struct FourStep {
    int logN1, logN2, N1, N2, lpcA, lpcB, groupsA, groupsB;
};
__host__ __device__ __forceinline__ FourStep four_step(int LN)
{
    FourStep f;
    f.logN2 = (LN + 1) >> 1;
    f.logN1 = LN - f.logN2;
    f.N1 = 1 << f.logN1;
    f.N2 = 1 << f.logN2;
    f.lpcA = kFftLineBatch >> f.logN2; if (f.lpcA < 1) f.lpcA = 1;
    f.lpcB = kFftLineBatch >> f.logN1; if (f.lpcB < 1) f.lpcB = 1;
    f.groupsA = (f.N1 + f.lpcA - 1) / f.lpcA;
    f.groupsB = (f.N2 + f.lpcB - 1) / f.lpcB;
    return f;
}

// 1 / psi^(alpha2 l): the correction of mode l of the inner FFT, in
// double-float (|l| <= N1 < 2^24 is exact in FP32).
__device__ __forceinline__ df mode_correction(const AsyBlock& B, const Tables& tab, int l)
{
    const df a2 = df_from_bits(B.alpha2);
    return df_recip(psihat_of(tab, df_mul(a2, df{(float)(l < 0 ? -l : l), 0.f})));
}

// FFT input / output of the forward (ADJ = false) and the transposed
// (ADJ = true) type-3 pipelines.  Forward: modes l (|l| <= N1) of the spread
// grid src (at b_off), corrected by 1/psi^(alpha2 l), transformed to every t
// and stored at dst + q_off.  Transposed: the target grid src (at q_off,
// every t) is transformed (the DFT matrix e^{2 pi i l t / nf2} is symmetric),
// and only the modes |l| <= N1 are kept, corrected, and stored at dst + b_off.
template <bool ADJ>
__device__ __forceinline__ float4 fft_in(const AsyBlock& B, const Tables& tab, const double2* __restrict__ src,
                                         int Q, int q, int tt)
{
    if (ADJ) return cdf_from(src[B.q_off + (int64_t)tt * Q + q]);
    const int l = (tt < (B.nf2 >> 1)) ? tt : tt - B.nf2;
    if (l < -B.N1 || l > B.N1) return make_float4(0.f, 0.f, 0.f, 0.f);
    return cdf_scale(cdf_from(src[B.b_off + (int64_t)(l + B.N1) * Q + q]), mode_correction(B, tab, l));
}

template <bool ADJ>
__device__ __forceinline__ void fft_out(const AsyBlock& B, const Tables& tab, float4* __restrict__ dst, int Q,
                                        int q, int tt, float4 v)
{
    if (!ADJ) {
        dst[B.q_off + (int64_t)tt * Q + q] = v;
        return;
    }
    const int l = (tt < (B.nf2 >> 1)) ? tt : tt - B.nf2;
    if (l < -B.N1 || l > B.N1) return;
    dst[B.b_off + (int64_t)(l + B.N1) * Q + q] = cdf_scale(v, mode_correction(B, tab, l));
}

template <bool ADJ, bool LOWP>
__global__ void k_asy_fft_small(const ProbParams* __restrict__ probs, const AsyBlock* __restrict__ blks,
                                const Tile* __restrict__ items, Tables tab,
                                const double2* __restrict__ src, float4* __restrict__ dst, int64_t src_stride,
                                int64_t dst_stride)
{
    extern __shared__ float4 Xs[];
    src += blockIdx.y * src_stride;   // member blockIdx.y of a batch of real components
    dst += blockIdx.y * dst_stride;
    const Tile it = items[blockIdx.x];
    const AsyBlock B = blks[it.blk];
    const int Q = probs[B.prob].Q;
    const int q = (int)it.start;
    const int N = B.nf2, logN = B.log2nf2;
    float2* Xf = reinterpret_cast<float2*>(Xs);   // LOWP: FP32 values
    for (int tt = threadIdx.x; tt < N; tt += blockDim.x) {
        const float4 v = fft_in<ADJ>(B, tab, src, Q, q, tt);
        if (LOWP) Xf[__brev(tt) >> (32 - logN)] = cf2_of(v);
        else Xs[__brev(tt) >> (32 - logN)] = v;
    }
    __syncthreads();
    if (LOWP) smem_fft_lines_f32(Xf, logN, 1, tab.tw2, tab.tw_log2);
    else smem_fft_lines<false>(Xs, logN, 1, tab.tw2, tab.tw_log2);
    for (int tt = threadIdx.x; tt < N; tt += blockDim.x)
        fft_out<ADJ>(B, tab, dst, Q, q, tt, LOWP ? cf4_of(Xf[tt]) : Xs[tt]);
}

// All Q grids of one small block (nf2 * Q <= kFftSmemMax) in one CTA: the
// deconvolution factor of each mode is computed once and used for every q;
// the Q transforms share every butterfly stage.  A launch takes the blocks
// with pts_lo < nf2 * Q <= pts_hi (the others return at once), so that small
// blocks run in CTAs sized for them.
template <bool ADJ, bool LOWP>
__global__ void k_asy_fft_block(const ProbParams* __restrict__ probs, const AsyBlock* __restrict__ blks,
                                const Tile* __restrict__ items, Tables tab,
                                const double2* __restrict__ src, float4* __restrict__ dst, int pts_lo, int pts_hi,
                                int64_t src_stride, int64_t dst_stride)
{
    extern __shared__ float4 Xs[];   // [Q][N], each grid bit-reversed
    src += blockIdx.y * src_stride;   // member blockIdx.y of a batch of real components
    dst += blockIdx.y * dst_stride;
    const Tile it = items[blockIdx.x];
    const AsyBlock B = blks[it.blk];
    const int Q = probs[B.prob].Q;
    const int pts = B.nf2 * Q;
    if (pts <= pts_lo || pts > pts_hi) return;
    const int N = B.nf2, logN = B.log2nf2, half = N >> 1;
    float2* Xf = reinterpret_cast<float2*>(Xs);   // LOWP: FP32 values
    auto put = [&](int i, float4 v) {
        if (LOWP) Xf[i] = cf2_of(v);
        else Xs[i] = v;
    };
    for (int tt = threadIdx.x; tt < N; tt += blockDim.x) {
        const int l = (tt < half) ? tt : tt - N;
        const int dst_i = __brev(tt) >> (32 - logN);
        if (ADJ) {
            const double2* row = src + B.q_off + (int64_t)tt * Q;
            for (int q = 0; q < Q; ++q) put(q * N + dst_i, cdf_from(row[q]));
        } else if (l < -B.N1 || l > B.N1) {
            for (int q = 0; q < Q; ++q) put(q * N + dst_i, make_float4(0.f, 0.f, 0.f, 0.f));
        } else {
            const df sc = mode_correction(B, tab, l);
            const double2* row = src + B.b_off + (int64_t)(l + B.N1) * Q;
            for (int q = 0; q < Q; ++q) put(q * N + dst_i, cdf_scale(cdf_from(row[q]), sc));
        }
    }
    __syncthreads();
    if (LOWP) smem_fft_lines_f32(Xf, logN, Q, tab.tw2, tab.tw_log2);
    else smem_fft_lines<false>(Xs, logN, Q, tab.tw2, tab.tw_log2);
    auto get = [&](int i) { return LOWP ? cf4_of(Xf[i]) : Xs[i]; };
    if (!ADJ) {
        float4* gq = dst + B.q_off;
        for (int idx = threadIdx.x; idx < N * Q; idx += blockDim.x) {
            const int tt = idx / Q, q = idx - tt * Q;
            gq[idx] = get(q * N + tt);
        }
    } else {
        const int nf1 = 2 * B.N1 + 1;
        float4* gb = dst + B.b_off;
        for (int li = threadIdx.x; li < nf1; li += blockDim.x) {
            const int l = li - B.N1;
            const df sc = mode_correction(B, tab, l);
            for (int q = 0; q < Q; ++q) gb[(int64_t)li * Q + q] = cdf_scale(get(q * N + (l & (N - 1))), sc);
        }
    }
}

// Two-pass (four-step) FFT for nf2 = N1 * N2 > kFftSingleMax.
// Pass A: for each n1, FFT over n2 of x[n1 + N1 n2], times e^{2 pi i n1 k2 / N},
// stored at tmp[n1 + N1 k2].  Pass B: for each k2, FFT over n1 of
// tmp[n1 + N1 k2], which is X[k2 + N2 k1].  Work item ordinal = g * Q + q,
// g a group of lines handled by one CTA: the Q CTAs of a group run side by
// side and read and write the same rows of the [point][Q] grids (one row is
// all Q values of a point), so a row moves through HBM once, not once per q.
template <bool ADJ, bool LOWP>
__global__ void k_asy_fft_pass_a(const ProbParams* __restrict__ probs, const AsyBlock* __restrict__ blks,
                                 const Tile* __restrict__ items, Tables tab,
                                 const double2* __restrict__ src, float4* __restrict__ tmp)
{
    extern __shared__ float4 Xs[];
    const Tile it = items[blockIdx.x];
    const AsyBlock B = blks[it.blk];
    const int Q = probs[B.prob].Q;
    const int N = B.nf2;
    const FourStep f = four_step(B.log2nf2);
    const int g = (int)(it.start / Q);
    const int iq = (int)(it.start - (int64_t)g * Q);
    const int l0 = g * f.lpcA;
    const int nl = (f.N1 - l0) < f.lpcA ? (f.N1 - l0) : f.lpcA;
    float2* Xf = reinterpret_cast<float2*>(Xs);   // LOWP: FP32 values
    for (int idx = threadIdx.x; idx < nl * f.N2; idx += blockDim.x) {
        const int li = idx >> f.logN2, n2 = idx & (f.N2 - 1);
        const int i = li * f.N2 + (__brev(n2) >> (32 - f.logN2));
        const float4 v = fft_in<ADJ>(B, tab, src, Q, iq, (l0 + li) + f.N1 * n2);
        if (LOWP) Xf[i] = cf2_of(v);
        else Xs[i] = v;
    }
    __syncthreads();
    if (LOWP) smem_fft_lines_f32(Xf, f.logN2, nl, tab.tw2, tab.tw_log2);
    else smem_fft_lines<false>(Xs, f.logN2, nl, tab.tw2, tab.tw_log2);
    for (int idx = threadIdx.x; idx < nl * f.N2; idx += blockDim.x) {
        const int li = idx >> f.logN2, k2 = idx & (f.N2 - 1);
        const int n1 = l0 + li;
        const long long m = ((long long)n1 * k2) & (N - 1);   // e^{2 pi i n1 k2 / N}
        const int64_t o = B.q_off + (int64_t)(n1 + f.N1 * k2) * Q + iq;
        if (LOWP) {
            // FP32 twiddle (m / N is exact in FP32, N <= 2^24); the pass
            // temporary holds FP32 complex values (float2, half the bytes)
            float sn, cs;
            sincospif(ldexpf(2.f * (float)m, -B.log2nf2), &sn, &cs);
            const float2 x = Xf[idx];
            reinterpret_cast<float2*>(tmp)[o] = make_float2(x.x * cs - x.y * sn, fmaf(x.x, sn, x.y * cs));
        } else {
            tmp[o] = cdf_mul(Xs[idx], cdf_twiddle(tab, B.log2nf2, m));
        }
    }
}

template <bool ADJ, bool LOWP>
__global__ void k_asy_fft_pass_b(const ProbParams* __restrict__ probs, const AsyBlock* __restrict__ blks,
                                 const Tile* __restrict__ items, Tables tab,
                                 const float4* __restrict__ tmp, float4* __restrict__ dst)
{
    extern __shared__ float4 Xs[];
    const Tile it = items[blockIdx.x];
    const AsyBlock B = blks[it.blk];
    const int Q = probs[B.prob].Q;
    const FourStep f = four_step(B.log2nf2);
    const int g = (int)(it.start / Q);
    const int iq = (int)(it.start - (int64_t)g * Q);
    const int k20 = g * f.lpcB;
    const int nl = (f.N2 - k20) < f.lpcB ? (f.N2 - k20) : f.lpcB;
    float2* Xf = reinterpret_cast<float2*>(Xs);   // LOWP: FP32 values
    for (int idx = threadIdx.x; idx < nl * f.N1; idx += blockDim.x) {
        const int li = idx >> f.logN1, n1 = idx & (f.N1 - 1);
        const int i = li * f.N1 + (f.logN1 > 0 ? (__brev(n1) >> (32 - f.logN1)) : 0);
        const int64_t o = B.q_off + (int64_t)(n1 + f.N1 * (k20 + li)) * Q + iq;
        if (LOWP) Xf[i] = reinterpret_cast<const float2*>(tmp)[o];
        else Xs[i] = tmp[o];
    }
    __syncthreads();
    if (LOWP) smem_fft_lines_f32(Xf, f.logN1, nl, tab.tw2, tab.tw_log2);
    else smem_fft_lines<false>(Xs, f.logN1, nl, tab.tw2, tab.tw_log2);
    for (int idx = threadIdx.x; idx < nl * f.N1; idx += blockDim.x) {
        const int li = idx >> f.logN1, k1 = idx & (f.N1 - 1);
        fft_out<ADJ>(B, tab, dst, Q, iq, (k20 + li) + f.N2 * k1, LOWP ? cf4_of(Xf[idx]) : Xs[idx]);
    }
}

// ------------------------------------------------------------ interpolate
// Shared bytes for the per-bin sums of a dense tile, per thread: room for
// threads / kMomMinPerBin bins (16 bins of a 256-frequency tile, 8 of a 128 one).
constexpr int kInterpHBytesPerThread = 128;
constexpr int kAdjInterpHBytes = kInterpHBytesPerThread * kAdjInterpThreads;

// Shared memory (bytes) of k_asy_interp for 2M = qmax.
__host__ __device__ __forceinline__ size_t interp_smem(int qmax, int w, int deg, int threads,
                                                      int hbytes)
{
    const int us = (deg + 1 > w ? deg + 1 : w) | 1;
    return sizeof(float4) * (size_t)kWinCells * qmax + sizeof(float2) * (size_t)((w * (deg + 1) + 1) & ~1) +
           hbytes + sizeof(float2) * (size_t)threads * us + sizeof(int) * threads;
}

// Per-bin sums of a staged window (dense interpolation tiles):
// H[b][d][q'] = sum_i A[i][d] G[b + i][q'], b < nbins, A[i][d] the taps in the
// Chebyshev basis (coef2, [w][nb]) and G the window ([cells][Q] of (re_h,
// re_l, im_h, im_l)); bin stride nb 2Q + 2 float2.  Double-float for d < dci
// and q < qs (the targets read only the FP32 part of the rest); each thread
// forms two degrees x (re, im) of one q, four independent sums over the w
// cells.
__device__ __forceinline__ void bin_sums_build(const float4* win, const float2* coef2, float2* H, int nbins,
                                               int w, int nb, int dci, int Q, int qs, const int8_t* dcp)
{
    const int Q2 = 2 * Q, hs = nb * Q2 + 2;
    const int npr = (nb + 1) >> 1;
    // a tile of one or two bins has few items: one degree per item then, so
    // that twice as many threads share the work
    const int g2 = (nbins * npr * Q * 2 <= (int)blockDim.x) ? 1 : 2;   // degrees per item
    const int nper = g2 == 2 ? npr : nb;
    // q is the slowest index, so that a warp's items mostly share q (and with
    // it the double-float / FP32 branch)
    for (int o = threadIdx.x; o < nbins * nper * Q; o += blockDim.x) {
        const int q = o / (nbins * nper), rem = o - q * (nbins * nper);
        const int b = rem / nper, dp = rem - b * nper;
        const int d0 = g2 * dp, d1 = d0 + 1;
        const bool has1 = g2 == 2 && d1 < nb;
        float2* h0 = H + b * hs + d0 * Q2 + 2 * q;
        if (d0 < min(dci, (int)dcp[q >> 1]) && q < qs) {
            acc2 a0r{0.f, 0.f}, a0i{0.f, 0.f}, a1r{0.f, 0.f}, a1i{0.f, 0.f};
            if (has1) {
#pragma unroll 4
                for (int i = 0; i < w; ++i) {
                    const float4 gv = win[(b + i) * Q + q];
                    const float2 c0 = coef2[i * nb + d0];
                    const float2 c1 = coef2[i * nb + d1];
                    const df gr{gv.x, gv.y}, gi{gv.z, gv.w};
                    acc_fma(a0r, df{c0.x, c0.y}, gr);
                    acc_fma(a0i, df{c0.x, c0.y}, gi);
                    acc_fma(a1r, df{c1.x, c1.y}, gr);
                    acc_fma(a1i, df{c1.x, c1.y}, gi);
                }
            } else {
#pragma unroll 4
                for (int i = 0; i < w; ++i) {
                    const float4 gv = win[(b + i) * Q + q];
                    const float2 c0 = coef2[i * nb + d0];
                    acc_fma(a0r, df{c0.x, c0.y}, df{gv.x, gv.y});
                    acc_fma(a0i, df{c0.x, c0.y}, df{gv.z, gv.w});
                }
            }
            df v = fast_two_sum(a0r.s, a0r.c);
            h0[0] = make_float2(v.h, v.l);
            v = fast_two_sum(a0i.s, a0i.c);
            h0[1] = make_float2(v.h, v.l);
            if (has1) {
                v = fast_two_sum(a1r.s, a1r.c);
                h0[Q2] = make_float2(v.h, v.l);
                v = fast_two_sum(a1i.s, a1i.c);
                h0[Q2 + 1] = make_float2(v.h, v.l);
            }
        } else {
            float a0r = 0.f, a0i = 0.f, a1r = 0.f, a1i = 0.f;
#pragma unroll 4
            for (int i = 0; i < w; ++i) {
                const float4 gv = win[(b + i) * Q + q];
                const float c0 = coef2[i * nb + d0].x;
                const float c1 = has1 ? coef2[i * nb + d1].x : 0.f;
                a0r = fmaf(c0, gv.x, a0r);
                a0i = fmaf(c0, gv.z, a0i);
                a1r = fmaf(c1, gv.x, a1r);
                a1i = fmaf(c1, gv.z, a1i);
            }
            h0[0] = make_float2(a0r, 0.f);
            h0[1] = make_float2(a0i, 0.f);
            if (has1) {
                h0[Q2] = make_float2(a1r, 0.f);
                h0[Q2 + 1] = make_float2(a1i, 0.f);
            }
        }
    }
}

// A target's Chebyshev basis T_d(v), d < nb, into u (double-float for d < dci).
__device__ __forceinline__ void cheb_basis_row(float2* u, float vh, float vl, int dci, int nb)
{
    u[0] = make_float2(1.f, 0.f);
    u[1] = make_float2(vh, vl);
    df tm{1.f, 0.f}, tc{vh, vl};
    const df v2{2.f * vh, 2.f * vl};
    int d = 2;
    for (; d < dci; ++d) {
        const df tn = cheb_step(v2, tc, tm);
        u[d] = make_float2(tn.h, tn.l);
        tm = tc;
        tc = tn;
    }
    float fm = tm.h, fc = tc.h;
    for (; d < nb; ++d) {
        const float fn = fmaf(2.f * vh, fc, -fm);
        u[d] = make_float2(fn, 0.f);
        fm = fc;
        fc = fn;
    }
}

// P_q = sum_d T_d(v) H[d][q], q < Q (Q = 2M is even), handed to
// combine(q, re, im) in increasing q: Hankel terms in pairs, four independent
// sums over the degrees, one basis load per degree; from q = qs on in FP32
// (small Hankel terms).
template <class F>
__device__ __forceinline__ void bin_sums_eval(const float2* Hb, const float2* u, int nb, int dci, int Q, int qs,
                                              const int8_t* dcp, F&& combine)
{
    const int Q2 = 2 * Q;
    for (int q = 0; q < Q; q += 2) {
        const float2* hq = Hb + 2 * q;
        if (q < qs) {
            acc2 a0r{0.f, 0.f}, a0i{0.f, 0.f}, a1r{0.f, 0.f}, a1i{0.f, 0.f};
            const int dq = min(dci, (int)dcp[q >> 1]);
            int d = 0;
#pragma unroll 3
            for (; d < dq; ++d) {
                const float2 tp = u[d];
                const df t{tp.x, tp.y};
                const float4 h0 = *(const float4*)(hq + d * Q2);
                const float4 h1 = *(const float4*)(hq + d * Q2 + 2);
                acc_fma(a0r, t, df{h0.x, h0.y});
                acc_fma(a0i, t, df{h0.z, h0.w});
                acc_fma(a1r, t, df{h1.x, h1.y});
                acc_fma(a1i, t, df{h1.z, h1.w});
            }
            float f0r = 0.f, f0i = 0.f, f1r = 0.f, f1i = 0.f;
#pragma unroll 3
            for (; d < nb; ++d) {
                const float tp = u[d].x;
                const float4 h0 = *(const float4*)(hq + d * Q2);
                const float4 h1 = *(const float4*)(hq + d * Q2 + 2);
                f0r = fmaf(tp, h0.x, f0r);
                f0i = fmaf(tp, h0.z, f0i);
                f1r = fmaf(tp, h1.x, f1r);
                f1i = fmaf(tp, h1.z, f1i);
            }
            a0r.c += f0r;
            a0i.c += f0i;
            a1r.c += f1r;
            a1i.c += f1i;
            combine(q, fast_two_sum(a0r.s, a0r.c), fast_two_sum(a0i.s, a0i.c));
            combine(q + 1, fast_two_sum(a1r.s, a1r.c), fast_two_sum(a1i.s, a1i.c));
        } else {
            float p0r = 0.f, p0i = 0.f, p1r = 0.f, p1i = 0.f;
#pragma unroll 4
            for (int d = 0; d < nb; ++d) {
                const float tp = u[d].x;
                const float4 h0 = *(const float4*)(hq + d * Q2);
                const float4 h1 = *(const float4*)(hq + d * Q2 + 2);
                p0r = fmaf(tp, h0.x, p0r);
                p0i = fmaf(tp, h0.z, p0i);
                p1r = fmaf(tp, h1.x, p1r);
                p1i = fmaf(tp, h1.z, p1i);
            }
            combine(q, df{p0r, 0.f}, df{p0i, 0.f});
            combine(q + 1, df{p1r, 0.f}, df{p1i, 0.f});
        }
    }
}

// P_q = sum_i psi_i(v) G[i][q], q < Q, from the taps psi_i(v) in u (sparse
// tiles); cell(i, q) returns the grid value; FP32 from q = qs on.
template <class C, class F>
__device__ __forceinline__ void tap_sums_eval(const float2* u, int w, int Q, int qs, C&& cell, F&& combine)
{
    for (int q = 0; q < Q; ++q) {
        if (q < qs) {
            acc2 pr{0.f, 0.f}, pi{0.f, 0.f};
            for (int i = 0; i < w; ++i) {
                const float4 gv = cell(i, q);
                const float2 tp = u[i];
                acc_fma(pr, df{tp.x, tp.y}, df{gv.x, gv.y});
                acc_fma(pi, df{tp.x, tp.y}, df{gv.z, gv.w});
            }
            combine(q, fast_two_sum(pr.s, pr.c), fast_two_sum(pi.s, pi.c));
        } else {
            float pr = 0.f, pi = 0.f;
            for (int i = 0; i < w; ++i) {
                const float4 gv = cell(i, q);
                const float tp = u[i].x;
                pr = fmaf(tp, gv.x, pr);
                pi = fmaf(tp, gv.z, pi);
            }
            combine(q, df{pr, 0.f}, df{pi, 0.f});
        }
    }
}

// One thread per frequency: interpolate the 2M FFT grids at theta = s h,
// deconvolve, post-phase, and combine the Hankel terms into g.  A frequency
// at FFT-grid position a + w/2 reads the cells t0 + i, i < w, t0 = ceil(a),
// with taps psi_i(v).  Dense tiles (many frequencies per t0) form, once per
// bin, H[d][q'] = sum_i A[i][d] G[t0 + i][q'] (the taps in the Chebyshev
// basis, A[i][d]), and each frequency sums P_q' = sum_d T_d(v) H[d][q'];
// sparse tiles evaluate the w taps of each frequency.  Each thread keeps its
// basis (or taps) in a row of shared memory.
// Members: V real components (FFT outputs grid_q + vm gq_stride, sums into
// g_s + vm g_stride) interpolated by the same CTAs: a frequency's cell, basis
// or taps, phase and deconvolution factor are formed once; the window, the
// per-bin sums and the frequency's sums per member.
__global__ void __launch_bounds__(kInterpTileThreads, 3) k_asy_interp(
    const ProbParams* __restrict__ probs, const AsyBlock* __restrict__ blks, const Tile* __restrict__ tiles,
    Tables tab, const double* __restrict__ w_s, const float2* __restrict__ w2, const float4* __restrict__ grid_q,
    int64_t gq_stride, int V, double* __restrict__ g_s, int64_t g_stride)
{
    extern __shared__ float4 win[];          // [kWinCells][Q] grid cells of this tile
    const Tile t = tiles[blockIdx.x];
    const AsyBlock B = blks[t.blk];
    const ProbParams& P = probs[B.prob];
    const int w = tab.w, deg = tab.deg, nb = tab.nb, dci = tab.dci;
    const int Q = P.Q, Q2 = 2 * Q;
    const int us = (deg + 1 > w ? deg + 1 : w) | 1;
    const int hs = nb * Q2 + 2;                                  // bin stride of H (float2)
    float2* coef2 = (float2*)(win + kWinCells * Q);              // [w][deg + 1] taps, or [w][nb] Chebyshev
    float2* H = coef2 + ((w * (deg + 1) + 1) & ~1);              // [bins][hs], 16-byte aligned
    const int hbytes = kInterpHBytesPerThread * (int)blockDim.x;
    float2* U = H + hbytes / sizeof(float2);                     // [threads][us]
    int* t0s = (int*)(U + blockDim.x * us);                      // [threads]
    const bool valid = (int)threadIdx.x < t.count;
    const int64_t k = t.start + (valid ? threadIdx.x : 0);
    long long Om, Sw, svw;
    const int t0 = interp_cell_sv(B, tab.w, w_s[k], &Om, &Sw, &svw);
    const df vdf = df_from_sv(svw);
    const float vh = vdf.h, vl = vdf.l;
    // the tile's targets are sorted, so their cells form one window
    if (valid) t0s[threadIdx.x] = t0;
    __syncthreads();
    const int wstart = t0s[0];
    const int nbins = t0s[t.count - 1] - wstart + 1;
    const int wlen = nbins - 1 + w;
    const int mask = B.nf2 - 1;
    const bool staged = wlen <= kWinCells;
    const int maxbins = hbytes / (int)(sizeof(float2) * hs);
    const bool mom = staged && nbins <= maxbins && t.count >= kMomMinPerBin * nbins;
    if (mom) {
        for (int i = threadIdx.x; i < w * nb; i += blockDim.x) {
            const int r = i / nb, d = i - r * nb;
            coef2[i] = tab.ch2[r * (deg + 1) + d];
        }
    } else {
        for (int i = threadIdx.x; i < w * (deg + 1); i += blockDim.x) coef2[i] = tab.es2[i];
    }
    __syncthreads();
    // this thread's Chebyshev basis T_d(v) (dense tile) or taps psi_i(v), and
    // the member-independent factors of its output
    float2* u = U + threadIdx.x * us;
    df mz{0.f, 0.f}, sn{0.f, 0.f}, cs{0.f, 0.f}, scale{0.f, 0.f};
    if (valid) {
        if (mom) {
            cheb_basis_row(u, vh, vl, dci, nb);
        } else {
            for (int i = 0; i < w; ++i) {
                const df tp = horner_comp(coef2 + i * (deg + 1), deg, vh, vl, tab.deg_comp);
                u[i] = make_float2(tp.h, tp.l);
            }
        }
        const float2 wk2 = w2[k];
        const df m1d = df_recip(df_mul(df{wk2.x, wk2.y}, df{B.rho_h, B.rho_l}));   // 1/(omega rho) < 1/z
        mz = df_mul(m1d, df{P.z2.x, P.z2.y});                                       // z/(omega rho) < 1
        df_sincos_turns_tab(mul128_bits(Om, B.KRc, B.sR), tab.tw2, &sn, &cs);
        // sqrt(2/pi) (omega rho)^(-1/2) (4 / w^2) / psi^(alpha s)
        scale = df_mul(df_mul(df_sqrt(m1d), df_recip(psihat_fx(tab, B, Sw))), df{tab.ic2.x, tab.ic2.y});
        if (P.sgn < 0) scale = df_negate(scale);
    }
    const float2* Hb = H + (t0 - wstart) * hs;
    const int qs = P.qs;
    const df cph{P.cphi2.x, P.cphi2.y}, sph{P.sphi2.x, P.sphi2.y};
    for (int vm = 0; vm < V; ++vm) {
        const float4* gq = grid_q + vm * gq_stride + B.q_off;
        if (vm > 0) __syncthreads();   // the previous member's reads of the window and H are done
        if (staged) {
            for (int idx = threadIdx.x; idx < wlen * Q; idx += blockDim.x) {
                const int cc = idx / Q;
                win[idx] = gq[(int64_t)((wstart + cc) & mask) * Q + (idx - cc * Q)];
            }
        }
        __syncthreads();
        if (mom) {
            bin_sums_build(win, coef2, H, nbins, w, nb, dci, Q, qs, P.dcp);
            __syncthreads();
        }
        if (!valid) continue;
        // T = sum_q a_q i^q (omega rho)^(-q) P_q, accumulated in double-float
        acc2 tr{0.f, 0.f}, ti{0.f, 0.f};
        df mq{1.f, 0.f};
        auto combine = [&](int q, df prd, df pid) {
            if (q >= qs) {
                // small terms (FP32 sums, weights below 1e-8 of the first):
                // products and sums in FP32, into the compensation parts
                const float cq = P.a2[q].x * mq.h;
                switch (q & 3) {
                    case 0: tr.c = fmaf(cq, prd.h, tr.c); ti.c = fmaf(cq, pid.h, ti.c); break;
                    case 1: tr.c = fmaf(-cq, pid.h, tr.c); ti.c = fmaf(cq, prd.h, ti.c); break;
                    case 2: tr.c = fmaf(-cq, prd.h, tr.c); ti.c = fmaf(-cq, pid.h, ti.c); break;
                    default: tr.c = fmaf(cq, pid.h, tr.c); ti.c = fmaf(-cq, prd.h, ti.c); break;
                }
                mq.h *= mz.h;
                return;
            }
            const df cq = df_mul(df{P.a2[q].x, P.a2[q].y}, mq);
            // multiply by i^q: (pr + i pi) i^q
            switch (q & 3) {
                case 0: acc_fma(tr, cq, prd); acc_fma(ti, cq, pid); break;
                case 1: acc_fma(tr, df{-cq.h, -cq.l}, pid); acc_fma(ti, cq, prd); break;
                case 2: acc_fma(tr, df{-cq.h, -cq.l}, prd); acc_fma(ti, df{-cq.h, -cq.l}, pid); break;
                default: acc_fma(tr, cq, pid); acc_fma(ti, df{-cq.h, -cq.l}, prd); break;
            }
            mq = df_mul(mq, mz);
        };
        if (mom)
            bin_sums_eval(Hb, u, nb, dci, Q, qs, P.dcp, combine);
        else
            tap_sums_eval(u, w, Q, qs, [&](int i, int q) {
                return staged ? win[(t0 + i - wstart) * Q + q] : gq[(int64_t)((t0 + i) & mask) * Q + q];
            }, combine);
        // Re(e^{i (omega r_c + phi)} T) = Re(e^{i omega r_c} (e^{i phi} T))
        const df tre = fast_two_sum(tr.s, tr.c), tim = fast_two_sum(ti.s, ti.c);
        const df ur = df_add(df_mul(cph, tre), df_negate(df_mul(sph, tim)));
        const df ui = df_add(df_mul(sph, tre), df_mul(cph, tim));
        const df re = df_add(df_mul(cs, ur), df_negate(df_mul(sn, ui)));
        Accum{g_s + vm * g_stride, P.fxs}.add(k, df_to(df_mul(scale, re)));
    }
}

// ------------------------------------------------------------------ adjoint
// Transposed asymptotic block.  The forward map is
//   g = Re( D_out I W C S D_in c ),
// D_in = e^{i w_c x_j} (r_j/rho)^(-q-1/2) (per q), S = spreading, C =
// 1/psi^(alpha2 l), W = the DFT e^{2 pi i l t / nf2}, I = interpolation at
// theta_k, D_out = sqrt(2/pi) (4/w^2) / psi^(alpha s_k) (omega_k rho)^(-1/2)
// e^{i (omega_k r_c + phi)} a_q i^q (omega_k rho)^(-q).  Its transpose on real
// vectors is c = Re( D_in S^T C W I^T D_out g ) (every diagonal factor is
// symmetric, W is symmetric, S and I are real): the frequencies spread
// g_k D_out onto the FFT grid (I^T), the same FFT and correction follow, and
// the points interpolate the corrected modes (S^T) with D_in.

// The weighted values of frequency omega_k in the transposed interpolation
// (g_k D_out, one per Hankel term):
//   x_q = g_k sqrt(2/pi) (4/w^2) / psi^(alpha s) (omega rho)^(-1/2)
//         e^{i (omega r_c + phi)} i^q a_q z^-q (z/(omega rho))^q,
// as double-float (re, im) pairs xq[2q], xq[2q + 1]; returns the FFT-grid cell
// t0 of omega_k and its kernel coordinate v.
// The factor of g_k in those values, split as f = fr + i fi (q = 0, without
// g_k) and the ratio mz = z/(omega rho) of consecutive terms: one frequency's
// part that the real components of a group share.
struct AdjFactor {
    df fr, fi, mz;
};

__device__ __forceinline__ int adj_spread_factor(const AsyBlock& B, const ProbParams& P, const Tables& tab,
                                                 double wk, df* v, AdjFactor* F)
{
    long long Om, Sw, svw;
    const int t0 = interp_cell_sv(B, tab.w, wk, &Om, &Sw, &svw);
    *v = df_from_sv(svw);
    const df m1d = df_recip(df_from(wk * B.rho));
    F->mz = df_mul(m1d, df{P.z2.x, P.z2.y});
    df sn, cs;
    df_sincos_turns_tab(mul128_bits(Om, B.KRc, B.sR), tab.tw2, &sn, &cs);
    const df cph{P.cphi2.x, P.cphi2.y}, sph{P.sphi2.x, P.sphi2.y};
    const df er = df_add(df_mul(cs, cph), df_negate(df_mul(sn, sph)));
    const df ei = df_add(df_mul(sn, cph), df_mul(cs, sph));
    const df amp = df_mul(df_mul(df_from((double)P.sgn * tab.interp_const), df_sqrt(m1d)),
                          df_recip(psihat_fx(tab, B, Sw)));
    F->fr = df_mul(amp, er);
    F->fi = df_mul(amp, ei);
    return t0;
}

// The 2M values x_q for g_k from the frequency's factor.
__device__ __forceinline__ void adj_values(const ProbParams& P, const AdjFactor& F, double gk, float2* xq)
{
    const df g = df_from(gk);
    const df fr = df_mul(F.fr, g), fi = df_mul(F.fi, g), mz = F.mz;
    df mq{1.f, 0.f};
    for (int q = 0; q < P.Q; ++q) {
        const df cq = df_mul(df{P.a2[q].x, P.a2[q].y}, mq);
        // (fr + i fi) i^q cq
        df ur, ui;
        switch (q & 3) {
            case 0: ur = fr; ui = fi; break;
            case 1: ur = df_negate(fi); ui = fr; break;
            case 2: ur = df_negate(fr); ui = df_negate(fi); break;
            default: ur = fi; ui = df_negate(fr); break;
        }
        ur = df_mul(ur, cq);
        ui = df_mul(ui, cq);
        xq[2 * q] = make_float2(ur.h, ur.l);
        xq[2 * q + 1] = make_float2(ui.h, ui.l);
        mq = df_mul(mq, mz);
    }
}

// Frequencies of a tile -> FFT grid (periodic, atomics into tgrid).  Dense
// tiles (many frequencies per cell) take the per-bin moment path of the
// forward spreading; sparse tiles evaluate each frequency's w taps and sum,
// per grid cell, the frequencies that reach it.  Members: V real components
// (g_s + vm g_stride into tgrid + vm tg_stride) share each frequency's cell,
// basis or taps and factor (MULTI: the instance for V > 1).
template <bool MULTI>
__global__ void k_asy_adj_spread(const ProbParams* __restrict__ probs, const AsyBlock* __restrict__ blks,
                                 const Tile* __restrict__ tiles, Tables tab,
                                 const double* __restrict__ w_s, const double* __restrict__ g_s,
                                 int64_t g_stride, int V, double2* __restrict__ tgrid, int64_t tg_stride)
{
    extern __shared__ float4 sma[];
    __shared__ int use_mom;
    const Tile t = tiles[blockIdx.x];
    const AsyBlock B = blks[t.blk];
    const ProbParams& P = probs[B.prob];
    const int Q = P.Q;
    const int w = tab.w, deg = tab.deg, nt = blockDim.x, tid = threadIdx.x;
    const int mask = B.nf2 - 1;
    const Accum tg = Accum{(double*)tgrid, P.fxs}.at(2 * B.q_off);
    const int cnt = t.count;
    if (cnt <= 0) return;
    if (tid == 0) {
        long long Om, Sw, svw;
        const int tfirst = interp_cell_sv(B, w, w_s[t.start], &Om, &Sw, &svw);
        const int nbins = interp_cell_sv(B, w, w_s[t.start + cnt - 1], &Om, &Sw, &svw) - tfirst + 1;
        use_mom = nbins <= kMaxTileBins && cnt >= kMomMinPerBin * nbins;
    }
    __syncthreads();
    if (use_mom) {
        AdjFactor F{};
        int64_t kt = 0;
        spread_moments(Q, P.qs, t, tab,
            [&](int64_t k, df* v, float2* xq) {
                const int t0 = adj_spread_factor(B, P, tab, w_s[k], v, &F);
                kt = k;
                adj_values(P, F, g_s[k], xq);
                return t0;
            },
            [&](int vm, float2* xq) { adj_values(P, F, g_s[vm * g_stride + kt], xq); }, MULTI ? V : 1,
            2 * tg_stride,
            [&](int c) -> int64_t { return c & mask; }, tg, (float2*)sma);
        return;
    }
    const int ncoef = w * (deg + 1);
    float4* uval = sma;                                 // [nt][Q]
    float2* coef = (float2*)(uval + nt * Q);            // [w][deg+1]
    float2* taps = coef + ncoef;                        // [nt][w]
    int* t0s = (int*)(taps + nt * w);                   // [nt]
    for (int i = tid; i < ncoef; i += nt) coef[i] = tab.es2[i];
    __syncthreads();
    AdjFactor F{};
    const int64_t k = t.start + tid;
    if (tid < cnt) {
        df vdf;
        const int t0 = adj_spread_factor(B, P, tab, w_s[k], &vdf, &F);
        adj_values(P, F, g_s[k], (float2*)(uval + tid * Q));
        for (int i = 0; i < w; ++i) {
            const df tp = horner_comp(coef + i * (deg + 1), deg, vdf.h, vdf.l, tab.deg_comp);
            taps[tid * w + i] = make_float2(tp.h, tp.l);
        }
        t0s[tid] = t0;
    }
    __syncthreads();
    const int tfirst = t0s[0];
    const int span = t0s[cnt - 1] - tfirst + w;
    const bool dense = span <= 2 * w;
    for (int vm = 0; vm < (MULTI ? V : 1); ++vm) {
    if (MULTI && vm > 0) {
        __syncthreads();   // the previous member's reads of uval are done
        if (tid < cnt) adj_values(P, F, g_s[vm * g_stride + k], (float2*)(uval + tid * Q));
        __syncthreads();
    }
    const Accum tgv = tg.at(2 * vm * tg_stride);
    for (int item = tid; item < span * Q; item += nt) {
        const int c = item / Q, q = item - c * Q;
        const int cell = tfirst + c;
        int p_lo = 0, p_hi = cnt;
        if (!dense) {
            int lo = 0, hi = cnt;
            const int key = cell - w + 1;
            while (lo < hi) { int mid = (lo + hi) >> 1; if (t0s[mid] < key) lo = mid + 1; else hi = mid; }
            p_lo = lo;
            hi = cnt;
            while (lo < hi) { int mid = (lo + hi) >> 1; if (t0s[mid] <= cell) lo = mid + 1; else hi = mid; }
            p_hi = lo;
        }
        acc2 ar{0.f, 0.f}, ai{0.f, 0.f};
        bool any = false;
        for (int p = p_lo; p < p_hi; ++p) {
            const int i = cell - t0s[p];
            if (i >= 0 && i < w) {
                const float2 k2 = taps[p * w + i];
                const float4 uv = uval[p * Q + q];
                const df kk{k2.x, k2.y};
                acc_fma(ar, kk, df{uv.x, uv.y});
                acc_fma(ai, kk, df{uv.z, uv.w});
                any = true;
            }
        }
        if (any) {
            const int64_t o = (int64_t)(cell & mask) * Q + q;
            tgv.add(2 * o, acc_value(ar));
            tgv.add(2 * o + 1, acc_value(ai));
        }
    }
    }
}

// Points of a tile: interpolate the corrected modes b' (split, at b_off) with
// the spreading kernel, apply D_in and sum the Hankel terms into c; the
// transpose of the spreading, computed like k_asy_interp (one thread per
// point, in passes of blockDim points).  A point at cell l0 reads the modes
// l0 + i, i < w (zero outside the 2 N1 + 1 modes).  Dense passes (many points
// per cell) form the per-bin sums H[d][q'] once per bin and each point sums
// P_q = sum_d T_d(v) H[d][q]; sparse passes evaluate the w taps of each point.
// Members: V real components (modes bgrid + vm bg_stride, sums into c_s + vm
// c_stride) share each point's cell, basis or taps and factors (MULTI: the
// instance for V > 1, which also forms the phase before the member loop).
template <bool MULTI>
__global__ void __launch_bounds__(kAdjInterpThreads) k_asy_adj_interp(
    const ProbParams* __restrict__ probs, const AsyBlock* __restrict__ blks, const Tile* __restrict__ tiles,
    Tables tab, const double* __restrict__ r_s, const float4* __restrict__ bgrid, int64_t bg_stride, int V,
    double* __restrict__ c_s, int64_t c_stride)
{
    extern __shared__ float4 win[];          // [kWinCells][Q] modes of this pass
    const Tile t = tiles[blockIdx.x];
    const AsyBlock B = blks[t.blk];
    const ProbParams& P = probs[B.prob];
    const int w = tab.w, deg = tab.deg, nb = tab.nb, dci = tab.dci;
    const int Q = P.Q, Q2 = 2 * Q, qs = P.qs;
    const int us = (deg + 1 > w ? deg + 1 : w) | 1;
    const int hs = nb * Q2 + 2;
    float2* coef2 = (float2*)(win + kWinCells * Q);              // [w][deg + 1] taps, or [w][nb] Chebyshev
    float2* H = coef2 + ((w * (deg + 1) + 1) & ~1);              // [bins][hs], 16-byte aligned
    float2* U = H + kAdjInterpHBytes / sizeof(float2);              // [threads][us]
    int* l0s = (int*)(U + kAdjInterpThreads * us);              // [threads]
    const int nf1 = 2 * B.N1 + 1;
    const int maxbins = kAdjInterpHBytes / (int)(sizeof(float2) * hs);
    for (int base = 0; base < t.count; base += blockDim.x) {
        const int cnt = t.count - base < (int)blockDim.x ? t.count - base : (int)blockDim.x;
        const bool valid = (int)threadIdx.x < cnt;
        const int64_t j = t.start + base + (valid ? threadIdx.x : 0);
        const double rj = r_s[j];
        long long X;
        df vd;
        const int l0 = spread_cell_fx(B, w, rj, &X, &vd);
        if (valid) l0s[threadIdx.x] = l0;
        __syncthreads();
        // the tile's points are sorted, so their cells form one window
        const int wstart = l0s[0];
        const int nbins = l0s[cnt - 1] - wstart + 1;
        const int wlen = nbins - 1 + w;
        const bool staged = wlen <= kWinCells;
        const bool mom = staged && nbins <= maxbins && cnt >= kMomMinPerBin * nbins;
        if (mom) {
            for (int i = threadIdx.x; i < w * nb; i += blockDim.x) {
                const int r = i / nb, d = i - r * nb;
                coef2[i] = tab.ch2[r * (deg + 1) + d];
            }
        } else {
            for (int i = threadIdx.x; i < w * (deg + 1); i += blockDim.x) coef2[i] = tab.es2[i];
        }
        __syncthreads();
        // this point's basis or taps, (r/rho)^(-1) and the phase e^{i w_c x}
        float2* u = U + threadIdx.x * us;
        df rat{0.f, 0.f}, sn{0.f, 0.f}, cs{0.f, 0.f};
        if (valid) {
            const float vh = vd.h, vl = vd.l;
            if (mom) {
                cheb_basis_row(u, vh, vl, dci, nb);
            } else {
                for (int i = 0; i < w; ++i) {
                    const df tp = horner_comp(coef2 + i * (deg + 1), deg, vh, vl, tab.deg_comp);
                    u[i] = make_float2(tp.h, tp.l);
                }
            }
            rat = df_mul(df_from(B.rho), df_recip(df_from(rj)));   // (r/rho)^(-1) <= 1
            if (MULTI) df_sincos_turns_tab(mul128_bits(X, B.KW, B.sW), tab.tw2, &sn, &cs);
        }
        for (int vm = 0; vm < (MULTI ? V : 1); ++vm) {
            const float4* gb = bgrid + vm * bg_stride + B.b_off;
            if (vm > 0) __syncthreads();   // the previous member's reads of the window and H are done
            if (staged)
                for (int idx = threadIdx.x; idx < wlen * Q; idx += blockDim.x) {
                    const int cc = idx / Q;
                    const int li = wstart + cc + B.N1;
                    win[idx] = (li >= 0 && li < nf1) ? gb[(int64_t)li * Q + (idx - cc * Q)]
                                                     : make_float4(0.f, 0.f, 0.f, 0.f);
                }
            __syncthreads();
            if (mom) {
                bin_sums_build(win, coef2, H, nbins, w, nb, dci, Q, qs, P.dcp);
                __syncthreads();
            }
            if (!valid) continue;
            // T = sum_q (r/rho)^(-q) P_q, P_q = sum_i psi_i(v) b'_{l0 + i, q}
            acc2 tr{0.f, 0.f}, ti{0.f, 0.f};
            df mq{1.f, 0.f};
            auto combine = [&](int, df prd, df pid) {
                acc_fma(tr, mq, prd);
                acc_fma(ti, mq, pid);
                mq = df_mul(mq, rat);
            };
            if (mom)
                bin_sums_eval(H + (l0 - wstart) * hs, u, nb, dci, Q, qs, P.dcp, combine);
            else
                tap_sums_eval(u, w, Q, qs, [&](int i, int q) {
                    const int li = l0 + i + B.N1;
                    if (staged) return win[(l0 + i - wstart) * Q + q];
                    return (li >= 0 && li < nf1) ? gb[(int64_t)li * Q + q] : make_float4(0.f, 0.f, 0.f, 0.f);
                }, combine);
            // c_j += Re( e^{i w_c x} (r/rho)^(-1/2) T )
            if (!MULTI) df_sincos_turns_tab(mul128_bits(X, B.KW, B.sW), tab.tw2, &sn, &cs);
            const df tre = fast_two_sum(tr.s, tr.c), tim = fast_two_sum(ti.s, ti.c);
            const df re = df_add(df_mul(cs, tre), df_negate(df_mul(sn, tim)));
            Accum{c_s + vm * c_stride, P.fxs}.add(j, df_to(df_mul(df_sqrt(rat), re)));
        }
        __syncthreads();   // l0s, the window and H are rewritten by the next pass
    }
}

// ------------------------------------------------------ mixed precision (FP32)
__device__ __forceinline__ float horner_f32(const float2* __restrict__ c, int deg, float v)
{
    float acc = c[deg].x;
    for (int k = deg - 1; k >= 0; --k) acc = fmaf(acc, v, c[k].x);
    return acc;
}

// Row stride (floats) for 16-byte loads by eight rows: = 4 mod 8.
__host__ __device__ __forceinline__ int f32_stride4(int n)
{
    const int r = (n + 3) & ~3;
    return (r & 4) ? r : r + 4;
}

// FP32 spreading, dense tile: the moment form of spread_moments in single
// precision (each of the 8 partial sums of a moment covers at most
// ceil(tile / 8) points).  The bins go in groups of up to kF32GroupBins: the
// moment items of all the group's bins share one pass (and one barrier), and
// each cell of the group's window then sums A[c - b] M_b over the group's bins
// b that reach it (each bin's sum in FP32 as before, the bins' sums combined
// with compensated additions) and adds it with one FP64 atomic.  Members
// (MULTI) as in spread_fold.
constexpr int kF32GroupBytes = 16384;

__host__ __device__ __forceinline__ int f32_group_bins(int dpad, int Q2)
{
    int g = kF32GroupBytes / (int)(sizeof(float) * dpad * Q2);
    if (g < 1) g = 1;
    return g < kMaxTileBins ? g : kMaxTileBins;
}

template <bool MULTI>
__device__ void spread_moments_f32(const AsyBlock& B, int Q, const Tile& t, const Tables& tab,
                                   const double* __restrict__ r_s, const float2* __restrict__ r2,
                                   const float2* __restrict__ c2, int64_t c_stride, int V, int64_t moff,
                                   Accum gb, float* sm)
{
    const int nt = blockDim.x, tid = threadIdx.x, cnt = t.count;
    const int w = tab.w, nb = tab.nb;
    const int Q2 = 2 * Q;
    const int ndp = (nb + 1) >> 1, dpad = 2 * ndp, nq = Q2 >> 2;
    const int su = mom_stride(nb), sx = f32_stride4(Q2);
    const int GB = f32_group_bins(dpad, Q2);
    float* U = sm;                               // [nt][su]
    float* X = U + nt * su;                      // [nt][sx]
    float* Mb = X + nt * sx;                     // [GB][dpad][Q2]
    float* Ach = Mb + GB * dpad * Q2;            // [w][dpad]
    int* l0s = (int*)(Ach + w * dpad);           // [nt]
    __shared__ int bstart[kMaxTileBins + 3];
    for (int i = tid; i < w * dpad; i += nt) {
        const int r = i / dpad, d = i - r * dpad;
        Ach[i] = d < nb ? tab.ch2[r * (tab.deg + 1) + d].x : 0.f;
    }
    const int64_t j = t.start + tid;
    float yr = 0.f, yi = 0.f, ratio = 0.f;   // this point's weight without c_j, and its ratio
    if (tid < cnt) {
        long long Xp;
        df vdf;
        l0s[tid] = spread_cell_fx(B, tab.w, r_s[j], &Xp, &vdf);
        const float v = vdf.h;
        float* u = U + tid * su;
        float tm = 1.f, tc = v;
        u[0] = 1.f;
        u[1] = v;
        for (int d = 2; d < nb; ++d) {
            const float tn = fmaf(2.f * v, tc, -tm);
            u[d] = tn;
            tm = tc;
            tc = tn;
        }
        for (int d = nb; d < su; ++d) u[d] = 0.f;
        float sn, cs;
        f32_sincos_turns(mul128_bits(Xp, B.KW, B.sW), &sn, &cs);
        ratio = B.rho_h / r2[j].x;
        const float w0 = sqrtf(ratio);
        yr = w0 * cs;
        yi = w0 * sn;
    }
    auto put = [&](int vm) {
        const float cv = c2[vm * c_stride + j].x;
        float wr = cv * yr, wi = cv * yi;
        float* xq = X + tid * sx;
        for (int q = 0; q < Q; ++q) {
            xq[2 * q] = wr;
            xq[2 * q + 1] = wi;
            wr *= ratio;
            wi *= ratio;
        }
    };
    if (tid < cnt) put(0);
    __syncthreads();
    const int lfirst = l0s[0];
    const int nbins = l0s[cnt - 1] - lfirst + 1;
    for (int b = tid; b <= nbins; b += nt) {
        const int key = lfirst + b;
        int lo = 0, hi = cnt;
        while (lo < hi) { const int mid = (lo + hi) >> 1; if (l0s[mid] < key) lo = mid + 1; else hi = mid; }
        bstart[b] = lo;
    }
    __syncthreads();
    const int nf1 = 2 * B.N1 + 1;
    const int nitems = ndp * nq * kSpreadSub;
    for (int vm = 0; vm < (MULTI ? V : 1); ++vm) {
    if (MULTI && vm > 0) {
        if (tid < cnt) put(vm);
        __syncthreads();
    }
    const Accum gv = gb.at(vm * moff);
    for (int g0 = 0; g0 < nbins; g0 += GB) {
        const int gn = nbins - g0 < GB ? nbins - g0 : GB;
        // (a) the moments of the group's bins: items (bin, degree pair, value quad, sub-range)
        const int gitems = gn * nitems;
        const int gitems_pad = (gitems + 31) & ~31;
        for (int it = tid; it < gitems_pad; it += nt) {
            const bool live = it < gitems;
            const int sub = it & (kSpreadSub - 1);
            const int ob = live ? it / kSpreadSub : 0;
            const int bb = ob / (ndp * nq), o = ob - bb * (ndp * nq);
            const int dp = o / nq, qq = o - dp * nq;
            const int p0 = bstart[g0 + bb], p1 = bstart[g0 + bb + 1];
            float A[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
            if (live) {
                for (int p = p0 + sub; p < p1; p += kSpreadSub) {
                    const float2 uu = *(const float2*)(U + p * su + 2 * dp);
                    const float4 xx = *(const float4*)(X + p * sx + 4 * qq);
                    const float xs[4] = {xx.x, xx.y, xx.z, xx.w};
#pragma unroll
                    for (int f = 0; f < 4; ++f) {
                        A[0][f] = fmaf(uu.x, xs[f], A[0][f]);
                        A[1][f] = fmaf(uu.y, xs[f], A[1][f]);
                    }
                }
            }
            float* mb = Mb + bb * dpad * Q2;
#pragma unroll
            for (int e = 0; e < 2; ++e)
#pragma unroll
                for (int f = 0; f < 4; ++f) {
                    float av = A[e][f];
#pragma unroll
                    for (int off = kSpreadSub >> 1; off > 0; off >>= 1) av += __shfl_xor_sync(0xffffffffu, av, off);
                    if (live && sub == 0) mb[(2 * dp + e) * Q2 + 4 * qq + f] = av;
                }
        }
        __syncthreads();
        // (c) cell lfirst + g0 + c: sum over the group's bins b with 0 <= c - b < w
        const int ncell = gn + w - 1;
        for (int o = tid; o < ncell * Q2; o += nt) {
            const int c = o / Q2, qv = o - c * Q2;
            const int idx = lfirst + g0 + c + B.N1;
            if (idx < 0 || idx >= nf1) continue;
            const int b_lo = c - w + 1 > 0 ? c - w + 1 : 0;
            const int b_hi = c < gn - 1 ? c : gn - 1;
            float ss = 0.f, sc = 0.f;
            for (int bb = b_lo; bb <= b_hi; ++bb) {
                const float* ar = Ach + (c - bb) * dpad;
                const float* mb = Mb + bb * dpad * Q2 + qv;
                float part = 0.f;
                for (int d = 0; d < nb; ++d) part = fmaf(ar[d], mb[d * Q2], part);
                float t, e;
                two_sum(ss, part, t, e);
                ss = t;
                sc += e;
            }
            const float sacc = ss + sc;
            if (sacc != 0.f) gv.add(2 * ((int64_t)idx * Q + (qv >> 1)) + (qv & 1), (double)ss + (double)sc);
        }
        __syncthreads();
    }
    }
}

__host__ __device__ __forceinline__ size_t spread_moments_f32_smem(int nt, int Q, int w, int nb)
{
    const int dpad = 2 * ((nb + 1) >> 1);
    return sizeof(float) * ((size_t)nt * mom_stride(nb) + (size_t)nt * f32_stride4(2 * Q) +
                            (size_t)f32_group_bins(dpad, 2 * Q) * dpad * 2 * Q + (size_t)w * dpad) +
           sizeof(int) * (size_t)nt;
}

// FP32 spreading, sparse tile: taps per point, one thread per (cell, q).
// Members (MULTI) as in spread_taps.
template <bool MULTI>
__device__ void spread_taps_f32(const AsyBlock& B, int Q, const Tile& t, const Tables& tab,
                                const double* __restrict__ r_s, const float2* __restrict__ r2,
                                const float2* __restrict__ c2, int64_t c_stride, int V, int64_t moff,
                                Accum gb, float2* smf)
{
    const int w = tab.w, deg = tab.deg, nt = blockDim.x, tid = threadIdx.x;
    const int ncoef = w * (deg + 1);
    float2* aval = smf;                              // [nt][Q]
    float2* coef = aval + nt * Q;                    // [w][deg+1]
    float* taps = (float*)(coef + ncoef);            // [nt][w]
    int* l0s = (int*)(taps + nt * w);                // [nt]
    for (int i = tid; i < ncoef; i += nt) coef[i] = tab.es2[i];
    __syncthreads();
    const int cnt = t.count;
    const int64_t j = t.start + tid;
    float yr = 0.f, yi = 0.f, ratio = 0.f;   // this point's weight without c_j, and its ratio
    if (tid < cnt) {
        long long Xp;
        df vdf;
        l0s[tid] = spread_cell_fx(B, tab.w, r_s[j], &Xp, &vdf);
        const float v = vdf.h;
        for (int i = 0; i < w; ++i) taps[tid * w + i] = horner_f32(coef + i * (deg + 1), deg, v);
        float sn, cs;
        f32_sincos_turns(mul128_bits(Xp, B.KW, B.sW), &sn, &cs);
        ratio = B.rho_h / r2[j].x;
        const float w0 = sqrtf(ratio);
        yr = w0 * cs;
        yi = w0 * sn;
    }
    auto put = [&](int vm) {
        const float cv = c2[vm * c_stride + j].x;
        float wr = cv * yr, wi = cv * yi;
        for (int q = 0; q < Q; ++q) {
            aval[tid * Q + q] = make_float2(wr, wi);
            wr *= ratio;
            wi *= ratio;
        }
    };
    if (tid < cnt) put(0);
    __syncthreads();
    const int lfirst = l0s[0];
    const int span = l0s[cnt - 1] - lfirst + w;
    const int nf1 = 2 * B.N1 + 1;
    const bool dense = span <= 2 * w;
    for (int vm = 0; vm < (MULTI ? V : 1); ++vm) {
    if (MULTI && vm > 0) {
        __syncthreads();   // the previous member's reads of aval are done
        if (tid < cnt) put(vm);
        __syncthreads();
    }
    const Accum gv = gb.at(vm * moff);
    for (int item = tid; item < span * Q; item += nt) {
        const int c = item / Q, q = item - c * Q;
        const int cell = lfirst + c;
        int p_lo = 0, p_hi = cnt;
        if (!dense) {
            int lo = 0, hi = cnt;
            const int key = cell - w + 1;
            while (lo < hi) { int mid = (lo + hi) >> 1; if (l0s[mid] < key) lo = mid + 1; else hi = mid; }
            p_lo = lo;
            hi = cnt;
            while (lo < hi) { int mid = (lo + hi) >> 1; if (l0s[mid] <= cell) lo = mid + 1; else hi = mid; }
            p_hi = lo;
        }
        float sr = 0.f, si = 0.f;
        for (int p = p_lo; p < p_hi; ++p) {
            const int i = cell - l0s[p];
            if (i >= 0 && i < w) {
                const float k = taps[p * w + i];
                const float2 av = aval[p * Q + q];
                sr = fmaf(k, av.x, sr);
                si = fmaf(k, av.y, si);
            }
        }
        const int idx = cell + B.N1;
        if (idx >= 0 && idx < nf1 && (sr != 0.f || si != 0.f)) {
            gv.add(2 * ((int64_t)idx * Q + q), (double)sr);
            gv.add(2 * ((int64_t)idx * Q + q) + 1, (double)si);
        }
    }
    }
}

// FP32 spreading (coordinates and phase reduction in FP64).
// Mixed precision: the plain moment path for every dense tile (mode != 0).
// Members as in k_asy_spread.
template <bool MULTI>
__global__ void k_asy_spread_f32(const ProbParams* __restrict__ probs, const AsyBlock* __restrict__ blks,
                                 const Tile* __restrict__ tiles, const int32_t* __restrict__ modes, Tables tab,
                                 const double* __restrict__ r_s, const float2* __restrict__ r2,
                                 const float2* __restrict__ c2, int64_t c_stride, int V,
                                 double2* __restrict__ grid_b, int64_t gb_stride)
{
    extern __shared__ float2 smf[];
    const Tile t = tiles[blockIdx.x];
    if (t.count <= 0) return;
    const AsyBlock B = blks[t.blk];
    const int Q = probs[B.prob].Q;
    const Accum gb = Accum{(double*)grid_b, probs[B.prob].fxs}.at(2 * B.b_off);
    if (modes[blockIdx.x] & 3)
        spread_moments_f32<MULTI>(B, Q, t, tab, r_s, r2, c2, c_stride, V, 2 * gb_stride, gb, (float*)smf);
    else
        spread_taps_f32<MULTI>(B, Q, t, tab, r_s, r2, c2, c_stride, V, 2 * gb_stride, gb, smf);
}

// Shared memory (bytes) of k_asy_interp_f32 for 2M = qmax.
__host__ __device__ __forceinline__ size_t interp_f32_smem(int qmax, int w, int deg, int threads)
{
    const int us = (deg + 1 > w ? deg + 1 : w) | 1;
    return sizeof(float4) * (size_t)kWinCells * qmax + sizeof(float2) * (size_t)((w * (deg + 1) + 1) & ~1) +
           (size_t)kInterpHBytesPerThread * threads + sizeof(float) * (size_t)threads * us + sizeof(int) * threads;
}

// FP32 interpolation and Hankel combination (coordinates and phase
// reduction in FP64); dense tiles by per-bin Chebyshev sums as in
// k_asy_interp, sparse tiles by taps.  Members as in k_asy_interp.
__global__ void __launch_bounds__(kInterpTileThreads, 4) k_asy_interp_f32(
    const ProbParams* __restrict__ probs, const AsyBlock* __restrict__ blks, const Tile* __restrict__ tiles,
    Tables tab, const double* __restrict__ w_s, const float2* __restrict__ w2, const float4* __restrict__ grid_q,
    int64_t gq_stride, int V, double* __restrict__ g_s, int64_t g_stride)
{
    extern __shared__ float4 winf[];
    const Tile t = tiles[blockIdx.x];
    const AsyBlock B = blks[t.blk];
    const ProbParams& P = probs[B.prob];
    const int w = tab.w, deg = tab.deg, nb = tab.nb;
    const int Q = P.Q, Q2 = 2 * Q;
    const int us = (deg + 1 > w ? deg + 1 : w) | 1;
    const int hs = nb * Q2 + 2;                                  // bin stride of H (floats, even)
    float2* coef2 = (float2*)(winf + kWinCells * Q);
    float* H = (float*)(coef2 + ((w * (deg + 1) + 1) & ~1));     // [bins][hs]
    const int hbytes = kInterpHBytesPerThread * (int)blockDim.x;
    float* U = H + hbytes / sizeof(float);                       // [threads][us]
    int* t0s = (int*)(U + blockDim.x * us);
    const bool valid = (int)threadIdx.x < t.count;
    const int64_t k = t.start + (valid ? threadIdx.x : 0);
    long long Om, Sw, svw;
    const int t0 = interp_cell_sv(B, tab.w, w_s[k], &Om, &Sw, &svw);
    const float v = df_from_sv(svw).h;
    if (valid) t0s[threadIdx.x] = t0;
    __syncthreads();
    const int wstart = t0s[0];
    const int nbins = t0s[t.count - 1] - wstart + 1;
    const int wlen = nbins - 1 + w;
    const int mask = B.nf2 - 1;
    const bool staged = wlen <= kWinCells;
    const int maxbins = hbytes / (int)(sizeof(float) * hs);
    const bool mom = staged && nbins <= maxbins && t.count >= kMomMinPerBin * nbins;
    if (mom) {
        for (int i = threadIdx.x; i < w * nb; i += blockDim.x) {
            const int r = i / nb, d = i - r * nb;
            coef2[i] = tab.ch2[r * (deg + 1) + d];
        }
    } else {
        for (int i = threadIdx.x; i < w * (deg + 1); i += blockDim.x) coef2[i] = tab.es2[i];
    }
    __syncthreads();
    // this thread's basis or taps, and the member-independent factors of its output
    float* u = U + threadIdx.x * us;
    float m1 = 0.f, outs = 0.f, sn = 0.f, cs = 0.f;
    if (valid) {
        if (mom) {
            float tm = 1.f, tc = v;
            u[0] = 1.f;
            u[1] = v;
            for (int d = 2; d < nb; ++d) {
                const float tn = fmaf(2.f * v, tc, -tm);
                u[d] = tn;
                tm = tc;
                tc = tn;
            }
        } else {
            for (int i = 0; i < w; ++i) u[i] = horner_f32(coef2 + i * (deg + 1), deg, v);
        }
        m1 = 1.f / (w2[k].x * B.rho_h);
        f32_sincos_turns(mul128_bits(Om, B.KRc, B.sR), &sn, &cs);
        // psi^(alpha s) in FP32 from the table's high parts
        const float sf = df_from_i64(Sw < 0 ? -Sw : Sw).h * ldexpf(1.f, -B.fw);
        const float xi = B.alpha_h * sf * tab.ph_scale2.x;
        int piece = (int)xi;
        if (piece > tab.ph_pieces - 1) piece = tab.ph_pieces - 1;
        const float ph = horner_f32(tab.ph2 + piece * (tab.ph_deg + 1), tab.ph_deg, 2.f * (xi - (float)piece) - 1.f);
        outs = tab.ic2.x * sqrtf(m1) / ph;
        if (P.sgn < 0) outs = -outs;
    }
    const float* Hb = H + (t0 - wstart) * hs;
    const float cph = P.cphi2.x, sph = P.sphi2.x;
    for (int vm = 0; vm < V; ++vm) {
        const float4* gq = grid_q + vm * gq_stride + B.q_off;
        if (vm > 0) __syncthreads();   // the previous member's reads of the window and H are done
        if (staged)
            for (int idx = threadIdx.x; idx < wlen * Q; idx += blockDim.x) {
                const int cc = idx / Q;
                winf[idx] = gq[(int64_t)((wstart + cc) & mask) * Q + (idx - cc * Q)];
            }
        __syncthreads();
        if (mom) {
            for (int o = threadIdx.x; o < nbins * nb * Q2; o += blockDim.x) {
                const int b = o / (nb * Q2), rem = o - b * nb * Q2;
                const int d = rem / Q2, qv = rem - d * Q2;
                const int q = qv >> 1, im = qv & 1;
                float acc = 0.f;
                for (int i = 0; i < w; ++i) {
                    const float4 gv = winf[(b + i) * Q + q];
                    acc = fmaf(coef2[i * nb + d].x, im ? gv.z : gv.x, acc);
                }
                H[b * hs + rem] = acc;
            }
            __syncthreads();
        }
        if (!valid) continue;
        float tr = 0.f, ti = 0.f, mq = 1.f;
        for (int q = 0; q < Q; ++q) {
            float pr = 0.f, pi = 0.f;
            if (mom) {
                for (int d = 0; d < nb; ++d) {
                    const float2 hv = *(const float2*)(Hb + d * Q2 + 2 * q);
                    pr = fmaf(u[d], hv.x, pr);
                    pi = fmaf(u[d], hv.y, pi);
                }
            } else {
                for (int i = 0; i < w; ++i) {
                    const float4 gv = staged ? winf[(t0 + i - wstart) * Q + q]
                                             : gq[(int64_t)((t0 + i) & mask) * Q + q];
                    pr = fmaf(u[i], gv.x, pr);
                    pi = fmaf(u[i], gv.z, pi);
                }
            }
            const float cq = P.a2[q].x * mq;
            switch (q & 3) {
                case 0: tr = fmaf(cq, pr, tr); ti = fmaf(cq, pi, ti); break;
                case 1: tr = fmaf(-cq, pi, tr); ti = fmaf(cq, pr, ti); break;
                case 2: tr = fmaf(-cq, pr, tr); ti = fmaf(-cq, pi, ti); break;
                default: tr = fmaf(cq, pi, tr); ti = fmaf(-cq, pr, ti); break;
            }
            mq *= m1 * P.z2.x;
        }
        const float ur = cph * tr - sph * ti, ui = sph * tr + cph * ti;
        const float re = cs * ur - sn * ui;
        Accum{g_s + vm * g_stride, P.fxs}.add(k, (double)(outs * re));
    }
}

}  // namespace

cudaError_t launch_asy_adj_spread(const ProbParams* probs, const AsyBlock* blks, const Tile* tiles,
                                  int ntiles, int qmax, int nt, Tables tab, const double* w_s, const double* g_s,
                                  int64_t g_stride, int members, double2* tgrid, int64_t tg_stride,
                                  cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    if (nt < 32 || nt > kInterpTileThreads || (nt & 31)) return cudaErrorInvalidValue;
    size_t smem = sizeof(float4) * (size_t)nt * qmax + sizeof(float2) * (size_t)tab.w * (tab.deg + 1) +
                  sizeof(float2) * (size_t)nt * tab.w + sizeof(int) * (size_t)nt;
    const size_t smem_mom = spread_moments_smem(nt, qmax, tab.w, tab.nb, tab.dcs);
    if (smem_mom > smem) smem = smem_mom;
    if (members < 1) return cudaErrorInvalidValue;
    auto kern = members > 1 ? k_asy_adj_spread<true> : k_asy_adj_spread<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<ntiles, nt, smem, s>>>(probs, blks, tiles, tab, w_s, g_s, g_stride, members, tgrid, tg_stride);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_asy_adj_interp(const ProbParams* probs, const AsyBlock* blks, const Tile* tiles,
                                  int ntiles, int qmax, Tables tab, const double* r_s, const float4* bgrid,
                                  int64_t bg_stride, int members, double* c_s, int64_t c_stride, cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    const size_t smem = interp_smem(qmax, tab.w, tab.deg, kAdjInterpThreads, kAdjInterpHBytes);
    if (members < 1) return cudaErrorInvalidValue;
    auto kern = members > 1 ? k_asy_adj_interp<true> : k_asy_adj_interp<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<ntiles, kAdjInterpThreads, smem, s>>>(probs, blks, tiles, tab, r_s, bgrid, bg_stride, members, c_s,
                                                 c_stride);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_asy_spread_f32(const ProbParams* probs, const AsyBlock* blks, const Tile* tiles,
                                  const int32_t* modes, int ntiles, int qmax, int nt, Tables tab,
                                  const double* r_s, const float2* r2, const float2* c2, int64_t c_stride,
                                  int members, double2* grid_b, int64_t gb_stride, cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    size_t smem = sizeof(float2) * (size_t)nt * qmax + sizeof(float2) * (size_t)tab.w * (tab.deg + 1) +
                  sizeof(float) * (size_t)nt * tab.w + sizeof(int) * (size_t)nt;
    const size_t smem_mom = spread_moments_f32_smem(nt, qmax, tab.w, tab.nb);
    if (smem_mom > smem) smem = smem_mom;
    if (members < 1) return cudaErrorInvalidValue;
    auto kern = members > 1 ? k_asy_spread_f32<true> : k_asy_spread_f32<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<ntiles, nt, smem, s>>>(probs, blks, tiles, modes, tab, r_s, r2, c2, c_stride, members, grid_b,
                                  gb_stride);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_asy_interp_f32(const ProbParams* probs, const AsyBlock* blks, const Tile* tiles,
                                  int ntiles, int qmax, int nt, Tables tab, const double* w_s, const float2* w2,
                                  const float4* grid_q, int64_t gq_stride, int members, double* g_s,
                                  int64_t g_stride, cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    if (nt < 32 || nt > kInterpTileThreads || (nt & 31)) return cudaErrorInvalidValue;
    const size_t smem = interp_f32_smem(qmax, tab.w, tab.deg, nt);
    cudaError_t e = cudaFuncSetAttribute(k_asy_interp_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (members < 1) return cudaErrorInvalidValue;
    k_asy_interp_f32<<<ntiles, nt, smem, s>>>(probs, blks, tiles, tab, w_s, w2, grid_q, gq_stride, members, g_s,
                                              g_stride);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_spread_modes(const ProbParams* probs, const AsyBlock* blks, const Tile* tiles, int ntiles,
                                Tables tab, const double* r_s, int32_t* modes, cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    const int nb = (ntiles + 255) / 256, cap = device_sm_count() * 16;
    k_spread_modes<<<nb < cap ? nb : cap, 256, 0, s>>>(probs, blks, tiles, ntiles, tab, r_s, modes);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_asy_spread(const ProbParams* probs, const AsyBlock* blks, const Tile* tiles,
                              const int32_t* modes, int ntiles, int qmax, int nt, Tables tab, const double* r_s,
                              const float2* r2, const float2* c2, int64_t c_stride, int members,
                              double2* grid_b, int64_t gb_stride, int det, cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    size_t smem = sizeof(float4) * (size_t)nt * qmax + sizeof(float2) * (size_t)tab.w * (tab.deg + 1) +
                  sizeof(float2) * (size_t)nt * tab.w + sizeof(int) * (size_t)nt;
    const size_t smem_mom = spread_moments_smem(nt, qmax, tab.w, tab.nb, tab.dcs);
    if (smem_mom > smem) smem = smem_mom;
    const size_t smem_fold = spread_fold_smem(nt, qmax, tab.w, tab.nb, tab.dcs);
    if (smem_fold > smem) smem = smem_fold;
    auto kern = det ? k_asy_spread<true, false>
                    : (members > 1 ? k_asy_spread<false, true> : k_asy_spread<false, false>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (members < 1 || (det && members != 1)) return cudaErrorInvalidValue;
    kern<<<ntiles, nt, smem, s>>>(probs, blks, tiles, modes, tab, r_s, r2, c2, c_stride, members, grid_b,
                                  gb_stride);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_asy_fft_small(const ProbParams* probs, const AsyBlock* blks, const Tile* items,
                                 int nitems, int max_nf2, Tables tab, const double2* src,
                                 float4* dst, cudaStream_t s, bool adj, bool lowp, int members,
                                 int64_t src_stride, int64_t dst_stride)
{
    if (nitems <= 0) return cudaSuccess;
    if (members < 1 || members > 65535) return cudaErrorInvalidValue;
    size_t smem = (lowp ? sizeof(float2) : sizeof(float4)) * (size_t)max_nf2;
    auto kern = adj ? (lowp ? k_asy_fft_small<true, true> : k_asy_fft_small<true, false>)
                    : (lowp ? k_asy_fft_small<false, true> : k_asy_fft_small<false, false>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int nt = max_nf2 / 2;
    if (nt > 256) nt = 256;
    if (nt < 32) nt = 32;
    kern<<<dim3(nitems, members), nt, smem, s>>>(probs, blks, items, tab, src, dst, src_stride, dst_stride);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_asy_fft_block(const ProbParams* probs, const AsyBlock* blks, const Tile* items,
                                 int nitems, int max_pts, Tables tab, const double2* src, float4* dst,
                                 cudaStream_t s, bool adj, bool lowp, int members, int64_t src_stride,
                                 int64_t dst_stride)
{
    if (nitems <= 0) return cudaSuccess;
    if (members < 1 || members > 65535) return cudaErrorInvalidValue;
    if (max_pts < 1 || max_pts > kFftSmemMax) max_pts = kFftSmemMax;
    auto kern = adj ? (lowp ? k_asy_fft_block<true, true> : k_asy_fft_block<true, false>)
                    : (lowp ? k_asy_fft_block<false, true> : k_asy_fft_block<false, false>);
    // blocks of up to kFftSmallPts points in small CTAs (16 KiB, many per SM),
    // the larger ones in CTAs sized for the largest; each launch skips the
    // other size class at once
    constexpr int kFftSmallPts = 1024;
    const int ranges[2][2] = {{0, max_pts < kFftSmallPts ? max_pts : kFftSmallPts}, {kFftSmallPts, max_pts}};
    int launched = 0;
    for (int r = 0; r < 2; ++r) {
        const int lo = ranges[r][0], hi = ranges[r][1];
        if (hi <= lo) continue;
        const size_t smem = (lowp ? sizeof(float2) : sizeof(float4)) * (size_t)hi;
        int nt = ((hi / 2 + 31) / 32) * 32;
        if (r == 0 && nt > 128) nt = 128;
        if (nt > 256) nt = 256;
        if (nt < 32) nt = 32;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<dim3(nitems, members), nt, smem, s>>>(probs, blks, items, tab, src, dst, lo, hi, src_stride,
                                                     dst_stride);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        ++launched;
    }
    count_launches(launched);
    return cudaSuccess;
}

cudaError_t launch_asy_fft_large(const ProbParams* probs, const AsyBlock* blks, const Tile* items_a,
                                 int nitems_a, const Tile* items_b, int nitems_b, Tables tab,
                                 const double2* src, float4* tmp, float4* dst,
                                 cudaStream_t s, bool adj, bool lowp)
{
    if (nitems_a <= 0) return cudaSuccess;
    size_t smem = (lowp ? sizeof(float2) : sizeof(float4)) * (size_t)kFftLineBatch;
    auto ka = adj ? (lowp ? k_asy_fft_pass_a<true, true> : k_asy_fft_pass_a<true, false>)
                  : (lowp ? k_asy_fft_pass_a<false, true> : k_asy_fft_pass_a<false, false>);
    auto kb = adj ? (lowp ? k_asy_fft_pass_b<true, true> : k_asy_fft_pass_b<true, false>)
                  : (lowp ? k_asy_fft_pass_b<false, true> : k_asy_fft_pass_b<false, false>);
    cudaError_t e = cudaFuncSetAttribute(ka, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kb, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    ka<<<nitems_a, 256, smem, s>>>(probs, blks, items_a, tab, src, tmp);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    kb<<<nitems_b, 256, smem, s>>>(probs, blks, items_b, tab, tmp, dst);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_asy_interp(const ProbParams* probs, const AsyBlock* blks, const Tile* tiles,
                              int ntiles, int qmax, int nt, Tables tab, const double* w_s, const float2* w2,
                              const float4* grid_q, int64_t gq_stride, int members, double* g_s,
                              int64_t g_stride, cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    if (nt < 32 || nt > kInterpTileThreads || (nt & 31)) return cudaErrorInvalidValue;
    const size_t smem = interp_smem(qmax, tab.w, tab.deg, nt, kInterpHBytesPerThread * nt);
    cudaError_t e = cudaFuncSetAttribute(k_asy_interp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (members < 1) return cudaErrorInvalidValue;
    k_asy_interp<<<ntiles, nt, smem, s>>>(probs, blks, tiles, tab, w_s, w2, grid_q, gq_stride, members, g_s,
                                          g_stride);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace nuht
