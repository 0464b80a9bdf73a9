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
// Arithmetic: per-point set-up (coordinates, phases, weights' base) in FP64;
// kernel taps, weighted values and all tap sums in double-float (df64.cuh,
// ~48 bits, on the FP32 pipes); grids and the FFT in FP64.  The FFT output is
// stored split into (hi, lo) floats so that the interpolation reads it as
// double-float without FP64 work.
#include <cstdint>

#include "device_math.cuh"
#include "df64.cuh"
#include "nuht_internal.h"

namespace nuht {

namespace {

__device__ __forceinline__ double horner(const double* c, int deg, double v)
{
    double acc = c[deg];
    for (int k = deg - 1; k >= 0; --k) acc = fma(acc, v, c[k]);
    return acc;
}

// psi^(xi) from the piecewise-polynomial table (xi >= 0 within the table).
__device__ __forceinline__ double psihat(const Tables& T, double xi)
{
    xi = fabs(xi);
    double t = xi * T.ph_scale;
    int piece = (int)t;
    if (piece > T.ph_pieces - 1) piece = T.ph_pieces - 1;
    double v = 2.0 * (t - (double)piece) - 1.0;
    return horner(T.ph + piece * (T.ph_deg + 1), T.ph_deg, v);
}

// ------------------------------------------------------------------ spread
// One CTA per tile of consecutive (sorted) points of one block.  Phase 1:
// each thread prepares one point (grid cell l0, w kernel taps, the 2M
// weighted, pre-phased values).  Phase 2: each (cell, q) output of the tile's
// window is owned by one thread, which sums over the points whose taps cover
// that cell and adds the sum to the block's global grid.
__global__ void k_asy_spread(const ProbParams* __restrict__ probs, const AsyBlock* __restrict__ blks,
                             const Tile* __restrict__ tiles, Tables tab,
                             const double* __restrict__ r_s, const double* __restrict__ c_s,
                             double2* __restrict__ grid_b)
{
    extern __shared__ float4 smem4[];
    const Tile t = tiles[blockIdx.x];
    const AsyBlock B = blks[t.blk];
    const int Q = probs[B.prob].Q;
    const int w = tab.w, deg = tab.deg, nt = blockDim.x, tid = threadIdx.x;
    const int ncoef = w * (deg + 1);
    float4* aval = smem4;                                   // [nt][Q]: (re.h, re.l, im.h, im.l)
    float2* coef = (float2*)(aval + nt * Q);                // [w][deg+1]
    float2* taps = coef + ncoef;                            // [nt][w]
    int* l0s = (int*)(taps + nt * w);                       // [nt]
    for (int i = tid; i < ncoef; i += nt) coef[i] = tab.es2[i];
    __syncthreads();
    const int cnt = t.count;
    if (tid < cnt) {
        const int64_t j = t.start + tid;
        const double rj = r_s[j];
        const double x = rj - B.rc;
        const double a = x * B.inv_h - tab.half_w;
        const double lf = ceil(a);
        double z0 = lf - a;
        z0 = fmin(fmax(z0, 0.0), 1.0);
        const double v = 2.0 * z0 - 1.0;
        const float vh = (float)v, vl = (float)(v - (double)vh);
        for (int i = 0; i < w; ++i) {
            const df tp = horner_comp(coef + i * (deg + 1), deg, vh, vl);
            taps[tid * w + i] = make_float2(tp.h, tp.l);
        }
        l0s[tid] = (int)lf;
        double sn, cs;
        sincos_prod(B.wc, x, &sn, &cs);
        const double ratio = B.rho / rj;              // (r/rho)^(-1)
        const double w0 = c_s[j] * sqrt(ratio);       // c_j (r/rho)^(-1/2)
        const df rat = df_from(ratio);
        df wr = df_from(w0 * cs), wi = df_from(w0 * sn);
        for (int q = 0; q < Q; ++q) {
            aval[tid * Q + q] = make_float4(wr.h, wr.l, wi.h, wi.l);
            wr = df_mul(wr, rat);
            wi = df_mul(wi, rat);
        }
    }
    __syncthreads();
    const int lfirst = l0s[0];
    const int span = l0s[cnt - 1] - lfirst + w;
    const int nf1 = 2 * B.N1 + 1;
    double2* gb = grid_b + B.b_off;
    for (int item = tid; item < span * Q; item += nt) {
        const int c = item / Q, q = item - c * Q;
        const int cell = lfirst + c;
        // points with l0 in [cell - w + 1, cell]: l0s is non-decreasing
        int lo = 0, hi = cnt;
        const int key = cell - w + 1;
        while (lo < hi) { int mid = (lo + hi) >> 1; if (l0s[mid] < key) lo = mid + 1; else hi = mid; }
        const int p_lo = lo;
        hi = cnt;
        while (lo < hi) { int mid = (lo + hi) >> 1; if (l0s[mid] <= cell) lo = mid + 1; else hi = mid; }
        const int p_hi = lo;
        acc2 ar{0.f, 0.f}, ai{0.f, 0.f};
        for (int p = p_lo; p < p_hi; ++p) {
            const float2 k2 = taps[p * w + (cell - l0s[p])];
            const float4 av = aval[p * Q + q];
            const df k{k2.x, k2.y};
            acc_fma(ar, k, df{av.x, av.y});
            acc_fma(ai, k, df{av.z, av.w});
        }
        const int idx = cell + B.N1;
        if (p_hi > p_lo && idx >= 0 && idx < nf1) {
            atomicAdd(&gb[(int64_t)idx * Q + q].x, acc_value(ar));
            atomicAdd(&gb[(int64_t)idx * Q + q].y, acc_value(ai));
        }
    }
}

// -------------------------------------------------------------------- FFT
// In-place radix-2 FFT (e^{+2 pi i k n / N}) of N = 2^logN complex values in
// shared memory that were stored in bit-reversed order.  tw[k] =
// e^{2 pi i k / 2^tw_log2}.
__device__ void smem_fft(double2* X, int logN, const double2* __restrict__ tw, int tw_log2)
{
    const int N = 1 << logN;
    for (int s = 0; s < logN; ++s) {
        const int len = 1 << s;
        const int tw_shift = tw_log2 - (s + 1);
        for (int b = threadIdx.x; b < N / 2; b += blockDim.x) {
            const int pos = b & (len - 1);
            const int i0 = ((b >> s) << (s + 1)) + pos;
            const int i1 = i0 + len;
            const double2 wv = tw[pos << tw_shift];
            const double2 u = X[i0], v = X[i1];
            const double2 vw = make_double2(v.x * wv.x - v.y * wv.y, v.x * wv.y + v.y * wv.x);
            X[i0] = make_double2(u.x + vw.x, u.y + vw.y);
            X[i1] = make_double2(u.x - vw.x, u.y - vw.y);
        }
        __syncthreads();
    }
}

// Spread-grid value at FFT index t (mode l = t or t - nf2), corrected by
// 1/psi^(alpha2 l); zero outside |l| <= N1.
__device__ __forceinline__ double2 corrected_mode(const AsyBlock& B, const Tables& tab,
                                                  const double2* __restrict__ gb, int Q, int q, int tt)
{
    const int l = (tt < (B.nf2 >> 1)) ? tt : tt - B.nf2;
    if (l < -B.N1 || l > B.N1) return make_double2(0.0, 0.0);
    const double2 v = gb[(int64_t)(l + B.N1) * Q + q];
    const double s = 1.0 / psihat(tab, B.alpha2 * (double)l);
    return make_double2(v.x * s, v.y * s);
}

// Complex FP64 value stored as double-float parts (re.h, re.l, im.h, im.l).
__device__ __forceinline__ float4 split4(double2 v)
{
    const float rh = (float)v.x, ih = (float)v.y;
    return make_float4(rh, (float)(v.x - (double)rh), ih, (float)(v.y - (double)ih));
}

__global__ void k_asy_fft_small(const ProbParams* __restrict__ probs, const AsyBlock* __restrict__ blks,
                                const FftItem* __restrict__ items, Tables tab,
                                const double2* __restrict__ grid_b, float4* __restrict__ grid_q)
{
    extern __shared__ double2 X[];
    const FftItem it = items[blockIdx.x];
    const AsyBlock B = blks[it.blk];
    const int Q = probs[B.prob].Q;
    const int N = B.nf2, logN = B.log2nf2;
    const double2* gb = grid_b + B.b_off;
    for (int tt = threadIdx.x; tt < N; tt += blockDim.x)
        X[__brev(tt) >> (32 - logN)] = corrected_mode(B, tab, gb, Q, it.q, tt);
    __syncthreads();
    smem_fft(X, logN, tab.tw, tab.tw_log2);
    float4* gq = grid_q + B.q_off;
    for (int tt = threadIdx.x; tt < N; tt += blockDim.x) gq[(int64_t)tt * Q + it.q] = split4(X[tt]);
}

// Four-step FFT for nf2 = N1 * N2 > kFftSmemMax, N2 = kFftSmemMax.
// Pass A (line = n1): FFT over n2 of x[n1 + N1 n2], times e^{2 pi i n1 k2 / N},
// stored at tmp[n1 + N1 k2].  Pass B (line = k2): FFT over n1 of
// tmp[n1 + N1 k2], stored at X[k2 + N2 k1].
__global__ void k_asy_fft_pass_a(const ProbParams* __restrict__ probs, const AsyBlock* __restrict__ blks,
                                 const FftItem* __restrict__ items, Tables tab,
                                 const double2* __restrict__ grid_b, double2* __restrict__ tmp)
{
    extern __shared__ double2 X[];
    const FftItem it = items[blockIdx.x];
    const AsyBlock B = blks[it.blk];
    const int Q = probs[B.prob].Q;
    const int N = B.nf2;
    const int logN2 = 12, N2 = 1 << logN2;
    const int N1 = N >> logN2;
    const int n1 = it.line;
    const double2* gb = grid_b + B.b_off;
    for (int n2 = threadIdx.x; n2 < N2; n2 += blockDim.x)
        X[__brev(n2) >> (32 - logN2)] = corrected_mode(B, tab, gb, Q, it.q, n1 + N1 * n2);
    __syncthreads();
    smem_fft(X, logN2, tab.tw, tab.tw_log2);
    double2* tq = tmp + B.q_off;
    for (int k2 = threadIdx.x; k2 < N2; k2 += blockDim.x) {
        double s, c;
        // e^{2 pi i n1 k2 / N}: the argument (2 n1 k2 mod 2N) / N is exact in FP64
        const long long num = (2LL * n1 * k2) % (2LL * N);
        sincospi((double)num / (double)N, &s, &c);
        const double2 v = X[k2];
        tq[(int64_t)(n1 + N1 * k2) * Q + it.q] = make_double2(v.x * c - v.y * s, v.x * s + v.y * c);
    }
}

__global__ void k_asy_fft_pass_b(const ProbParams* __restrict__ probs, const AsyBlock* __restrict__ blks,
                                 const FftItem* __restrict__ items, Tables tab,
                                 const double2* __restrict__ tmp, float4* __restrict__ grid_q)
{
    extern __shared__ double2 X[];
    const FftItem it = items[blockIdx.x];
    const AsyBlock B = blks[it.blk];
    const int Q = probs[B.prob].Q;
    const int N = B.nf2;
    const int logN2 = 12, N2 = 1 << logN2;
    const int logN1 = B.log2nf2 - logN2, N1 = 1 << logN1;
    const int k2 = it.line;
    const double2* tq = tmp + B.q_off;
    for (int n1 = threadIdx.x; n1 < N1; n1 += blockDim.x)
        X[logN1 > 0 ? (__brev(n1) >> (32 - logN1)) : 0] = tq[(int64_t)(n1 + N1 * k2) * Q + it.q];
    __syncthreads();
    smem_fft(X, logN1, tab.tw, tab.tw_log2);
    float4* gq = grid_q + B.q_off;
    for (int k1 = threadIdx.x; k1 < N1; k1 += blockDim.x)
        gq[(int64_t)(k2 + N2 * k1) * Q + it.q] = split4(X[k1]);
    (void)N;
}

// ------------------------------------------------------------ interpolate
// One thread per frequency: interpolate the 2M FFT grids at theta = s h,
// deconvolve, post-phase, and combine the Hankel terms into g.
__global__ void k_asy_interp(const ProbParams* __restrict__ probs, const AsyBlock* __restrict__ blks,
                             const Tile* __restrict__ tiles, Tables tab,
                             const double* __restrict__ w_s, const float4* __restrict__ grid_q,
                             double* __restrict__ g_s)
{
    extern __shared__ float2 coef2[];
    const Tile t = tiles[blockIdx.x];
    const AsyBlock B = blks[t.blk];
    const ProbParams& P = probs[B.prob];
    const int w = tab.w, deg = tab.deg;
    for (int i = threadIdx.x; i < w * (deg + 1); i += blockDim.x) coef2[i] = tab.es2[i];
    __syncthreads();
    if ((int)threadIdx.x >= t.count) return;
    const int64_t k = t.start + threadIdx.x;
    const double wk = w_s[k];
    const double s = wk - B.wc;
    const double a = s * B.h * B.inv_delta - tab.half_w;
    const double tf = ceil(a);
    double z0 = tf - a;
    z0 = fmin(fmax(z0, 0.0), 1.0);
    const double v = 2.0 * z0 - 1.0;
    const float vh = (float)v, vl = (float)(v - (double)vh);
    float th[kMaxW], tl[kMaxW];
#pragma unroll
    for (int i = 0; i < kMaxW; ++i) {
        if (i < w) {
            const df tp = horner_comp(coef2 + i * (deg + 1), deg, vh, vl);
            th[i] = tp.h;
            tl[i] = tp.l;
        } else {
            th[i] = 0.f;
            tl[i] = 0.f;
        }
    }
    const int t0 = (int)tf;
    const int mask = B.nf2 - 1;
    const int Q = P.Q;
    const float4* gq = grid_q + B.q_off;
    const double m1 = 1.0 / (wk * B.rho);     // 1/(omega rho) < 1/z
    const df m1d = df_from(m1);
    // T = sum_q a_q i^q (omega rho)^(-q) P_q, accumulated in double-float
    acc2 tr{0.f, 0.f}, ti{0.f, 0.f};
    df mq{1.f, 0.f};
    for (int q = 0; q < Q; ++q) {
        acc2 pr{0.f, 0.f}, pi{0.f, 0.f};
#pragma unroll
        for (int i = 0; i < kMaxW; ++i) {
            if (i < w) {
                const float4 gv = gq[(int64_t)((t0 + i) & mask) * Q + q];
                const df tp{th[i], tl[i]};
                acc_fma(pr, tp, df{gv.x, gv.y});
                acc_fma(pi, tp, df{gv.z, gv.w});
            }
        }
        const df prd = fast_two_sum(pr.s, pr.c), pid = fast_two_sum(pi.s, pi.c);
        const df cq = df_mul(df{P.a2[q].x, P.a2[q].y}, mq);
        // multiply by i^q: (pr + i pi) i^q
        switch (q & 3) {
            case 0: acc_fma(tr, cq, prd); acc_fma(ti, cq, pid); break;
            case 1: acc_fma(tr, df{-cq.h, -cq.l}, pid); acc_fma(ti, cq, prd); break;
            case 2: acc_fma(tr, df{-cq.h, -cq.l}, prd); acc_fma(ti, df{-cq.h, -cq.l}, pid); break;
            default: acc_fma(tr, cq, pid); acc_fma(ti, df{-cq.h, -cq.l}, prd); break;
        }
        mq = df_mul(mq, m1d);
    }
    double sn, cs;
    sincos_prod(wk, B.rc, &sn, &cs);
    // e^{i (omega r_c + phi)}
    const double er = cs * P.cphi - sn * P.sphi;
    const double ei = sn * P.cphi + cs * P.sphi;
    const double scale = 0.7978845608028654 * sqrt(m1) * (4.0 / ((double)w * (double)w)) /
                         psihat(tab, B.alpha * s);
    const double val = scale * (er * acc_value(tr) - ei * acc_value(ti));
    atomicAdd(&g_s[k], (double)P.sgn * val);
}

}  // namespace

cudaError_t launch_asy_spread(const ProbParams* probs, const AsyBlock* blks, const Tile* tiles,
                              int ntiles, int qmax, Tables tab, const double* r_s,
                              const double* c_s, double2* grid_b, cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    const int nt = (qmax > 16) ? 128 : 256;
    size_t smem = sizeof(float4) * (size_t)nt * qmax + sizeof(float2) * (size_t)tab.w * (tab.deg + 1) +
                  sizeof(float2) * (size_t)nt * tab.w + sizeof(int) * (size_t)nt;
    cudaError_t e = cudaFuncSetAttribute(k_asy_spread, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_asy_spread<<<ntiles, nt, smem, s>>>(probs, blks, tiles, tab, r_s, c_s, grid_b);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_asy_fft_small(const ProbParams* probs, const AsyBlock* blks, const FftItem* items,
                                 int nitems, int max_nf2, Tables tab, const double2* grid_b,
                                 float4* grid_q, cudaStream_t s)
{
    if (nitems <= 0) return cudaSuccess;
    size_t smem = sizeof(double2) * (size_t)max_nf2;
    cudaError_t e = cudaFuncSetAttribute(k_asy_fft_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int nt = max_nf2 / 2;
    if (nt > 256) nt = 256;
    if (nt < 32) nt = 32;
    k_asy_fft_small<<<nitems, nt, smem, s>>>(probs, blks, items, tab, grid_b, grid_q);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_asy_fft_large(const ProbParams* probs, const AsyBlock* blks, const FftItem* items_a,
                                 int nitems_a, const FftItem* items_b, int nitems_b, Tables tab,
                                 const double2* grid_b, double2* tmp, float4* grid_q,
                                 cudaStream_t s)
{
    if (nitems_a <= 0) return cudaSuccess;
    size_t smem = sizeof(double2) * (size_t)kFftSmemMax;
    cudaError_t e = cudaFuncSetAttribute(k_asy_fft_pass_a, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_asy_fft_pass_b, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_asy_fft_pass_a<<<nitems_a, 256, smem, s>>>(probs, blks, items_a, tab, grid_b, tmp);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_asy_fft_pass_b<<<nitems_b, 256, smem, s>>>(probs, blks, items_b, tab, tmp, grid_q);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_asy_interp(const ProbParams* probs, const AsyBlock* blks, const Tile* tiles,
                              int ntiles, Tables tab, const double* w_s, const float4* grid_q,
                              double* g_s, cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    size_t smem = sizeof(float2) * (size_t)tab.w * (tab.deg + 1);
    k_asy_interp<<<ntiles, 128, smem, s>>>(probs, blks, tiles, tab, w_s, grid_q, g_s);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace nuht
