// Local blocks (Wimp expansion, Sec. 3.1) and direct blocks (Sec. 4.1).
//
// A local block A(k0:k1, j0:j1) with R = max r of the block is applied as the
// rank-(L+1) product of Sec. 3.1:
//     moments   mu_l = sum_j c_j T_{2l(+1)}(r_j / R),       l = 0..L
//     evaluate  g_k += sum_l C_l(omega_k R) mu_l,
// C_l(x) = delta_l J_{nu/2+l}(x/2) J_{nu/2-l}(x/2) for even nu and
// 2 J_{(nu+1)/2+l}(x/2) J_{(nu-1)/2-l}(x/2) with T_{2l+1} for odd nu (the
// argument x/2 follows the proof of Lemma 3.1; the odd form is Graf's addition
// theorem with both arguments x/2).  All in FP64.
//
// Direct blocks are small mixed blocks summed entry by entry with a device
// J_nu: Miller recurrence (or the power series) where omega r <= z, and the
// M-term Hankel expansion, accurate to eps there by the choice of z, where
// omega r > z.
#include <cstdint>

#include "device_math.cuh"
#include "nuht_internal.h"

namespace nuht {

namespace {

constexpr int kMomThreads = 128;

// One CTA per tile of columns of one local block.  Each thread keeps its own
// column of partial moments in shared memory (acc[l * blockDim + tid]); the
// columns are summed at the end and added to the block's moments.
__global__ void __launch_bounds__(kMomThreads)
k_local_moments(const ProbParams* __restrict__ probs, const LocalBlock* __restrict__ blks,
                const Tile* __restrict__ tiles, const double* __restrict__ r_s,
                const double* __restrict__ c_s, double* __restrict__ mom)
{
    extern __shared__ double acc[];
    const Tile t = tiles[blockIdx.x];
    const LocalBlock B = blks[t.blk];
    const int L = probs[B.prob].L;
    const int odd = probs[B.prob].nu & 1;
    const int nt = blockDim.x, tid = threadIdx.x;
    for (int l = 0; l <= L; ++l) acc[l * nt + tid] = 0.0;
    const double invR = B.R > 0.0 ? 1.0 / B.R : 0.0;
    for (int64_t j = t.start + tid; j < t.start + t.count; j += nt) {
        const double y = r_s[j] * invR;
        const double cj = c_s[j];
        const double u = fma(2.0 * y, y, -1.0);   // T_2(y)
        const double u2 = 2.0 * u;
        // even: T_{2l}(y) = T_l(u); odd: T_{2l+1}(y) with T_1 = y, T_3 = y (2u - 1)
        double t0 = odd ? y : 1.0;
        double t1 = odd ? y * (u2 - 1.0) : u;
        acc[tid] += cj * t0;
        if (L >= 1) acc[nt + tid] += cj * t1;
        for (int l = 2; l <= L; ++l) {
            double t2 = fma(u2, t1, -t0);
            acc[l * nt + tid] = fma(cj, t2, acc[l * nt + tid]);
            t0 = t1;
            t1 = t2;
        }
    }
    __syncthreads();
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    for (int l = warp; l <= L; l += nw) {
        double s = 0.0;
        for (int k = lane; k < nt; k += 32) s += acc[l * nt + k];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
        if (lane == 0) atomicAdd(&mom[B.mom_off + l], s);
    }
}

// One thread per row of a local block.  J_0..J_ntop(x/2) by Miller's backward
// recurrence, kept (unnormalised) in this thread's column of shared memory,
// then sum_l C_l mu_l divided by the square of the normalisation.
__global__ void k_local_eval(const ProbParams* __restrict__ probs, const LocalBlock* __restrict__ blks,
                             const Tile* __restrict__ tiles, const double* __restrict__ w_s,
                             const double* __restrict__ mom, double* __restrict__ g_s)
{
    extern __shared__ double jb[];
    const Tile t = tiles[blockIdx.x];
    const LocalBlock B = blks[t.blk];
    const ProbParams& P = probs[B.prob];
    const int nt = blockDim.x, tid = threadIdx.x;
    if (tid >= t.count) return;
    const int64_t k = t.start + tid;
    const int nu = P.nu, L = P.L;
    const double* mu = mom + B.mom_off;
    const double x = w_s[k] * B.R;
    const double y = 0.5 * x;
    double val;
    if (y < 1e-100) {
        // J_n(y) = delta_n0 to far below rounding: only C_0 survives, and only for nu = 0
        val = (nu == 0) ? mu[0] : 0.0;
    } else {
        const int hp = (nu & 1) ? (nu + 1) / 2 : nu / 2;   // index paired with +l
        const int hm = (nu & 1) ? (nu - 1) / 2 : nu / 2;   // index paired with -l
        const int ntop = hp + L;
        const int ns = miller_start(ntop, y);
        const double inv2y = 2.0 / y;
        double jp1 = 0.0, jc = 1.0, S = 2.0;
        if (ns <= ntop) jb[ns * nt + tid] = jc;
        for (int i = ns; i >= 2; i -= 2) {
            double jm = fma((double)i * inv2y, jc, -jp1);
            double jmm = fma((double)(i - 1) * inv2y, jm, -jc);
            if (i - 1 <= ntop) jb[(i - 1) * nt + tid] = jm;
            if (i - 2 <= ntop) jb[(i - 2) * nt + tid] = jmm;
            S = fma(2.0, jmm, S);
            jp1 = jm;
            jc = jmm;
            if (too_big(jc)) {
                const double sc = 1e-150;
                jc *= sc; jp1 *= sc; S *= sc;
                int top = ntop < ns ? ntop : ns;
                for (int q = i - 2; q <= top; ++q) jb[q * nt + tid] *= sc;
            }
        }
        S -= jc;
        double sum = 0.0;
        for (int l = 0; l <= L; ++l) {
            int a = hp + l;
            int b = hm - l;
            double jbv;
            if (b >= 0) {
                jbv = jb[b * nt + tid];
            } else {
                jbv = jb[(-b) * nt + tid];
                if ((-b) & 1) jbv = -jbv;
            }
            double cl = jb[a * nt + tid] * jbv;
            if (l > 0 || (nu & 1)) cl *= 2.0;
            sum = fma(cl, mu[l], sum);
        }
        val = sum / (S * S);
    }
    atomicAdd(&g_s[k], (double)P.sgn * val);
}

// One CTA per direct block (area <= min_size): entries in parallel, row sums
// in shared memory, then one atomic add per row.
__global__ void k_direct(const ProbParams* __restrict__ probs, const DirectBlock* __restrict__ blks,
                         const double* __restrict__ r_s, const double* __restrict__ w_s,
                         const double* __restrict__ c_s, double* __restrict__ g_s)
{
    extern __shared__ double rowacc[];
    const DirectBlock B = blks[blockIdx.x];
    const ProbParams& P = probs[B.prob];
    const int rows = B.k1 - B.k0 + 1, cols = B.j1 - B.j0 + 1;
    const int area = rows * cols;
    for (int i = threadIdx.x; i < rows; i += blockDim.x) rowacc[i] = 0.0;
    __syncthreads();
    for (int e = threadIdx.x; e < area; e += blockDim.x) {
        const int rr = e / cols, cc = e - rr * cols;
        const double w = w_s[B.k0 + rr], r = r_s[B.j0 + cc];
        const double x = w * r;
        const double v = (x <= P.z) ? jn_small_arg(P.nu, x) : jn_hankel(P, w, r);
        atomicAdd(&rowacc[rr], v * c_s[B.j0 + cc]);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < rows; i += blockDim.x)
        atomicAdd(&g_s[B.k0 + i], (double)P.sgn * rowacc[i]);
}

}  // namespace

cudaError_t launch_local_moments(const ProbParams* probs, const LocalBlock* blks, const Tile* tiles,
                                 int ntiles, int lmax, const double* r_s, const double* c_s,
                                 double* mom, cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    size_t smem = sizeof(double) * (size_t)(lmax + 1) * kMomThreads;
    cudaError_t e = cudaFuncSetAttribute(k_local_moments, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_local_moments<<<ntiles, kMomThreads, smem, s>>>(probs, blks, tiles, r_s, c_s, mom);
    count_launches(1);
    return cudaGetLastError();
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
                                   int ntiles, int ntop_max, int threads, const double* w_s,
                                   const double* mom, double* g_s, cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    size_t smem = sizeof(double) * (size_t)(ntop_max + 1) * threads;
    cudaError_t e = cudaFuncSetAttribute(k_local_eval, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_local_eval<<<ntiles, threads, smem, s>>>(probs, blks, tiles, w_s, mom, g_s);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_direct(const ProbParams* probs, const DirectBlock* blks, int nblk, int max_rows,
                               const double* r_s, const double* w_s, const double* c_s, double* g_s,
                               cudaStream_t s)
{
    if (nblk <= 0) return cudaSuccess;
    size_t smem = sizeof(double) * (size_t)(max_rows > 0 ? max_rows : 1);
    cudaError_t e = cudaFuncSetAttribute(k_direct, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_direct<<<nblk, 128, smem, s>>>(probs, blks, r_s, w_s, c_s, g_s);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace nuht
