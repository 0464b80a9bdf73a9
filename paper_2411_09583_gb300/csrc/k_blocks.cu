// Work lists of a plan, built on the device from the block lists of the
// subdivision (Algorithm 1): per-block descriptors (local expansion, Sec. 3.1;
// type-3 geometry of the asymptotic blocks, Sec. 3.2 / 4.2; direct blocks),
// the offsets of their moments and grids, and the tile segments of every
// kernel.  Three kernels: sizes (one thread per block), column-wise exclusive
// prefix sums (one CTA), fill (one thread per block).  The block counts are
// read from device memory, so nothing here waits for the host.
#include <cmath>
#include <cstdint>

#include "nuht_internal.h"

namespace nuht {

// streaming multiprocessors of the current device, cached per device (k_det.cu)
int device_sm_count();

namespace {

__device__ __forceinline__ int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

__device__ __forceinline__ void atomic_max64(int64_t* p, int64_t v)
{
    atomicMax((unsigned long long*)p, (unsigned long long)v);   // values are non-negative
}

__device__ __forceinline__ int64_t clamp_count(int64_t c, int64_t cap) { return c < cap ? c : cap; }

__global__ void k_block_sizes(BlockBuild bb)
{
    const int64_t nl = clamp_count(bb.res[0], bb.ocap), na = clamp_count(bb.res[1], bb.ocap),
                  nd = clamp_count(bb.res[2], bb.ocap);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nl + na + nd;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (i < nl) {
            const SubBlk b = bb.sub[i];
            const ProbParams& P = bb.probs[b.prob];
            LocalBlock lb{};
            lb.prob = b.prob;
            lb.k0 = (int32_t)(b.k0 + P.w_off); lb.k1 = (int32_t)(b.k1 + P.w_off);
            lb.j0 = (int32_t)(b.j0 + P.r_off); lb.j1 = (int32_t)(b.j1 + P.r_off);
            lb.R = bb.bl[i];
            lb.R_h = (float)lb.R;
            lb.R_l = (float)(lb.R - (double)lb.R_h);
            const double iR = lb.R > 0.0 ? 1.0 / lb.R : 0.0;
            lb.iR_h = (float)iR;
            lb.iR_l = (float)(iR - (double)lb.iR_h);
            bb.loc[i] = lb;
            const int64_t rows = b.k1 - b.k0 + 1, cols = b.j1 - b.j0 + 1;
            int64_t* c = bb.lcnt + i * kLocalCols;
            c[LC_MOM] = P.L + 1;
            c[LC_TMOM] = ceil_div(cols, bb.mom_tile);
            c[LC_TEVAL] = ceil_div(rows, bb.eval_tile);
            c[LC_RC] = rows + cols;
        } else if (i < nl + na) {
            const int64_t a = i - nl;
            const SubBlk b = bb.sub[bb.ocap + a];
            const ProbParams& P = bb.probs[b.prob];
            const double4 e = bb.ba[a];   // r_j0, r_j1, omega_k0, omega_k1
            const int Q = P.Q;
            AsyBlock ab{};
            ab.prob = b.prob;
            ab.k0 = (int32_t)(b.k0 + P.w_off); ab.k1 = (int32_t)(b.k1 + P.w_off);
            ab.j0 = (int32_t)(b.j0 + P.r_off); ab.j1 = (int32_t)(b.j1 + P.r_off);
            // r_c rounded to a multiple of 2^(10 - fr) (any centre serves the
            // type-3 transform); the fixed-point frame keeps r < 2^(62 - fr)
            int er;
            frexp(e.y, &er);
            ab.fr = 62 - er;
            ab.rc = ldexp(rint(ldexp(0.5 * (e.x + e.y), ab.fr - 10)), 10 - ab.fr);
            ab.Rc_fx = (int64_t)ldexp(ab.rc, ab.fr);
            const double X = 0.5 * (e.y - e.x);
            {
                // w_c rounded to a multiple of 2^(10 - fw), like r_c
                int eo;
                frexp(e.w, &eo);
                ab.fw = 62 - eo;
                ab.wc = ldexp(rint(ldexp(0.5 * (e.z + e.w), ab.fw - 10)), 10 - ab.fw);
                ab.Wc_fx = (int64_t)ldexp(ab.wc, ab.fw);
            }
            const double S = 0.5 * (e.w - e.z);
            // a single frequency (S = 0) takes any spacing: one that puts the
            // block's points within a few cells (scale-free, unlike a constant)
            const double Seff = S > 0.0 ? S : (X > 0.0 ? 1.0 / X : 1.0);
            ab.h = M_PI / (2.0 * Seff);
            ab.inv_h = (2.0 / M_PI) * Seff;
            {
                int eh, ew;
                frexp(ab.inv_h, &eh);
                ab.KH = (int64_t)ldexp(ab.inv_h, 62 - eh);      // exact: 53-bit mantissa
                ab.sA = ab.fr + 62 - eh - 41;
                // w_c / (2 pi) in double-double, then 62 bits of it
                const double c_hi = 0.15915494309189535, c_lo = -9.839338337591243e-18;
                const double p = ab.wc * c_hi;
                const double err = fma(ab.wc, c_hi, -p) + ab.wc * c_lo;
                frexp(p, &ew);
                int64_t kw = llrint(ldexp(p, 62 - ew)) + llrint(ldexp(err, 62 - ew));
                int sw = ab.fr + 62 - ew - 64;
                if (sw > 64) {
                    kw = sw - 64 < 63 ? kw >> (sw - 64) : 0;
                    sw = 64;
                }
                ab.KW = kw;
                ab.sW = sw;
            }
            const bool fx_bad = ab.sA < 1 || ab.sA > 127 || ab.sW < 0;
            const double n1f = ceil(X * ab.inv_h + 0.5 * bb.w) + 1.0;   // one cell of rounding margin
            int64_t* c = bb.acnt + a * kAsyCols;
            for (int k = 0; k < kAsyCols; ++k) c[k] = 0;
            bb.fcls[a] = -1;
            if (fx_bad || !(n1f <= (double)(1 << 22))) {
                atomic_max64(&bb.maxv[MX_ERR], 1);
                continue;
            }
            ab.N1 = (int32_t)n1f;
            const int64_t nf1 = 2 * (int64_t)ab.N1 + 1;
            int lg = 64 - __clzll((long long)(2 * nf1 - 1));   // smallest 2^lg >= 2 nf1
            if (lg < 5) lg = 5;
            if (lg > kFftMaxLog2) {
                atomic_max64(&bb.maxv[MX_ERR], 1);
                continue;
            }
            ab.log2nf2 = lg;
            ab.nf2 = 1 << lg;
            ab.rho = e.x;
            ab.alpha = 0.5 * bb.w * ab.h;
            ab.alpha2 = ldexp(bb.w * M_PI, -lg);
            ab.inv_delta = ab.nf2 * (0.5 / M_PI);
            ab.hd = ab.h * ab.inv_delta;
            ab.alpha_h = (float)ab.alpha;
            ab.alpha_l = (float)(ab.alpha - (double)ab.alpha_h);
            {
                int ed, er2;
                frexp(ab.hd, &ed);
                ab.KD = (int64_t)ldexp(ab.hd, 62 - ed);          // exact: 53-bit mantissa
                ab.sD = ab.fw + 62 - ed - 40;   // 40 fractional bits: |s hd| <= nf2 / 4 <= 2^22
                const double c_hi = 0.15915494309189535, c_lo = -9.839338337591243e-18;
                const double p = ab.rc * c_hi;
                const double err = fma(ab.rc, c_hi, -p) + ab.rc * c_lo;
                frexp(p, &er2);
                int64_t kr = llrint(ldexp(p, 62 - er2)) + llrint(ldexp(err, 62 - er2));
                int sr = ab.fw + 62 - er2 - 64;
                if (sr > 64) {
                    kr = sr - 64 < 63 ? kr >> (sr - 64) : 0;
                    sr = 64;
                }
                ab.KRc = kr;
                ab.sR = sr;
                if (ab.sD < 1 || ab.sD > 127 || sr < 0) {
                    atomic_max64(&bb.maxv[MX_ERR], 1);
                    continue;
                }
            }
            ab.rho_h = (float)ab.rho;
            ab.rho_l = (float)(ab.rho - (double)ab.rho_h);
            bb.asy[a] = ab;
            const int64_t rows = b.k1 - b.k0 + 1, cols = b.j1 - b.j0 + 1;
            c[AC_GB] = nf1 * Q;
            c[AC_GQ] = (int64_t)ab.nf2 * Q;
            c[AC_TSPREAD] = ceil_div(cols, bb.spread_tile);
            c[AC_TINTERP] = ceil_div(rows, bb.interp_tile);
            if ((int64_t)ab.nf2 * Q <= kFftSmemMax) {             // all Q grids in one CTA
                bb.fcls[a] = 0;
                c[AC_NFK] = 1;
                c[AC_IFK] = 1;
                atomic_max64(&bb.maxv[MX_FBLOCK_PTS], (int64_t)ab.nf2 * Q);
            } else if (ab.nf2 <= kFftSingleMax) {                 // one CTA per grid
                bb.fcls[a] = 1;
                c[AC_NFS] = 1;
                c[AC_IFS] = Q;
                atomic_max64(&bb.maxv[MX_NF2_SMALL], ab.nf2);
            } else {                                              // two passes, groups of lines
                bb.fcls[a] = 2;
                c[AC_NFL] = 1;
                const int logN2 = (lg + 1) >> 1, logN1 = lg - logN2;
                const int lpcA = (kFftLineBatch >> logN2) > 0 ? (kFftLineBatch >> logN2) : 1;
                const int lpcB = (kFftLineBatch >> logN1) > 0 ? (kFftLineBatch >> logN1) : 1;
                c[AC_IFA] = (int64_t)Q * (((1 << logN1) + lpcA - 1) / lpcA);
                c[AC_IFB] = (int64_t)Q * (((1 << logN2) + lpcB - 1) / lpcB);
                atomic_max64(&bb.maxv[MX_LARGE], 1);
            }
            c[AC_RC] = rows + cols;
            c[AC_NF2] = ab.nf2;
        } else {
            const int64_t d = i - nl - na;
            const SubBlk b = bb.sub[2 * bb.ocap + d];
            const ProbParams& P = bb.probs[b.prob];
            bb.dir[d] = DirectBlock{b.prob, (int32_t)(b.k0 + P.w_off), (int32_t)(b.k1 + P.w_off),
                                    (int32_t)(b.j0 + P.r_off), (int32_t)(b.j1 + P.r_off), 0};
            const int64_t rows = b.k1 - b.k0 + 1, cols = b.j1 - b.j0 + 1;
            bb.dcnt[d] = rows * cols;
            atomic_max64(&bb.maxv[MX_DIR_ROWS], rows);
            atomic_max64(&bb.maxv[MX_DIR_COLS], cols);
            atomic_max64(&bb.maxv[MX_DIR_AREA], rows * cols);
        }
    }
}

// Exclusive prefix sums of the columns of the three counter matrices
// (row-major, rows = blocks) in place, and the column totals: tile sums (one
// CTA per kScanTile rows), one CTA over the tile sums, then each tile again
// with its offset.  blockIdx.y picks the matrix.
constexpr int kScanTile = 256;

struct ScanMat {
    int64_t* mat;
    int64_t n;
    int ncol;
    int64_t* totals;
};

__device__ __forceinline__ ScanMat scan_mat(const BlockBuild& bb, int which)
{
    if (which == 0) return ScanMat{bb.lcnt, clamp_count(bb.res[0], bb.ocap), kLocalCols, bb.totals + TOT_LOCAL};
    if (which == 1) return ScanMat{bb.acnt, clamp_count(bb.res[1], bb.ocap), kAsyCols, bb.totals + TOT_ASY};
    return ScanMat{bb.dcnt, clamp_count(bb.res[2], bb.ocap), kDirCols, bb.totals + TOT_DIR};
}

// block-wide inclusive scan of one value per thread (kScanTile threads)
__device__ __forceinline__ int64_t block_incl_scan(int64_t v, int64_t* wsum, int64_t* total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int64_t s = lane < kScanTile / 32 ? wsum[lane] : 0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, s, off);
            if (lane >= off) s += y;
        }
        if (lane < kScanTile / 32) wsum[lane] = s;
    }
    __syncthreads();
    const int64_t r = x + (wid > 0 ? wsum[wid - 1] : 0);
    *total = wsum[kScanTile / 32 - 1];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanTile) k_scan_tiles(BlockBuild bb, int64_t* part, int64_t ptiles)
{
    __shared__ int64_t wsum[kScanTile / 32];
    const ScanMat S = scan_mat(bb, blockIdx.y);
    const int64_t row = blockIdx.x * (int64_t)kScanTile + threadIdx.x;
    if ((int64_t)blockIdx.x * kScanTile >= S.n) return;   // whole CTA
    for (int c = 0; c < S.ncol; ++c) {
        int64_t tot;
        block_incl_scan(row < S.n ? S.mat[row * S.ncol + c] : 0, wsum, &tot);
        if (threadIdx.x == 0) part[((int64_t)blockIdx.y * ptiles + blockIdx.x) * kAsyCols + c] = tot;
    }
}

__global__ void __launch_bounds__(kScanTile) k_scan_top(BlockBuild bb, int64_t* part, int64_t ptiles)
{
    __shared__ int64_t wsum[kScanTile / 32];
    for (int which = 0; which < 3; ++which) {
        const ScanMat S = scan_mat(bb, which);
        const int64_t nt = (S.n + kScanTile - 1) / kScanTile;
        for (int c = 0; c < S.ncol; ++c) {
            int64_t carry = 0;
            for (int64_t t0 = 0; t0 < nt; t0 += kScanTile) {
                const int64_t t = t0 + threadIdx.x;
                int64_t* pp = part + ((int64_t)which * ptiles + t) * kAsyCols + c;
                const int64_t v = t < nt ? *pp : 0;
                int64_t tot;
                const int64_t incl = block_incl_scan(v, wsum, &tot);
                if (t < nt) *pp = carry + incl - v;   // exclusive offset of the tile
                carry += tot;
            }
            if (threadIdx.x == 0) S.totals[c] = carry;
        }
    }
}

__global__ void __launch_bounds__(kScanTile) k_scan_apply(BlockBuild bb, const int64_t* part, int64_t ptiles)
{
    __shared__ int64_t wsum[kScanTile / 32];
    const ScanMat S = scan_mat(bb, blockIdx.y);
    const int64_t row = blockIdx.x * (int64_t)kScanTile + threadIdx.x;
    if ((int64_t)blockIdx.x * kScanTile >= S.n) return;
    for (int c = 0; c < S.ncol; ++c) {
        const int64_t v = row < S.n ? S.mat[row * S.ncol + c] : 0;
        int64_t tot;
        const int64_t incl = block_incl_scan(v, wsum, &tot);
        if (row < S.n)
            S.mat[row * S.ncol + c] = part[((int64_t)blockIdx.y * ptiles + blockIdx.x) * kAsyCols + c] + incl - v;
    }
}

__device__ __forceinline__ void put_seg(const BuildLists& L, int list, int64_t idx, int32_t blk, int32_t len,
                                        int64_t first, int64_t last, int64_t prefix)
{
    L.seg[list][idx] = Seg{blk, len, first, last};
    L.pre[list][idx] = (int32_t)prefix;
}

__global__ void k_block_fill(BlockBuild bb, BuildLists L)
{
    const int64_t nl = clamp_count(bb.res[0], bb.ocap), na = clamp_count(bb.res[1], bb.ocap),
                  nd = clamp_count(bb.res[2], bb.ocap);
    const int64_t* tl = bb.totals + TOT_LOCAL;
    const int64_t* ta = bb.totals + TOT_ASY;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        // closing entries of the prefix arrays
        L.pre[LIST_MOM][nl] = (int32_t)tl[LC_TMOM];
        L.pre[LIST_EVAL][nl] = (int32_t)tl[LC_TEVAL];
        L.pre[LIST_SPREAD][na] = (int32_t)ta[AC_TSPREAD];
        L.pre[LIST_INTERP][na] = (int32_t)ta[AC_TINTERP];
        L.pre[LIST_FBLOCK][ta[AC_NFK]] = (int32_t)ta[AC_IFK];
        L.pre[LIST_FSMALL][ta[AC_NFS]] = (int32_t)ta[AC_IFS];
        L.pre[LIST_FA][ta[AC_NFL]] = (int32_t)ta[AC_IFA];
        L.pre[LIST_FB][ta[AC_NFL]] = (int32_t)ta[AC_IFB];
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nl + na + nd;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (i < nl) {
            const int64_t* c = bb.lcnt + i * kLocalCols;
            LocalBlock lb = bb.loc[i];
            lb.mom_off = c[LC_MOM];
            L.loc[i] = lb;
            put_seg(L, LIST_MOM, i, (int32_t)i, bb.mom_tile, lb.j0, lb.j1, c[LC_TMOM]);
            put_seg(L, LIST_EVAL, i, (int32_t)i, bb.eval_tile, lb.k0, lb.k1, c[LC_TEVAL]);
            L.blk[i] = SubBlk{lb.k0, lb.k1, lb.j0, lb.j1, lb.prob};
        } else if (i < nl + na) {
            const int64_t a = i - nl;
            const int64_t* c = bb.acnt + a * kAsyCols;
            AsyBlock ab = bb.asy[a];
            ab.b_off = c[AC_GB];
            ab.q_off = c[AC_GQ];
            L.asy[a] = ab;
            put_seg(L, LIST_SPREAD, a, (int32_t)a, bb.spread_tile, ab.j0, ab.j1, c[AC_TSPREAD]);
            put_seg(L, LIST_INTERP, a, (int32_t)a, bb.interp_tile, ab.k0, ab.k1, c[AC_TINTERP]);
            const int Q = bb.probs[ab.prob].Q;
            if (bb.fcls[a] == 0) {
                put_seg(L, LIST_FBLOCK, c[AC_NFK], (int32_t)a, 1, 0, 0, c[AC_IFK]);
            } else if (bb.fcls[a] == 1) {
                put_seg(L, LIST_FSMALL, c[AC_NFS], (int32_t)a, 1, 0, Q - 1, c[AC_IFS]);
            } else {
                const int lg = ab.log2nf2;
                const int logN2 = (lg + 1) >> 1, logN1 = lg - logN2;
                const int lpcA = (kFftLineBatch >> logN2) > 0 ? (kFftLineBatch >> logN2) : 1;
                const int lpcB = (kFftLineBatch >> logN1) > 0 ? (kFftLineBatch >> logN1) : 1;
                const int64_t ia = (int64_t)Q * (((1 << logN1) + lpcA - 1) / lpcA);
                const int64_t ib = (int64_t)Q * (((1 << logN2) + lpcB - 1) / lpcB);
                put_seg(L, LIST_FA, c[AC_NFL], (int32_t)a, 1, 0, ia - 1, c[AC_IFA]);
                put_seg(L, LIST_FB, c[AC_NFL], (int32_t)a, 1, 0, ib - 1, c[AC_IFB]);
            }
            L.blk[nl + a] = SubBlk{ab.k0, ab.k1, ab.j0, ab.j1, ab.prob};
        } else {
            const int64_t d = i - nl - na;
            const DirectBlock db = bb.dir[d];
            L.dir[d] = db;
            L.blk[nl + na + d] = SubBlk{db.k0, db.k1, db.j0, db.j1, db.prob};
        }
    }
}

}  // namespace

int64_t block_scan_scratch(int64_t cap) { return 3 * ((cap + kScanTile - 1) / kScanTile) * kAsyCols; }

cudaError_t launch_block_build(const BlockBuild& bb, int64_t* scratch, cudaStream_t s)
{
    k_block_sizes<<<device_sm_count() * 8, 256, 0, s>>>(bb);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t ptiles = (bb.ocap + kScanTile - 1) / kScanTile;
    if (ptiles > 0) {
        const dim3 grid((unsigned)ptiles, 3);
        k_scan_tiles<<<grid, kScanTile, 0, s>>>(bb, scratch, ptiles);
        k_scan_top<<<1, kScanTile, 0, s>>>(bb, scratch, ptiles);
        k_scan_apply<<<grid, kScanTile, 0, s>>>(bb, scratch, ptiles);
    }
    count_launches(4);
    return cudaGetLastError();
}

cudaError_t launch_block_fill(const BlockBuild& bb, const BuildLists& L, cudaStream_t s)
{
    k_block_fill<<<device_sm_count() * 8, 256, 0, s>>>(bb, L);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace nuht
