// Internal types of the GB300 NUHT library (host + device).
//
// A plan holds one or more problems (a batch).  Every block of the
// subdivision (Algorithm 1) carries the index of its problem, so the same
// kernels serve a single transform and a batch of uneven ones.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "nuht.h"
#include "det_acc.cuh"

namespace nuht {

constexpr int kMaxM = 20;           // Hankel term pairs (Sec. 3.3 caps M at 20)
constexpr int kMaxQ = 2 * kMaxM;    // weight powers q = 0..2M-1
constexpr int kMaxW = 16;           // ES kernel width
constexpr int kMaxDeg = 20;         // degree of the kernel piece polynomials
// An asymptotic block whose half-widths X (in r) and S (in omega) have
// X S above this is cut into quadrants (all asymptotic) until it is not: its
// spreading grid then has N1 ~ 2 X S / pi + w/2 <= ~2.04e6 cells and its FFT
// at most 2^23 points (the single-FFT limit is 2^kFftMaxLog2).
constexpr double kAsyMaxXS = 3.2e6;
constexpr int kMomFold = 32;        // FP32 partial sums of the spreading moments span at most this many points
constexpr int kMaxNtop = 400;       // largest Bessel index kept by the local evaluation
                                    // (the transposed moments then stay within 205 KB of shared memory)
constexpr int kFftSmemMax = 4096;   // points of all Q grids of a block FFT'd by one CTA
constexpr int kFftSingleMax = 8192; // largest single-grid FFT done by one CTA (128 KiB)
constexpr int kFftLineBatch = 4096; // points per CTA in the passes of a two-pass FFT
constexpr int kFftMaxLog2 = 24;     // largest FFT (two passes of <= 4096-point lines)

// Per-problem constants.
struct ProbParams {
    int nu;        // |nu|
    int sgn;       // (-1)^nu when the user order was negative, else +1
    int M, L, Q;   // Q = 2M
    int qs;        // terms q >= qs are small enough to be summed in FP32
    int ntop;      // largest Bessel index used by the local evaluation
    int fxs;       // accumulation: kFxOff = FP64 atomics; else the deterministic mode's
                   // fixed-point scale kFxScale (contributions add round(v 2^fxs) exactly)
    int8_t dcp[kMaxQ / 2];   // per Hankel pair (2p, 2p+1): double-float degrees of the interpolation sums
    double z;      // crossover
    double cphi, sphi;           // cos, sin of phi = -(2 nu + 1) pi / 4
    float2 cphi2, sphi2;         // the same as double-float
    double a[kMaxQ];             // Hankel coefficients a_q(nu), q < Q
    float2 a2[kMaxQ];            // a_q z^-q as double-float (in FP32 range for every order)
    float2 z2;                   // z as double-float
    int64_t r_off, w_off;        // offsets of this problem in the sorted arrays
    int64_t n, m;
    int64_t c_off, g_off;        // offsets of this problem's c and g (batched)
    const float4* tw2;           // the plan's table e^{2 pi i k / 8192}, k < 4096, as double-float
                                 // (cos h, cos l, sin h, sin l): phases of the direct entries
};

// Local block: rows k0..k1 (omega), columns j0..j1 (r), absolute indices into
// the concatenated sorted arrays.  R = largest r of the block.
struct LocalBlock {
    int32_t prob, k0, k1, j0, j1, pad;
    double R;
    int64_t mom_off;   // offset of the block's L+1 moments
    float R_h, R_l;    // R as double-float
    float iR_h, iR_l;  // 1 / R as double-float (0 when R = 0)
};

// Asymptotic block: type-3 NUFFT geometry (centres, grid spacings, sizes).
struct AsyBlock {
    int32_t prob, k0, k1, j0, j1;
    int32_t N1;        // spread grid cells l = -N1..N1
    int32_t nf2;       // FFT size (power of two)
    int32_t log2nf2;
    int64_t b_off;     // complex offset of the spread grid  [2 N1 + 1][Q]
    int64_t q_off;     // complex offset of the FFT output   [nf2][Q]
    double rc, wc;     // centres of the r and omega ranges
    double h;          // spread grid spacing in r: h = pi / (sigma S)
    double inv_h;
    double rho;        // smallest r of the block (weights are (r/rho)^(-q-1/2))
    double alpha;      // w h / 2: outer deconvolution argument scale
    double alpha2;     // w Delta / 2 with Delta = 2 pi / nf2
    double inv_delta;  // nf2 / (2 pi)
    double hd;         // h * inv_delta: a frequency offset s sits at FFT-grid position s * hd
    float rho_h, rho_l;   // rho as double-float
    // Fixed-point frame of the points (integer arithmetic instead of FP64,
    // whose rate is 1/64 of FP32 here): R = round(r 2^fr) < 2^62, X = R - Rc_fx
    // (r_c is a multiple of 2^(10 - fr), so Rc_fx is exact); the cell
    // coordinate a = x / h is bits [sA, sA + 63] of X * KH (41 fractional
    // bits; KH = inv_h 2^(sA + 41 - fr) exactly), and the phase w_c x / (2 pi)
    // in turns is bits [sW, sW + 63] of X * KW (64 fractional bits).
    int64_t Rc_fx, KH, KW;
    int32_t fr, sA, sW, pad_fx;
    // The same for the frequencies: Om = round(omega 2^fw) < 2^62, S = Om - Wc_fx
    // (w_c a multiple of 2^(10 - fw)); the FFT-grid coordinate s hd is bits
    // [sD, sD + 63] of S * KD (40 fractional bits), the phase omega r_c / (2 pi)
    // in turns bits [sR, sR + 63] of Om * KRc (64 fractional bits).
    int64_t Wc_fx, KD, KRc;
    int32_t fw, sD, sR;
    float alpha_h, alpha_l;   // alpha as double-float
    int32_t pad_fx2;
};

struct DirectBlock {
    int32_t prob, k0, k1, j0, j1, pad;
};

// A contiguous run of points (or frequencies) of one block.
struct Tile {
    int32_t blk;
    int32_t count;
    int64_t start;     // absolute index into the sorted array
};

// A run of tiles: indices first..last of block blk cut into tiles of len.
// Tile lists are expanded from these on the device (k_expand_tiles).  FFT work
// items are tiles of length one whose start is the item's ordinal in its
// block (q for single-pass FFTs, q * lines + line for the two-pass passes).
struct Seg {
    int32_t blk, len;
    int64_t first, last;
};

// A block of the subdivision in problem-local sorted indices: rows k0..k1
// (frequencies), columns j0..j1 (points), problem prob of a batch.
struct SubBlk {
    int32_t k0, k1, j0, j1, prob;
};

// Building the work lists on the device (k_blocks.cu): per-block counters
// (columns), their exclusive prefix sums and totals, maxima, and the tile lists.
enum { LC_MOM, LC_TMOM, LC_TEVAL, LC_RC, kLocalCols };
enum { AC_GB, AC_GQ, AC_TSPREAD, AC_TINTERP, AC_NFK, AC_NFS, AC_NFL, AC_IFK, AC_IFS, AC_IFA, AC_IFB,
       AC_RC, AC_NF2, kAsyCols };
enum { DC_ENTRIES, kDirCols };
enum { TOT_LOCAL = 0, TOT_ASY = kLocalCols, TOT_DIR = kLocalCols + kAsyCols,
       kTotals = kLocalCols + kAsyCols + kDirCols };
enum { MX_DIR_ROWS, MX_DIR_COLS, MX_DIR_AREA, MX_NF2_SMALL, MX_LARGE, MX_ERR, MX_FBLOCK_PTS, kMaxv };
enum { LIST_MOM, LIST_EVAL, LIST_SPREAD, LIST_INTERP, LIST_FSMALL, LIST_FA, LIST_FB, LIST_FBLOCK, kLists };

struct BlockBuild {
    const int64_t* res;       // counts of local, asymptotic, direct blocks (device)
    const SubBlk* sub;        // [3][ocap] the subdivision's lists, problem-local indices
    int64_t ocap;
    const double* bl;         // [nl] r at the last column of each local block
    const double4* ba;        // [na] (r_j0, r_j1, omega_k0, omega_k1) of each asymptotic block
    const ProbParams* probs;
    int w, mom_tile, eval_tile, spread_tile, interp_tile;
    LocalBlock* loc;          // descriptors before their offsets are known
    AsyBlock* asy;
    DirectBlock* dir;
    int8_t* fcls;             // FFT class of each asymptotic block (0 one CTA, 1 per grid, 2 two passes)
    int64_t* lcnt;            // [nl][kLocalCols] counters, then exclusive prefix sums
    int64_t* acnt;            // [na][kAsyCols]
    int64_t* dcnt;            // [nd][kDirCols]
    int64_t* totals;          // [kTotals] column sums
    int64_t* maxv;            // [kMaxv]
};

struct BuildLists {
    LocalBlock* loc;
    AsyBlock* asy;
    DirectBlock* dir;
    Seg* seg[kLists];
    int32_t* pre[kLists];     // [nseg + 1] tiles before each segment
    SubBlk* blk;              // [nl + na + nd] every block in global sorted indices
};

int64_t block_scan_scratch(int64_t cap);   // int64 elements of scratch for launch_block_build
cudaError_t launch_block_build(const BlockBuild& bb, int64_t* scratch, cudaStream_t s);
cudaError_t launch_block_fill(const BlockBuild& bb, const BuildLists& L, cudaStream_t s);

// Kernel tables shared by every asymptotic block of a plan.
struct Tables {
    const double* es;      // [w][deg + 1] monomial coefficients in v = 2 z0 - 1
    const float2* es2;     // the same as double-float (hi, lo)
    int w, deg;
    int deg_comp;          // degrees above this one are evaluated in plain FP32
    const float2* ch2;     // [w][deg + 1] pieces in the Chebyshev basis T_d(v), double-float
    int nb;                // Chebyshev terms kept (tail below 1e-3 eps)
    int dcs;               // spreading moments of degree >= dcs accumulate in plain FP32
    int dci;               // interpolation terms of degree >= dci are summed in plain FP32
    float fold_tol;        // truncation of the spreading weights' Chebyshev form within a bin
    float fold_df_tol;     // weights' Chebyshev terms above this need double-float moments
    double half_w;         // w / 2
    const double* ph;      // psi-hat pieces [ph_pieces][ph_deg + 1] in v in [-1, 1]
    const float2* ph2;     // the same as double-float
    double interp_const;   // sqrt(2/pi) * 4 / w^2
    float2 ic2;            // the same as double-float
    float2 ph_scale2;      // ph_scale as double-float
    int ph_pieces, ph_deg;
    int ph_comp;           // psi-hat degrees above this one are evaluated in plain FP32
    double ph_scale;       // pieces per unit of xi
    double ph_xmax;        // table covers xi in [0, ph_xmax]
    const double2* tw;     // e^{2 pi i k / 2^tw_log2}, k < 2^(tw_log2 - 1)
    const float4* tw2;     // the same as double-float (cos.h, cos.l, sin.h, sin.l)
    int tw_log2;
};

// ------------------------------------------------------------ device launches
// (each returns cudaGetLastError() of its launch and adds the number of
// kernels it launched to the library's launch counter)
void count_launches(int k);
cudaError_t launch_check_domain(const double* x, int64_t n, int* flag, cudaStream_t s);
cudaError_t radix_sort_f64(const double* in, int64_t n, double* out, int32_t* perm,
                           void* scratch, size_t scratch_bytes, cudaStream_t s,
                           const int64_t* seg_off = nullptr, int nseg = 1);
size_t radix_sort_scratch_bytes(int64_t n);

cudaError_t launch_staircase(const double* r, int64_t n, const double* w, int64_t m, double z,
                             int32_t* s_out, cudaStream_t s);
// Algorithm 1 on the device: lists out[0..ocap) local, out[ocap..2 ocap)
// asymptotic, out[2 ocap..3 ocap) direct; res = {counts, overflow}.  With
// grid_ctas > 1 (subdivide_grid_ctas(): one per SM where cooperative launches
// work, else 0) a cooperative launch of that many CTAs (scratch ctot[grid_ctas],
// gst[8]); otherwise, or if that launch is refused, one CTA.  The lists are the
// same either way.
constexpr int kSubGridMax = 1024;
int subdivide_grid_ctas();
cudaError_t launch_subdivide(const int32_t* stair, const double* r_s, const double* w_s, const ProbParams* probs,
                             int nprob, int64_t min_size,
                             int n_cand, SubBlk* qa, SubBlk* qb, int64_t qcap, SubBlk* out, int64_t ocap,
                             int64_t* res, int4* ctot, int64_t* gst, int grid_ctas, cudaStream_t s);
cudaError_t launch_block_bounds(const SubBlk* loc, const SubBlk* asy, const int64_t* res, const ProbParams* probs,
                                const double* r_s, const double* w_s, double* bl, double4* ba, cudaStream_t s);
cudaError_t launch_staircase_many(const double* r, const double* w, int64_t m, const ProbParams* probs,
                                  int nprob, int32_t* s_out, cudaStream_t s);
// per-call input scaling (k_det.cu): *mx = the bits of the largest |x_i|
// (gather scales the inputs by 2^-E of it, scatter the outputs back,
// input_exponent); Fx128 sums to FP64
cudaError_t launch_input_scale(const double* x, int64_t count, unsigned long long* mx, cudaStream_t s);
cudaError_t launch_fx_decode(const void* src, double* dst, int64_t count, const ProbParams* probs, cudaStream_t s);
// derivative plans (k_sort.cu): weighted gather into both problems' copies,
// the weighted input maximum, and the half difference scattered times y
cudaError_t launch_gather_deriv(const double* x, const int32_t* perm, const double* ws, int64_t nb, int stride,
                                int comp, const unsigned long long* mx, double* out, float2* out2, cudaStream_t s);
cudaError_t launch_absmax_weighted(const double* x, const int32_t* perm, const double* ws, int64_t nb, int comps,
                                   unsigned long long* mx, cudaStream_t s);
cudaError_t launch_scatter_deriv(const double* gs, const int32_t* perm, int64_t mb, int stride, int comp,
                                 const unsigned long long* mx, const double* y, double* out, cudaStream_t s);
cudaError_t launch_gather(const double* c, const int32_t* perm, int64_t n, int stride, int comp,
                          const unsigned long long* mx, double* out, float2* out2, cudaStream_t s);
cudaError_t launch_expand_tiles(const Seg* segs, const int32_t* prefix, int nseg, int total, Tile* out,
                                cudaStream_t s);
cudaError_t launch_scatter(const double* gs, const int32_t* perm, int64_t m, int stride, int comp,
                           const unsigned long long* mx, double* g, cudaStream_t s);

cudaError_t launch_local_moments(const ProbParams* probs, const LocalBlock* blks, const Tile* tiles,
                                 int ntiles, int lmax, const float2* r2, const float2* c2,
                                 double* mom, cudaStream_t s);
cudaError_t launch_local_moments2(const ProbParams* probs, const LocalBlock* blks, const Tile* tiles,
                                  int ntiles, int lmax, const float2* r2, const float2* c2, const float2* c2b,
                                  double* mom, double* momb, cudaStream_t s);
bool local_moments2_fits(int lmax);
cudaError_t launch_local_persistent(const ProbParams* probs, const LocalBlock* blks, const Tile* tmom, int n_tmom,
                                    const Tile* teval, int n_teval, const int32_t* mom_pre, int lmax, int ntop_max,
                                    int threads, const float2* r2, const float2* c2, const float2* c2b,
                                    const float2* w2, double* mom, double* momb, double* g_s, double* g_sb, int* q,
                                    int nloc, int* status, int wait_limit, int stall, cudaStream_t s);
int local_moment_threads(int lmax);
int local_eval_threads(int ntop_max);
// Mixed precision: k_local_eval with the recurrence and the sum in FP32.
// momb / g_sb (may be null): a second real component's moments and sums,
// evaluated with the same Bessel values.
cudaError_t launch_local_eval_f32(const ProbParams* probs, const LocalBlock* blks, const Tile* tiles,
                                  int ntiles, int ntop_max, int threads, const float2* w2, const double* mom,
                                  double* g_s, const double* momb, double* g_sb, cudaStream_t s);
cudaError_t launch_local_eval(const ProbParams* probs, const LocalBlock* blks, const Tile* tiles,
                              int ntiles, int ntop_max, bool column, int threads, const float2* w2,
                              const double* mom, double* g_s, const double* momb, double* g_sb,
                              cudaStream_t s);
// Mode of the direct kernel (0 double-float; 1 FP32 entries, FP64 sums; 2 FP32
// entries and sums) for tolerance eps and the tallest and widest direct blocks.
int direct_sum_mode(double eps, int max_rows, int max_cols);
cudaError_t launch_direct(const ProbParams* probs, const DirectBlock* blks, int nblk, int max_rows,
                          int max_area, int mode, const double* r_s, const double* w_s, const float2* r2,
                          const float2* w2, const double* c_s, const float2* c2, double* g_s,
                          const double* c_sb, const float2* c2b, double* g_sb, int det, cudaStream_t s);
// Vector groups: G <= kGroupMax real components applied together (their
// data at v times c_stride / mom_stride / g_stride from the first's).
// local_group_fits: the group moment kernel's outputs ((lmax + 1) G) fit its
// CTA, and both group kernels' shared memory stays within 200 KB.
constexpr int kGroupMax = NUHT_MAX_VEC_GROUP;
int local_group_fits(int lmax, int ntop_max, int eval_threads, int G);
cudaError_t launch_local_moments_group(const ProbParams* probs, const LocalBlock* blks, const Tile* tiles,
                                       int ntiles, int lmax, const float2* r2, const float2* c2,
                                       int64_t c_stride, int G, double* mom, int64_t mom_stride, cudaStream_t s);
cudaError_t launch_local_eval_group(const ProbParams* probs, const LocalBlock* blks, const Tile* tiles,
                                    int ntiles, int ntop_max, int threads, const float2* w2, const double* mom,
                                    int64_t mom_stride, int G, double* g_s, int64_t g_stride, cudaStream_t s);
cudaError_t launch_direct_group(const ProbParams* probs, const DirectBlock* blks, int nblk, int max_area,
                                int lowp, const double* r_s, const double* w_s, const float2* r2, const float2* w2,
                                const float2* c2, int64_t c_stride, int G, double* g_s, int64_t g_stride,
                                cudaStream_t s);
int local_adj_threads(int ntop_max);
// Adjoint local blocks for a group of G components (g_s + v g_stride, moments
// mom + v mom_stride, sums into c_s + v c_stride): moments (row tiles teval,
// threads from local_adj_group_threads) or evaluation (column tiles tmom).
int local_adj_group_threads(int ntop_max);
cudaError_t launch_local_adj_group(const ProbParams* probs, const LocalBlock* blks, const Tile* teval, int n_teval,
                                   const Tile* tmom, int n_tmom, int lmax, int ntop_max, int threads,
                                   const float2* w2, const float2* r2, const double* g_s, int64_t g_stride, int G,
                                   double* mom, int64_t mom_stride, double* c_s, int64_t c_stride, bool moments,
                                   cudaStream_t s);
// g_sb / momb (both null, or both set): a second real component's g and
// moments, summed with the same Bessel values.
cudaError_t launch_local_adj_moments(const ProbParams* probs, const LocalBlock* blks, const Tile* tiles,
                                     int ntiles, int ntop_max, int threads, const float2* w2,
                                     const double* g_s, double* mom, const double* g_sb, double* momb,
                                     cudaStream_t s);
cudaError_t launch_local_adj_eval(const ProbParams* probs, const LocalBlock* blks, const Tile* tiles,
                                  int ntiles, int lmax, const float2* r2, const double* mom, double* c_s,
                                  cudaStream_t s);
cudaError_t launch_direct_adj(const ProbParams* probs, const DirectBlock* blks, int nblk, int max_cols,
                              int max_area, int lowp, const double* r_s, const double* w_s, const float2* r2,
                              const float2* w2, const double* g_s, double* c_s, int det, cudaStream_t s);
// x[i] as double-float (hi, lo)
cudaError_t launch_split_f64(const double* x, int64_t n, float2* out, cudaStream_t s);
// Per spreading tile, the path of k_asy_spread (plan time; modes[ntiles]).
cudaError_t launch_spread_modes(const ProbParams* probs, const AsyBlock* blks, const Tile* tiles, int ntiles,
                                Tables tab, const double* r_s, int32_t* modes, cudaStream_t s);
// members: real components spread by one launch (coefficients c2 + v c_stride,
// grids grid_b + v gb_stride); 1 in the deterministic mode.
cudaError_t launch_asy_spread(const ProbParams* probs, const AsyBlock* blks, const Tile* tiles,
                              const int32_t* modes, int ntiles, int qmax, int nt, Tables tab, const double* r_s,
                              const float2* r2, const float2* c2, int64_t c_stride, int members,
                              double2* grid_b, int64_t gb_stride, int det, cudaStream_t s);
// members as in launch_asy_spread (inputs g_s + v g_stride, grids tgrid + v tg_stride)
cudaError_t launch_asy_adj_spread(const ProbParams* probs, const AsyBlock* blks, const Tile* tiles,
                                  int ntiles, int qmax, int nt, Tables tab, const double* w_s, const double* g_s,
                                  int64_t g_stride, int members, double2* tgrid, int64_t tg_stride,
                                  cudaStream_t s);
// members as in launch_asy_interp (modes bgrid + v bg_stride, sums into c_s + v c_stride)
cudaError_t launch_asy_adj_interp(const ProbParams* probs, const AsyBlock* blks, const Tile* tiles,
                                  int ntiles, int qmax, Tables tab, const double* r_s, const float4* bgrid,
                                  int64_t bg_stride, int members, double* c_s, int64_t c_stride, cudaStream_t s);
cudaError_t launch_asy_spread_f32(const ProbParams* probs, const AsyBlock* blks, const Tile* tiles,
                                  const int32_t* modes, int ntiles, int qmax, int nt, Tables tab,
                                  const double* r_s, const float2* r2, const float2* c2, int64_t c_stride,
                                  int members, double2* grid_b, int64_t gb_stride, cudaStream_t s);
cudaError_t launch_asy_interp_f32(const ProbParams* probs, const AsyBlock* blks, const Tile* tiles,
                                  int ntiles, int qmax, int nt, Tables tab, const double* w_s, const float2* w2,
                                  const float4* grid_q, int64_t gq_stride, int members, double* g_s,
                                  int64_t g_stride, cudaStream_t s);
// lowp: FP32 butterflies on the FP32 parts of the values (mixed precision).
// members: a batch of real components (grids src + v src_stride -> dst + v
// dst_stride) in one launch.
cudaError_t launch_asy_fft_small(const ProbParams* probs, const AsyBlock* blks, const Tile* items,
                                 int nitems, int max_nf2, Tables tab, const double2* src,
                                 float4* dst, cudaStream_t s, bool adj = false, bool lowp = false,
                                 int members = 1, int64_t src_stride = 0, int64_t dst_stride = 0);
// max_pts: the largest nf2 * Q among the blocks of the list (sizes the CTA).
cudaError_t launch_asy_fft_block(const ProbParams* probs, const AsyBlock* blks, const Tile* items,
                                 int nitems, int max_pts, Tables tab, const double2* src, float4* dst,
                                 cudaStream_t s, bool adj = false, bool lowp = false, int members = 1,
                                 int64_t src_stride = 0, int64_t dst_stride = 0);
cudaError_t launch_asy_fft_large(const ProbParams* probs, const AsyBlock* blks, const Tile* items_a,
                                 int nitems_a, const Tile* items_b, int nitems_b, Tables tab,
                                 const double2* src, float4* tmp, float4* dst,
                                 cudaStream_t s, bool adj = false, bool lowp = false);
// members: real components interpolated by one launch (FFT outputs grid_q + v
// gq_stride, sums into g_s + v g_stride).
cudaError_t launch_asy_interp(const ProbParams* probs, const AsyBlock* blks, const Tile* tiles,
                              int ntiles, int qmax, int nt, Tables tab, const double* w_s, const float2* w2,
                              const float4* grid_q, int64_t gq_stride, int members, double* g_s,
                              int64_t g_stride, cudaStream_t s);

}  // namespace nuht
