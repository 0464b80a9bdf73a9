// Algorithm 1 (Subdivide) with SplitIndices (Sec. 4.1) on the device.
//
// The host version (subdivide.cpp) walks a first-in first-out work list.
// Here one CTA processes that list level by level: every mixed block of a
// level is split at once (16 candidate rows read from the staircase), its
// four children are classified, and block-wide prefix sums give each child
// its place in the local / asymptotic / direct lists or in the next level.
// Children are placed in the order the sequential walk would append them
// (parents in list order, children upper-left, lower-right, upper-right,
// lower-left), so for one problem the lists equal the host's, entry for
// entry.  A batch's roots start together; the host orders the lists by
// problem afterwards (a stable reordering).
//
// The staircase stair[w_off + k] = max{j : omega_k r_j <= z} (problem-local
// column, or -1) is non-increasing in k, so a block is all local iff
// stair[k1] >= j1 and all asymptotic iff stair[k0] < j0.
#include <cooperative_groups.h>
#include <cstdint>

#include "nuht_internal.h"

namespace nuht {

// streaming multiprocessors of the current device, cached per device (k_det.cu)
int device_sm_count();

namespace {

constexpr int kSubThreads = 1024;
constexpr int kSubCandUnroll = 16;   // candidate rows loaded together (the default n_cand)
constexpr int kSubWarps = kSubThreads / 32;

// An asymptotic block too large for one FFT (X S > kAsyMaxXS) is queued like
// a mixed one, flagged in its problem index, and cut into quadrants; the host
// walk does the same in the same order.
constexpr int32_t kQuadFlag = 0x40000000;

__device__ __forceinline__ bool asy_too_big(const double* __restrict__ r, const double* __restrict__ w,
                                            const SubBlk& b)
{
    return 0.5 * (r[b.j1] - r[b.j0]) * 0.5 * (w[b.k1] - w[b.k0]) > kAsyMaxXS;
}

// 0 empty, 1 local, 2 asymptotic, 3 direct, 4 mixed (split further), 5
// asymptotic but too large (cut into quadrants)
__device__ __forceinline__ int classify(const int32_t* __restrict__ st, const SubBlk& b, int64_t min_size)
{
    if (b.k1 < b.k0 || b.j1 < b.j0) return 0;
    if (st[b.k1] >= b.j1) return 1;
    if (st[b.k0] < b.j0) return 2;
    if ((int64_t)(b.k1 - b.k0 + 1) * (int64_t)(b.j1 - b.j0 + 1) <= min_size) return 3;
    return 4;
}

// classify with the staircase values at the block's first and last rows given
__device__ __forceinline__ int classify_v(const SubBlk& b, int s0, int s1, int64_t min_size)
{
    if (b.k1 < b.k0 || b.j1 < b.j0) return 0;
    if (s1 >= b.j1) return 1;
    if (s0 < b.j0) return 2;
    if ((int64_t)(b.k1 - b.k0 + 1) * (int64_t)(b.j1 - b.j0 + 1) <= min_size) return 3;
    return 4;
}

// Exclusive block-wide prefix sum of a 64-bit value (four 16-bit counters
// packed; no carries since a chunk adds at most 4 x kSubThreads per field).
__device__ __forceinline__ uint64_t block_scan(uint64_t v, uint64_t* wsum, uint64_t* total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint64_t x = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint64_t s = wsum[lane];
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint64_t y = __shfl_up_sync(0xffffffffu, s, off);
            if (lane >= off) s += y;
        }
        wsum[lane] = s;
    }
    __syncthreads();
    const uint64_t before = (wid > 0 ? wsum[wid - 1] : 0) + x - v;
    *total = wsum[kSubWarps - 1];
    __syncthreads();
    return before;
}

struct SubState {
    int64_t nout[3];   // local, asymptotic, direct blocks written so far
    int64_t nnext;     // blocks of the next level written so far
    int ovf;
};

// Places up to four children per thread (classes cls[i], 0 = none) in
// order: class lists out[c * ocap ...] and the next level's queue.
__device__ __forceinline__ void emit(const SubBlk* ch, const int* cls, int nch, SubState& S, uint64_t* wsum,
                                     SubBlk* __restrict__ out, int64_t ocap, SubBlk* __restrict__ next,
                                     int64_t qcap)
{
    uint64_t cnt = 0;
    for (int i = 0; i < nch; ++i)
        if (cls[i] > 0) cnt += (uint64_t)1 << (16 * ((cls[i] < 4 ? cls[i] : 4) - 1));
    uint64_t total;
    const uint64_t off = block_scan(cnt, wsum, &total);
    int64_t pos[4];
    for (int c = 0; c < 3; ++c) pos[c] = S.nout[c] + (int64_t)((off >> (16 * c)) & 0xffff);
    pos[3] = S.nnext + (int64_t)(off >> 48);
    bool fits = S.ovf == 0;
    for (int c = 0; c < 3; ++c) fits = fits && S.nout[c] + (int64_t)((total >> (16 * c)) & 0xffff) <= ocap;
    fits = fits && S.nnext + (int64_t)(total >> 48) <= qcap;
    if (fits) {
        for (int i = 0; i < nch; ++i) {
            const int c = cls[i];
            if (c == 0) continue;
            if (c >= 4) {
                SubBlk q = ch[i];
                if (c == 5) q.prob |= kQuadFlag;
                next[pos[3]++] = q;
            } else {
                out[(c - 1) * ocap + pos[c - 1]++] = ch[i];
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (fits) {
            for (int c = 0; c < 3; ++c) S.nout[c] += (int64_t)((total >> (16 * c)) & 0xffff);
            S.nnext += (int64_t)(total >> 48);
        } else {
            S.ovf = 1;   // the counts stay at what was written (within the capacities)
        }
    }
    __syncthreads();
}

// The four children of mixed block qa[i] (SplitIndices at up to n_cand
// candidate rows), or the quadrants of a flagged asymptotic block, and their
// classes (0 none / empty, 1..3 a list, 4 the next level, 5 quadrants next);
// nothing for i >= na.
__device__ __forceinline__ void make_children(int64_t i, int64_t na, const SubBlk* qa,
                                              const int32_t* __restrict__ stair, const double* __restrict__ r_s,
                                              const double* __restrict__ w_s, const ProbParams* __restrict__ probs,
                                              int64_t min_size, int n_cand, SubBlk* ch, int* cls)
{
    if (i < na && (qa[i].prob & kQuadFlag)) {
        // an asymptotic block too large for one FFT: its quadrants
        SubBlk b = qa[i];
        b.prob &= ~kQuadFlag;
        const ProbParams& P = probs[b.prob];
        const int km = (b.k0 + b.k1) >> 1, jm = (b.j0 + b.j1) >> 1;
        ch[0] = SubBlk{b.k0, km, b.j0, jm, b.prob};
        ch[1] = SubBlk{km + 1, b.k1, jm + 1, b.j1, b.prob};
        ch[2] = SubBlk{b.k0, km, jm + 1, b.j1, b.prob};
        ch[3] = SubBlk{km + 1, b.k1, b.j0, jm, b.prob};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const bool ne = ch[c].k1 >= ch[c].k0 && ch[c].j1 >= ch[c].j0;
            cls[c] = ne ? (asy_too_big(r_s + P.r_off, w_s + P.w_off, ch[c]) ? 5 : 2) : 0;
        }
    } else if (i < na) {
        const SubBlk b = qa[i];
        const int32_t* st = stair + probs[b.prob].w_off;
        // SplitIndices: the candidate row minimising the mixed area,
        // its column the last local one (ties keep the first)
        const int rows = b.k1 - b.k0 + 1;
        const int nc = rows <= n_cand ? rows : n_cand;
        int64_t best = -1;
        int bk = b.k0, bj = b.j0 - 1;
        auto cand_row = [&](int c) {
            return rows <= n_cand ? b.k0 + c : b.k0 + (int)(((int64_t)c * (b.k1 - b.k0)) / (n_cand - 1));
        };
        auto consider = [&](int k, int j) {
            if (j > b.j1) j = b.j1;
            if (j < b.j0) j = b.j0 - 1;
            const int64_t area = (int64_t)(k - b.k0 + 1) * (b.j1 - j) + (int64_t)(b.k1 - k) * (j - b.j0 + 1);
            if (best < 0 || area < best) {
                best = area;
                bk = k;
                bj = j;
            }
        };
        if (nc <= kSubCandUnroll) {
            // all candidate loads in flight at once
            int jv[kSubCandUnroll];
#pragma unroll
            for (int c = 0; c < kSubCandUnroll; ++c) jv[c] = c < nc ? st[cand_row(c)] : 0;
#pragma unroll
            for (int c = 0; c < kSubCandUnroll; ++c)
                if (c < nc) consider(cand_row(c), jv[c]);
        } else {
            for (int c = 0; c < nc; ++c) {
                const int k = cand_row(c);
                consider(k, st[k]);
            }
        }
        ch[0] = SubBlk{b.k0, bk, b.j0, bj, b.prob};           // upper left: local
        ch[1] = SubBlk{bk + 1, b.k1, bj + 1, b.j1, b.prob};   // lower right: asymptotic
        ch[2] = SubBlk{b.k0, bk, bj + 1, b.j1, b.prob};       // upper right: mixed
        ch[3] = SubBlk{bk + 1, b.k1, b.j0, bj, b.prob};       // lower left: mixed
        // the children's end rows, loaded together
        int sk1[4], sk0[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const bool ne = ch[c].k1 >= ch[c].k0 && ch[c].j1 >= ch[c].j0;
            sk1[c] = ne ? st[ch[c].k1] : 0;
            sk0[c] = ne ? st[ch[c].k0] : 0;
        }
        const ProbParams& P = probs[b.prob];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            cls[c] = classify_v(ch[c], sk0[c], sk1[c], min_size);
            if (cls[c] == 2 && asy_too_big(r_s + P.r_off, w_s + P.w_off, ch[c])) cls[c] = 5;
        }
    }
}

__global__ void __launch_bounds__(kSubThreads) k_subdivide(
    const int32_t* __restrict__ stair, const double* __restrict__ r_s, const double* __restrict__ w_s,
    const ProbParams* __restrict__ probs, int nprob, int64_t min_size,
    int n_cand, SubBlk* qa, SubBlk* qb, int64_t qcap, SubBlk* __restrict__ out, int64_t ocap,
    int64_t* __restrict__ res)
{
    __shared__ uint64_t wsum[kSubWarps];
    __shared__ SubState S;
    if (threadIdx.x == 0) {
        S.nout[0] = S.nout[1] = S.nout[2] = 0;
        S.nnext = 0;
        S.ovf = 0;
    }
    __syncthreads();
    // the roots, one per problem
    for (int base = 0; base < nprob; base += kSubThreads) {
        const int p = base + threadIdx.x;
        SubBlk ch{0, -1, 0, -1, 0};
        int cls = 0;
        if (p < nprob) {
            const ProbParams& P = probs[p];
            ch = SubBlk{0, (int32_t)P.m - 1, 0, (int32_t)P.n - 1, p};
            cls = classify(stair + P.w_off, ch, min_size);
            if (cls == 2 && asy_too_big(r_s + P.r_off, w_s + P.w_off, ch)) cls = 5;
        }
        emit(&ch, &cls, 1, S, wsum, out, ocap, qa, qcap);
    }
    int64_t na = S.nnext;
    while (na > 0 && S.ovf == 0) {
        __syncthreads();   // every thread has read S.nnext and S.ovf
        if (threadIdx.x == 0) S.nnext = 0;
        __syncthreads();
        for (int64_t base = 0; base < na; base += kSubThreads) {
            const int64_t i = base + threadIdx.x;
            SubBlk ch[4];
            int cls[4] = {0, 0, 0, 0};
            make_children(i, na, qa, stair, r_s, w_s, probs, min_size, n_cand, ch, cls);
            emit(ch, cls, 4, S, wsum, out, ocap, qb, qcap);
        }
        na = S.nnext;
        SubBlk* tmp = qa;
        qa = qb;
        qb = tmp;
    }
    if (threadIdx.x == 0) {
        res[0] = S.nout[0];
        res[1] = S.nout[1];
        res[2] = S.nout[2];
        res[3] = S.ovf;
    }
}

// Multi-CTA form of k_subdivide (cooperative launch).  CTA 0 walks the first
// levels alone, as k_subdivide, while a level holds at most kSubSolo blocks;
// from the first larger level on, every CTA takes consecutive chunks of
// kSubThreads blocks of a level.  After its block-wide scan a CTA publishes
// its four counts (ctot), and after a grid-wide barrier each CTA forms its
// chunk's offsets from the counts of the chunks before it: the offsets of the
// one-CTA walk, so the lists are the same entry for entry.  Every CTA keeps
// the same copy of the list counts (SubState), so all take the same number of
// barriers.  gst carries CTA 0's state to the others.
constexpr int64_t kSubSolo = 2 * kSubThreads;

__global__ void __launch_bounds__(kSubThreads) k_subdivide_grid(
    const int32_t* __restrict__ stair, const double* __restrict__ r_s, const double* __restrict__ w_s,
    const ProbParams* __restrict__ probs, int nprob, int64_t min_size,
    int n_cand, SubBlk* qa, SubBlk* qb, int64_t qcap, SubBlk* __restrict__ out, int64_t ocap,
    int64_t* __restrict__ res, int4* ctot, int64_t* gst)
{
    namespace cg = cooperative_groups;
    cg::grid_group grid = cg::this_grid();
    __shared__ uint64_t wsum[kSubWarps];
    __shared__ SubState S;
    __shared__ int64_t cpre[4], ctall[4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (blockIdx.x == 0) {
        if (threadIdx.x == 0) {
            S.nout[0] = S.nout[1] = S.nout[2] = 0;
            S.nnext = 0;
            S.ovf = 0;
        }
        __syncthreads();
        for (int base = 0; base < nprob; base += kSubThreads) {
            const int p = base + threadIdx.x;
            SubBlk ch{0, -1, 0, -1, 0};
            int cls = 0;
            if (p < nprob) {
                const ProbParams& P = probs[p];
                ch = SubBlk{0, (int32_t)P.m - 1, 0, (int32_t)P.n - 1, p};
                cls = classify(stair + P.w_off, ch, min_size);
                if (cls == 2 && asy_too_big(r_s + P.r_off, w_s + P.w_off, ch)) cls = 5;
            }
            emit(&ch, &cls, 1, S, wsum, out, ocap, qa, qcap);
        }
        int64_t na = S.nnext;
        int swapped = 0;
        while (na > 0 && na <= kSubSolo && S.ovf == 0) {
            __syncthreads();   // every thread has read S.nnext and S.ovf
            if (threadIdx.x == 0) S.nnext = 0;
            __syncthreads();
            for (int64_t base = 0; base < na; base += kSubThreads) {
                const int64_t i = base + threadIdx.x;
                SubBlk ch[4];
                int cls[4] = {0, 0, 0, 0};
                make_children(i, na, qa, stair, r_s, w_s, probs, min_size, n_cand, ch, cls);
                emit(ch, cls, 4, S, wsum, out, ocap, qb, qcap);
            }
            na = S.nnext;
            SubBlk* tmp = qa;
            qa = qb;
            qb = tmp;
            swapped ^= 1;
        }
        if (threadIdx.x == 0) {
            gst[0] = S.nout[0];
            gst[1] = S.nout[1];
            gst[2] = S.nout[2];
            gst[3] = na;
            gst[4] = S.ovf;
            gst[5] = swapped;
        }
    }
    grid.sync();
    if (threadIdx.x == 0) {
        S.nout[0] = gst[0];
        S.nout[1] = gst[1];
        S.nout[2] = gst[2];
        S.nnext = gst[3];
        S.ovf = (int)gst[4];
    }
    __syncthreads();
    if (blockIdx.x != 0 && gst[5]) {
        // the pending level is in the queue CTA 0 last wrote (CTA 0's own
        // pointers were swapped by its walk already)
        SubBlk* tmp = qa;
        qa = qb;
        qb = tmp;
    }
    int64_t na = S.nnext;
    const int64_t per_round = (int64_t)gridDim.x * kSubThreads;
    while (na > 0 && S.ovf == 0) {
        __syncthreads();   // every thread has read S.nnext and S.ovf
        if (threadIdx.x == 0) S.nnext = 0;
        __syncthreads();
        for (int64_t r0 = 0; r0 < na; r0 += per_round) {
            const int64_t i = r0 + (int64_t)blockIdx.x * kSubThreads + threadIdx.x;
            SubBlk ch[4];
            int cls[4] = {0, 0, 0, 0};
            make_children(i, na, qa, stair, r_s, w_s, probs, min_size, n_cand, ch, cls);
            uint64_t cnt = 0;
            for (int c = 0; c < 4; ++c)
                if (cls[c] > 0) cnt += (uint64_t)1 << (16 * ((cls[c] < 4 ? cls[c] : 4) - 1));
            uint64_t total;
            const uint64_t off = block_scan(cnt, wsum, &total);
            if (threadIdx.x == 0)
                ctot[blockIdx.x] = make_int4((int)(total & 0xffff), (int)((total >> 16) & 0xffff),
                                             (int)((total >> 32) & 0xffff), (int)(total >> 48));
            grid.sync();
            if (warp == 0) {
                // counts of the chunks before this CTA's, and of the round
                int64_t a[4] = {0, 0, 0, 0}, tt[4] = {0, 0, 0, 0};
                for (int b = lane; b < (int)gridDim.x; b += 32) {
                    const int4 c = ctot[b];
                    const int64_t v[4] = {c.x, c.y, c.z, c.w};
                    for (int f = 0; f < 4; ++f) {
                        tt[f] += v[f];
                        if (b < (int)blockIdx.x) a[f] += v[f];
                    }
                }
                for (int f = 0; f < 4; ++f) {
                    for (int o = 16; o > 0; o >>= 1) {
                        a[f] += __shfl_xor_sync(0xffffffffu, a[f], o);
                        tt[f] += __shfl_xor_sync(0xffffffffu, tt[f], o);
                    }
                    if (lane == 0) {
                        cpre[f] = a[f];
                        ctall[f] = tt[f];
                    }
                }
            }
            __syncthreads();
            bool fits = S.ovf == 0;
            for (int c = 0; c < 3; ++c) fits = fits && S.nout[c] + ctall[c] <= ocap;
            fits = fits && S.nnext + ctall[3] <= qcap;
            if (fits) {
                int64_t pos[4];
                for (int c = 0; c < 3; ++c) pos[c] = S.nout[c] + cpre[c] + (int64_t)((off >> (16 * c)) & 0xffff);
                pos[3] = S.nnext + cpre[3] + (int64_t)(off >> 48);
                for (int c = 0; c < 4; ++c) {
                    const int k = cls[c];
                    if (k == 0) continue;
                    if (k >= 4) {
                        SubBlk q = ch[c];
                        if (k == 5) q.prob |= kQuadFlag;
                        qb[pos[3]++] = q;
                    } else {
                        out[(k - 1) * ocap + pos[k - 1]++] = ch[c];
                    }
                }
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                if (fits) {
                    for (int c = 0; c < 3; ++c) S.nout[c] += ctall[c];
                    S.nnext += ctall[3];
                } else {
                    S.ovf = 1;
                }
            }
            grid.sync();   // ctot is rewritten by the next round; the next level reads this one's queue
        }
        na = S.nnext;
        SubBlk* tmp = qa;
        qa = qb;
        qb = tmp;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        res[0] = S.nout[0];
        res[1] = S.nout[1];
        res[2] = S.nout[2];
        res[3] = S.ovf;
    }
}

// Sorted values at the block edges: local blocks R = r_{j1}; asymptotic
// blocks (r_{j0}, r_{j1}, omega_{k0}, omega_{k1}).  Counts from res (device).
__global__ void k_block_bounds(const SubBlk* __restrict__ loc, const SubBlk* __restrict__ asy,
                               const int64_t* __restrict__ res, const ProbParams* __restrict__ probs,
                               const double* __restrict__ r_s, const double* __restrict__ w_s,
                               double* __restrict__ bl, double4* __restrict__ ba)
{
    const int64_t nl = res[0], na = res[1];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nl + na;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (i < nl) {
            const SubBlk b = loc[i];
            bl[i] = r_s[probs[b.prob].r_off + b.j1];
        } else {
            const SubBlk b = asy[i - nl];
            const ProbParams& P = probs[b.prob];
            ba[i - nl] = make_double4(r_s[P.r_off + b.j0], r_s[P.r_off + b.j1], w_s[P.w_off + b.k0],
                                      w_s[P.w_off + b.k1]);
        }
    }
}

}  // namespace

int subdivide_grid_ctas()
{
    int dev = 0, sms = 0, coop = 0, nb = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_subdivide_grid, kSubThreads, 0) != cudaSuccess ||
        nb < 1)
        return 0;
    return sms < kSubGridMax ? sms : kSubGridMax;
}

cudaError_t launch_subdivide(const int32_t* stair, const double* r_s, const double* w_s, const ProbParams* probs,
                             int nprob, int64_t min_size,
                             int n_cand, SubBlk* qa, SubBlk* qb, int64_t qcap, SubBlk* out, int64_t ocap,
                             int64_t* res, int4* ctot, int64_t* gst, int grid_ctas, cudaStream_t s)
{
    if (grid_ctas > 1 && grid_ctas <= kSubGridMax && ctot && gst) {
        void* args[] = {(void*)&stair, (void*)&r_s, (void*)&w_s, (void*)&probs, (void*)&nprob, (void*)&min_size,
                        (void*)&n_cand, (void*)&qa, (void*)&qb, (void*)&qcap, (void*)&out, (void*)&ocap,
                        (void*)&res, (void*)&ctot, (void*)&gst};
        const cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_subdivide_grid, dim3(grid_ctas),
                                                          dim3(kSubThreads), args, 0, s);
        if (e == cudaSuccess) {
            count_launches(1);
            return cudaSuccess;
        }
        (void)cudaGetLastError();   // not launched: the one-CTA walk below
    }
    k_subdivide<<<1, kSubThreads, 0, s>>>(stair, r_s, w_s, probs, nprob, min_size, n_cand, qa, qb, qcap, out, ocap,
                                          res);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_block_bounds(const SubBlk* loc, const SubBlk* asy, const int64_t* res, const ProbParams* probs,
                                const double* r_s, const double* w_s, double* bl, double4* ba, cudaStream_t s)
{
    k_block_bounds<<<device_sm_count() * 8, 256, 0, s>>>(loc, asy, res, probs, r_s, w_s, bl, ba);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace nuht
