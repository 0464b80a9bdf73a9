// Plan-time device kernels: input domain check, LSD radix sort of FP64 keys
// with their original indices, and the execute-time gather / scatter between
// user order and sorted order.
//
// The subdivision of Algorithm 1 and the complexity theorem of Sec. 4.2 take
// the points and frequencies sorted ascending; the inputs are unsorted, so the
// plan sorts them once and keeps the permutations.
//
// Keys are non-negative doubles (checked first), whose IEEE bit patterns
// compare like unsigned integers, so an 8-pass, 8-bit LSD radix sort on the
// raw 64-bit patterns sorts them.  Each pass: per-tile digit histogram,
// one exclusive scan over (digit, tile), then a stable scatter in which each
// warp ranks its run of the tile (warp match + per-warp digit counts) and one
// prefix over the warps places the runs, so equal keys keep their input order.
#include <cstdint>

#include "nuht_internal.h"

namespace nuht {

// streaming multiprocessors of the current device, cached per device (k_det.cu)
int device_sm_count();

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 4;                       // elements per thread per tile
constexpr int kSortTile = kSortThreads * kSortItems; // 1024: ~4 CTAs per SM at n = 1e6 (4096 left the scatter passes latency-bound)
constexpr int kRadix = 256;
static_assert(kSortThreads == kRadix, "the scatter kernel scans one digit total per thread");

__global__ void k_check_domain(const double* __restrict__ x, int64_t n, int* flag)
{
    int bad = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double v = x[i];
        // rejects negatives, NaN and +-inf; -0.0 is accepted
        if (!(v >= 0.0) || !(v <= 1.7976931348623157e308)) bad = 1;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

// keys: bit patterns (with -0.0 folded onto +0.0), values: 0..n-1
__global__ void k_sort_init(const double* __restrict__ in, int64_t n, uint64_t* __restrict__ keys,
                            int32_t* __restrict__ vals)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double v = in[i];
        if (v == 0.0) v = 0.0;  // -0.0 -> +0.0
        keys[i] = (uint64_t)__double_as_longlong(v);
        vals[i] = (int32_t)i;
    }
}

__global__ void k_sort_hist(const uint64_t* __restrict__ keys, int64_t n, int shift, int ntiles,
                            uint32_t* __restrict__ hist)
{
    __shared__ uint32_t h[kRadix];
    for (int i = threadIdx.x; i < kRadix; i += blockDim.x) h[i] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int it = 0; it < kSortItems; ++it) {
        int64_t i = base + it * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 0xFF], 1u);
    }
    __syncthreads();
    // digit-major layout: hist[d * ntiles + tile]
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x)
        hist[(int64_t)d * ntiles + blockIdx.x] = h[d];
}

// One CTA per digit: exclusive scan of that digit's per-tile counts (in place,
// hist[d * ntiles + tile]) and the digit's total in tot[d].
__global__ void k_sort_rowscan(uint32_t* __restrict__ hist, int ntiles, uint32_t* __restrict__ tot)
{
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* a = hist + (int64_t)blockIdx.x * ntiles;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < ntiles; base += 1024) {
        const int i = base + threadIdx.x;
        const uint32_t v = (i < ntiles) ? a[i] : 0u;
        uint32_t x = v;
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, x, off);
            if (lane >= off) x += t;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            uint32_t y = wsum[lane];
            for (int off = 1; off < 32; off <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, y, off);
                if (lane >= off) y += t;
            }
            wsum[lane] = y;
        }
        __syncthreads();
        const uint32_t incl = x + (warp > 0 ? wsum[warp - 1] : 0u);
        if (i < ntiles) a[i] = carry + incl - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) tot[blockIdx.x] = carry;
}

// Stable scatter of one pass.  Warp w of a tile owns its 128 consecutive
// elements, in rounds of 32, so (warp, round, lane) is the input order: each
// warp ranks its elements among equal digits with a per-warp digit count in
// shared memory (warp-synchronous, no CTA barrier per round), then one
// exclusive prefix over the warps per digit places every warp's run after
// the earlier warps' in the tile's part of each digit bucket.
__global__ void __launch_bounds__(kSortThreads) k_sort_scatter(
    const uint64_t* __restrict__ kin, const int32_t* __restrict__ vin, int64_t n, int shift, int ntiles,
    const uint32_t* __restrict__ offs, const uint32_t* __restrict__ tot, uint64_t* __restrict__ kout,
    int32_t* __restrict__ vout)
{
    constexpr int kWarps = kSortThreads / 32;
    __shared__ uint32_t wcnt[kWarps][kRadix];   // per-warp digit counts, then the warps' starts
    __shared__ uint32_t wsum[kWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // start of digit threadIdx.x's bucket for this tile: exclusive scan of the
    // 256 digit totals plus this tile's offset inside the bucket
    uint32_t mybase;
    {
        const uint32_t v = tot[threadIdx.x];     // blockDim.x == kRadix
        uint32_t x = v;
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, x, off);
            if (lane >= off) x += t;
        }
        if (lane == 31) wsum[warp] = x;
        for (int i = threadIdx.x; i < kWarps * kRadix; i += blockDim.x) (&wcnt[0][0])[i] = 0;
        __syncthreads();
        uint32_t pre = 0;
        for (int w = 0; w < warp; ++w) pre += wsum[w];
        mybase = pre + x - v + offs[(int64_t)threadIdx.x * ntiles + blockIdx.x];
    }
    const unsigned lt = (1u << lane) - 1u;
    const int64_t wbase = (int64_t)blockIdx.x * kSortTile + (int64_t)warp * (32 * kSortItems);
    uint64_t key[kSortItems];
    int32_t val[kSortItems];
    unsigned dig[kSortItems];
    uint32_t rk[kSortItems];
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        const int64_t i = wbase + it * 32 + lane;
        const bool valid = i < n;
        key[it] = valid ? kin[i] : 0ull;
        val[it] = valid ? vin[i] : 0;
        const unsigned d = valid ? (unsigned)((key[it] >> shift) & 0xFF) : 0x100u;
        dig[it] = d;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const uint32_t prior = valid ? wcnt[warp][d] : 0u;
        __syncwarp();
        if (valid && (peers & lt) == 0) wcnt[warp][d] = prior + __popc(peers);
        __syncwarp();
        rk[it] = prior + __popc(peers & lt);
    }
    __syncthreads();
    {
        const int d = threadIdx.x;
        uint32_t run = mybase;
        for (int w = 0; w < kWarps; ++w) {
            const uint32_t t = wcnt[w][d];
            wcnt[w][d] = run;
            run += t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        if (dig[it] < 0x100u) {
            const uint32_t pos = wcnt[warp][dig[it]] + rk[it];
            kout[pos] = key[it];
            vout[pos] = val[it];
        }
    }
}

__global__ void k_sort_finish(const uint64_t* __restrict__ keys, int64_t n, double* __restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = __longlong_as_double((long long)keys[i]);
}

__global__ void k_gather(const double* __restrict__ c, const int32_t* __restrict__ perm, int64_t n,
                         int stride, int comp, const unsigned long long* __restrict__ mx,
                         double* __restrict__ out, float2* __restrict__ out2)
{
    const int e = -input_exponent(*mx);   // inputs scaled by 2^-E (exact)
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double v = scalbn(c[(int64_t)perm[i] * stride + comp], e);
        out[i] = v;
        if (out2) {
            const float h = (float)v;
            out2[i] = make_float2(h, (float)(v - (double)h));
        }
    }
}

// x as double-float pairs (hi = nearest float, lo = nearest float to the rest)
__global__ void k_split_f64(const double* __restrict__ x, int64_t n, float2* __restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double v = x[i];
        const float h = (float)v;
        out[i] = make_float2(h, (float)(v - (double)h));
    }
}

__global__ void k_scatter(const double* __restrict__ gs, const int32_t* __restrict__ perm, int64_t m,
                          int stride, int comp, const unsigned long long* __restrict__ mx,
                          double* __restrict__ g)
{
    const int e = input_exponent(*mx);   // back to the input's scale (exact)
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x)
        g[(int64_t)perm[i] * stride + comp] = scalbn(gs[i], e);
}

// Derivative plans (two problems over two copies of the sorted arrays): the
// input x (user order) weighted by the sorted values ws (r for the omega
// gradient, omega for the r gradient), scaled by 2^-E, into both copies.
__global__ void k_gather_deriv(const double* __restrict__ x, const int32_t* __restrict__ perm,
                               const double* __restrict__ ws, int64_t nb, int stride, int comp,
                               const unsigned long long* __restrict__ mx, double* __restrict__ out,
                               float2* __restrict__ out2)
{
    const int e = -input_exponent(*mx);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 2 * nb;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i0 = i < nb ? i : i - nb;
        const double v = scalbn(x[(int64_t)perm[i0] * stride + comp] * ws[i0], e);
        out[i] = v;
        if (out2) {
            const float h = (float)v;
            out2[i] = make_float2(h, (float)(v - (double)h));
        }
    }
}

// The largest |x_u ws_i| (u = perm[i], every vector), as bits (k_absmax_bits).
__global__ void k_absmax_weighted(const double* __restrict__ x, const int32_t* __restrict__ perm,
                                  const double* __restrict__ ws, int64_t nb, int comps,
                                  unsigned long long* __restrict__ mx)
{
    unsigned long long m = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nb * comps;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i0 = i / comps, v = i - i0 * comps;
        const double a = x[(int64_t)perm[i0] * comps + v] * ws[i0];
        const unsigned long long b = (unsigned long long)__double_as_longlong(a) & 0x7fffffffffffffffull;
        m = b > m ? b : m;
    }
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, m, off);
        m = o > m ? o : m;
    }
    if ((threadIdx.x & 31) == 0 && m) atomicMax(mx, m);
}

// out[u] (+)= y_u (gs[k] + gs[mb + k]) / 2 back at the input's scale, u = perm[k]:
// the two problems' sums (orders nu - 1 and nu + 1, the second negated) give
// J_nu' = (J_{nu-1} - J_{nu+1}) / 2 (DLMF 10.6.1); vectors after the first add on.
__global__ void k_scatter_deriv(const double* __restrict__ gs, const int32_t* __restrict__ perm, int64_t mb,
                                int stride, int comp, const unsigned long long* __restrict__ mx,
                                const double* __restrict__ y, double* __restrict__ out)
{
    const int e = input_exponent(*mx) - 1;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < mb;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t u = perm[k];
        const double v = scalbn(gs[k] + gs[mb + k], e) * y[u * stride + comp];
        out[u] = comp == 0 ? v : out[u] + v;
    }
}

// First j in [lo, hi) with wk * r_j > z (hi if none); r ascending.
__device__ __forceinline__ int64_t first_above(const double* __restrict__ r, int64_t lo, int64_t hi, double wk,
                                               double z)
{
    while (lo < hi) {
        const int64_t mid = lo + ((hi - lo) >> 1);
        if (wk * r[mid] <= z) lo = mid + 1; else hi = mid;
    }
    return lo;
}

constexpr int kStairThreads = 256;
constexpr int kStairRows = 4;   // rows per thread

// s[k] = max{j : omega_k * r_j <= z} (or -1): the boundary of the local region
// in row k of the sorted matrix.  f(k) = s[k] + 1 is non-increasing in k (the
// FP64 product is monotone in both factors), so each CTA searches its first
// and last rows over all of r and its other rows only between those two
// bounds: one full search of latency per CTA instead of one per row.
__global__ void __launch_bounds__(kStairThreads) k_staircase(const double* __restrict__ r, int64_t n,
                                                             const double* __restrict__ w, int64_t m, double z,
                                                             int32_t* __restrict__ s)
{
    __shared__ int64_t fb[2];
    const int64_t span = (int64_t)kStairThreads * kStairRows;
    for (int64_t base = (int64_t)blockIdx.x * span; base < m; base += (int64_t)gridDim.x * span) {
        const int64_t last = (base + span < m ? base + span : m) - 1;
        if (threadIdx.x < 2) fb[threadIdx.x] = first_above(r, 0, n, w[threadIdx.x == 0 ? base : last], z);
        __syncthreads();
        const int64_t hi = fb[0], lo = fb[1];   // f(last) <= f(k) <= f(base)
#pragma unroll
        for (int i = 0; i < kStairRows; ++i) {
            const int64_t k = base + threadIdx.x + (int64_t)i * kStairThreads;
            if (k <= last) s[k] = (int32_t)(first_above(r, lo, hi, w[k], z) - 1);
        }
        __syncthreads();   // fb is rewritten by the next range
    }
}

// Tile i of a list: segment b with prefix[b] <= i < prefix[b + 1] (binary
// search), then its start and count inside the segment's index range.
__global__ void k_expand_tiles(const Seg* __restrict__ segs, const int32_t* __restrict__ prefix, int nseg,
                               int total, Tile* __restrict__ out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        int lo = 0, hi = nseg;   // last b with prefix[b] <= i
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (prefix[mid] <= i) lo = mid; else hi = mid;
        }
        const Seg sg = segs[lo];
        const int64_t start = sg.first + (int64_t)(i - prefix[lo]) * sg.len;
        const int64_t rem = sg.last - start + 1;
        out[i] = Tile{sg.blk, (int32_t)(rem < sg.len ? rem : sg.len), start};
    }
}

inline int grid_for(int64_t n, int threads)
{
    int64_t b = (n + threads - 1) / threads;
    const int64_t cap = (int64_t)device_sm_count() * 32;
    if (b > cap) b = cap;
    return b < 1 ? 1 : (int)b;
}

inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

cudaError_t launch_check_domain(const double* x, int64_t n, int* flag, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_check_domain<<<grid_for(n, 256), 256, 0, s>>>(x, n, flag);
    count_launches(1);
    return cudaGetLastError();
}

size_t radix_sort_scratch_bytes(int64_t n)
{
    int64_t ntiles = (n + kSortTile - 1) / kSortTile;
    return 2 * align256(sizeof(uint64_t) * (size_t)n) + align256(sizeof(int32_t) * (size_t)n) +
           align256(sizeof(uint32_t) * (size_t)kRadix * (size_t)(ntiles > 0 ? ntiles : 1)) +
           align256(sizeof(uint32_t) * (size_t)kRadix);
}

// seg[i] = segment of the element at input index perm[i] (offsets off[0..nseg]),
// as a radix key.
__global__ void k_seg_keys(const int32_t* __restrict__ perm, int64_t n, const int64_t* __restrict__ off,
                           int nseg, uint64_t* __restrict__ keys)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = perm[i];
        int lo = 0, hi = nseg;   // last segment with off[seg] <= x
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (off[mid] <= x) lo = mid; else hi = mid;
        }
        keys[i] = (uint64_t)lo;
    }
}

__global__ void k_gather_keys(const double* __restrict__ in, const int32_t* __restrict__ perm, int64_t n,
                              double* __restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double v = in[perm[i]];
        out[i] = (v == 0.0) ? 0.0 : v;
    }
}

// Sorts in[0..n) ascending into out, perm[i] = input index of out[i].  With
// nseg > 1 segments (device offsets off[0..nseg], nseg <= 65536) each segment
// is sorted on its own: the value passes are followed by two stable passes on
// the segment number, so the output keeps the segments in order.
cudaError_t radix_sort_f64(const double* in, int64_t n, double* out, int32_t* perm, void* scratch,
                           size_t scratch_bytes, cudaStream_t s, const int64_t* off, int nseg)
{
    if (n <= 0) return cudaSuccess;
    if (scratch_bytes < radix_sort_scratch_bytes(n)) return cudaErrorInvalidValue;
    int ntiles = (int)((n + kSortTile - 1) / kSortTile);
    char* p = (char*)scratch;
    uint64_t* k0 = (uint64_t*)p; p += align256(sizeof(uint64_t) * (size_t)n);
    uint64_t* k1 = (uint64_t*)p; p += align256(sizeof(uint64_t) * (size_t)n);
    int32_t* v1 = (int32_t*)p; p += align256(sizeof(int32_t) * (size_t)n);
    uint32_t* hist = (uint32_t*)p; p += align256(sizeof(uint32_t) * (size_t)kRadix * (size_t)ntiles);
    uint32_t* tot = (uint32_t*)p;
    int32_t* v0 = perm;   // ping-pong between perm and v1; 8 passes end in perm
    k_sort_init<<<grid_for(n, 256), 256, 0, s>>>(in, n, k0, v0);
    uint64_t* ka = k0; uint64_t* kb = k1;
    int32_t* va = v0; int32_t* vb = v1;
    for (int pass = 0; pass < 8; ++pass) {
        int shift = 8 * pass;
        k_sort_hist<<<ntiles, kSortThreads, 0, s>>>(ka, n, shift, ntiles, hist);
        k_sort_rowscan<<<kRadix, 1024, 0, s>>>(hist, ntiles, tot);
        k_sort_scatter<<<ntiles, kSortThreads, 0, s>>>(ka, va, n, shift, ntiles, hist, tot, kb, vb);
        uint64_t* tk = ka; ka = kb; kb = tk;
        int32_t* tv = va; va = vb; vb = tv;
    }
    // after an even number of passes the data is back in (k0, perm)
    if (nseg <= 1) {
        k_sort_finish<<<grid_for(n, 256), 256, 0, s>>>(ka, n, out);
        count_launches(2 + 8 * 3);
        return cudaGetLastError();
    }
    k_seg_keys<<<grid_for(n, 256), 256, 0, s>>>(perm, n, off, nseg, ka);
    for (int pass = 0; pass < 2; ++pass) {
        const int shift = 8 * pass;
        k_sort_hist<<<ntiles, kSortThreads, 0, s>>>(ka, n, shift, ntiles, hist);
        k_sort_rowscan<<<kRadix, 1024, 0, s>>>(hist, ntiles, tot);
        k_sort_scatter<<<ntiles, kSortThreads, 0, s>>>(ka, va, n, shift, ntiles, hist, tot, kb, vb);
        uint64_t* tk = ka; ka = kb; kb = tk;
        int32_t* tv = va; va = vb; vb = tv;
    }
    k_gather_keys<<<grid_for(n, 256), 256, 0, s>>>(in, perm, n, out);
    count_launches(1 + 10 * 3 + 2);
    return cudaGetLastError();
}

// Staircase of every row of a batch: row k belongs to the problem p with
// w_off <= k < w_off + m (binary search); the search runs over that problem's
// points and the result is a column index local to the problem.
__global__ void k_staircase_many(const double* __restrict__ r, const double* __restrict__ w, int64_t m,
                                 const ProbParams* __restrict__ probs, int nprob, int32_t* __restrict__ s)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m;
         k += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = nprob;   // last problem with w_off <= k
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (probs[mid].w_off <= k) lo = mid; else hi = mid;
        }
        const ProbParams& P = probs[lo];
        s[k] = (int32_t)(first_above(r + P.r_off, 0, P.n, w[k], P.z) - 1);
    }
}

cudaError_t launch_staircase(const double* r, int64_t n, const double* w, int64_t m, double z,
                             int32_t* s_out, cudaStream_t s)
{
    if (m <= 0) return cudaSuccess;
    k_staircase<<<grid_for(m, kStairThreads * kStairRows), kStairThreads, 0, s>>>(r, n, w, m, z, s_out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_staircase_many(const double* r, const double* w, int64_t m, const ProbParams* probs,
                                  int nprob, int32_t* s_out, cudaStream_t s)
{
    if (m <= 0) return cudaSuccess;
    k_staircase_many<<<grid_for(m, 256), 256, 0, s>>>(r, w, m, probs, nprob, s_out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_expand_tiles(const Seg* segs, const int32_t* prefix, int nseg, int total, Tile* out,
                                cudaStream_t s)
{
    if (total <= 0 || nseg <= 0) return cudaSuccess;
    k_expand_tiles<<<grid_for(total, 256), 256, 0, s>>>(segs, prefix, nseg, total, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_gather(const double* c, const int32_t* perm, int64_t n, int stride, int comp,
                          const unsigned long long* mx, double* out, float2* out2, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_gather<<<grid_for(n, 256), 256, 0, s>>>(c, perm, n, stride, comp, mx, out, out2);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_gather_deriv(const double* x, const int32_t* perm, const double* ws, int64_t nb, int stride,
                                int comp, const unsigned long long* mx, double* out, float2* out2, cudaStream_t s)
{
    if (nb <= 0) return cudaSuccess;
    k_gather_deriv<<<grid_for(2 * nb, 256), 256, 0, s>>>(x, perm, ws, nb, stride, comp, mx, out, out2);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_absmax_weighted(const double* x, const int32_t* perm, const double* ws, int64_t nb, int comps,
                                   unsigned long long* mx, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(mx, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess || nb <= 0) return e;
    k_absmax_weighted<<<grid_for(nb * comps, 256), 256, 0, s>>>(x, perm, ws, nb, comps, mx);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_scatter_deriv(const double* gs, const int32_t* perm, int64_t mb, int stride, int comp,
                                 const unsigned long long* mx, const double* y, double* out, cudaStream_t s)
{
    if (mb <= 0) return cudaSuccess;
    k_scatter_deriv<<<grid_for(mb, 256), 256, 0, s>>>(gs, perm, mb, stride, comp, mx, y, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_split_f64(const double* x, int64_t n, float2* out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_split_f64<<<grid_for(n, 256), 256, 0, s>>>(x, n, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_scatter(const double* gs, const int32_t* perm, int64_t m, int stride, int comp,
                           const unsigned long long* mx, double* g, cudaStream_t s)
{
    if (m <= 0) return cudaSuccess;
    k_scatter<<<grid_for(m, 256), 256, 0, s>>>(gs, perm, m, stride, comp, mx, g);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace nuht
