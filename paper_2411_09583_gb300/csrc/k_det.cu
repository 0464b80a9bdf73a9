// Per-call input scaling, and the deterministic mode's conversion of the
// exact 128-bit sums (det_acc.cuh) back to FP64.
//
// The execute kernels hold the coefficients as double-float numbers (pairs of
// FP32), whose exponent range is FP32's.  Every call therefore first scales
// its input vector by 2^-E, E the exponent of the largest |x_i|, so that the
// largest magnitude lies in [1, 2), and scales the output back by 2^E: both
// exact in FP64, and the transform is linear, so any finite input range works.
#include <cstdint>

#include "nuht_internal.h"

namespace nuht {

int device_sm_count();

namespace {

constexpr int kDetThreads = 256;

// *mx = max |x_i| as the bit pattern of a non-negative double (whose integer
// order is the order of the values): a maximum does not depend on the order
// of the updates, so the scale is the same on every run.
__global__ void __launch_bounds__(kDetThreads) k_absmax_bits(const double* __restrict__ x, int64_t count,
                                                             unsigned long long* __restrict__ mx)
{
    unsigned long long m = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(x[i]) & 0x7fffffffffffffffull;
        m = b > m ? b : m;
    }
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, m, off);
        m = o > m ? o : m;
    }
    if ((threadIdx.x & 31) == 0 && m) atomicMax(mx, m);
}

__global__ void __launch_bounds__(kDetThreads) k_fx_decode(const Fx128* __restrict__ src, double* __restrict__ dst,
                                                           int64_t count, const ProbParams* __restrict__ probs)
{
    const int fxs = probs[0].fxs;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = fx_decode(src[i], fxs);
}

int grid_for(int64_t count)
{
    const int64_t need = (count + kDetThreads - 1) / kDetThreads;
    const int64_t cap = (int64_t)device_sm_count() * 8;
    return (int)(need < 1 ? 1 : (need < cap ? need : cap));
}

}  // namespace

int device_sm_count()
{
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (dev >= 0 && dev < 64 && cache[dev] > 0) return cache[dev];
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) return 1;
    if (dev >= 0 && dev < 64) cache[dev] = sms;
    return sms;
}

cudaError_t launch_input_scale(const double* x, int64_t count, unsigned long long* mx, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(mx, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    if (count > 0) {
        k_absmax_bits<<<grid_for(count), kDetThreads, 0, s>>>(x, count, mx);
        count_launches(1);
    }
    return cudaGetLastError();
}

cudaError_t launch_fx_decode(const void* src, double* dst, int64_t count, const ProbParams* probs, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    k_fx_decode<<<grid_for(count), kDetThreads, 0, s>>>((const Fx128*)src, dst, count, probs);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace nuht
