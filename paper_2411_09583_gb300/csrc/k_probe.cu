// Arithmetic throughput probe: the issue rate of the operations the transform's
// kernels are built from, measured on the device that runs them.  The execute
// kernels do their tap and moment arithmetic in double-float (df64.cuh), so
// their roofline is the rate of the compensated multiply-add acc_fma on the
// FP32 pipes; plain FP32 and FP64 fused multiply-adds are measured beside it.
//
// Every thread runs kChains independent chains (enough independent work per
// warp to keep the pipes busy), on a grid of kBlocksPerSm CTAs of kThreads
// threads per SM.  An empty asm statement marks the operands as rewritten each
// iteration, so the compiler cannot hoist the loop-invariant products out of
// the loop; it emits no instruction.
#include <cstdint>

#include "df64.cuh"
#include "nuht_host.h"

namespace nuht {

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 4;

__global__ void __launch_bounds__(kThreads) k_probe_ffma(int64_t iters, float* out)
{
    float a[kChains];
    const float b = 0.99999994f, c = 5.9604645e-08f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    out[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_probe_dfma(int64_t iters, double* out)
{
    double a[kChains];
    const double b = 0.9999999999999999, c = 1.1102230246251565e-16;
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = (double)(threadIdx.x + k) * 1e-3;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    out[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = s;
}

// acc_fma (df64.cuh) exactly as the kernels call it: a double-float product
// added to a compensated FP32 accumulator.
__global__ void __launch_bounds__(kThreads) k_probe_acc_fma(int64_t iters, double* out)
{
    acc2 A[kChains];
    df x[kChains];
    const df y = df{1.0009765625f, 1.1920929e-10f};
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
        A[k] = acc2{0.f, 0.f};
        x[k] = df{1e-4f * (float)(threadIdx.x + k + 1), 3e-12f};
    }
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) {
            asm volatile("" : "+f"(x[k].h), "+f"(x[k].l));
            acc_fma(A[k], x[k], y);
        }
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += acc_value(A[k]);
    out[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = s;
}

}  // namespace

}  // namespace nuht

using namespace nuht;

extern "C" int nuht_probe_alu(int kind, int64_t iters, double* ms, double* ops, void* stream)
{
    if (kind < 0 || kind > 2 || iters < 1 || iters > ((int64_t)1 << 32) || !ms || !ops)
        return NUHT_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return NUHT_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return NUHT_ERR_CUDA;
    const int blocks = sms * kBlocksPerSm;
    const size_t nthr = (size_t)blocks * kThreads;
    double* out = nullptr;
    if (pool_alloc((void**)&out, sizeof(double) * nthr, s) != cudaSuccess) return NUHT_ERR_NOMEM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = NUHT_OK;
    do {
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) { rc = NUHT_ERR_CUDA; break; }
        for (int pass = 0; pass < 2; ++pass) {   // the first pass warms up
            const int64_t it = pass == 0 ? (iters < 64 ? iters : 64) : iters;
            if (pass == 1 && cudaEventRecord(e0, s) != cudaSuccess) { rc = NUHT_ERR_CUDA; break; }
            if (kind == 0) k_probe_ffma<<<blocks, kThreads, 0, s>>>(it, (float*)out);
            else if (kind == 1) k_probe_dfma<<<blocks, kThreads, 0, s>>>(it, out);
            else k_probe_acc_fma<<<blocks, kThreads, 0, s>>>(it, out);
            count_launches(1);
            if (cudaGetLastError() != cudaSuccess) { rc = NUHT_ERR_CUDA; break; }
            if (pass == 1 && cudaEventRecord(e1, s) != cudaSuccess) { rc = NUHT_ERR_CUDA; break; }
        }
        if (rc != NUHT_OK) break;
        float t = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
            rc = NUHT_ERR_CUDA;
            break;
        }
        *ms = t;
        *ops = (double)nthr * (double)iters * kChains;
    } while (0);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    pool_free(out, s);
    if (cudaStreamSynchronize(s) != cudaSuccess && rc == NUHT_OK) rc = NUHT_ERR_CUDA;
    return rc;
}
