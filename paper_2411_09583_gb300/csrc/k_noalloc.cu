// No-allocation variant of the local (Wimp) block apply.
//
// Some callers cannot let a library call cudaMalloc: frameworks that reserve
// nearly all device memory for their own pool up front (a library allocation
// then fails or fragments that pool), and latency-critical loops in which
// cudaMalloc / cudaFree would stall on an implicit device synchronisation.
// nuht_local_apply_noalloc serves them for transforms whose whole matrix is
// local (every omega_k r_j <= z): it allocates nothing.  Its only scratch --
// the Wimp moments mu_l, l = 0..L, of each coefficient vector -- lives in the
// file-scope device array below, of fixed size kNoallocMoments doubles.
//
// That array exists once per GPU that loads the library and is held until the
// process exits.  Every call on a device uses the same array and it keeps the
// previous call's contents, so each call clears the part it uses first; calls
// that overlap on the GPU (for instance on two streams) race on it.
//
// Host code must not pass the symbol g_noalloc_moments to a kernel: on the
// host that name is only a stand-in.  The device address is looked up with
// cudaGetSymbolAddress the first time the entry point runs on a device (with
// that device current) and cached; that first call therefore does a little
// set-up and should come before any stream capture.  The cached address is
// that of the device's current context: after cudaDeviceReset the module is
// loaded again and the array may move, so the entry point must not be used
// across a device reset.
#include <cstdint>
#include <mutex>

#include "device_math.cuh"
#include "nuht_host.h"

namespace nuht {

namespace {

constexpr int kNoallocMoments = NUHT_NOALLOC_MAX_MOMENTS;   // 256 KiB per GPU
constexpr int kNoallocThreads = 128;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_moments[kNoallocMoments];

std::mutex g_noalloc_mu;
double* g_noalloc_ptr[kMaxDevices] = {nullptr};

// Device address of g_noalloc_moments on the current device (looked up once).
cudaError_t noalloc_scratch(double** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_moments);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = (double*)p;
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

// Moments mu[v][l] = sum_j c[j][v] T_{2l(+1)}(r_j / R) (Sec. 3.1), one vector
// per blockIdx.y; per-thread partial sums in shared memory, then one atomic
// add per (CTA, l) into the static scratch.
__global__ void __launch_bounds__(kNoallocThreads)
k_noalloc_moments(int nu, int L, const double* __restrict__ r, int64_t n, double invR,
                  const double* __restrict__ c, int nvec, double* __restrict__ mom)
{
    extern __shared__ double acc[];
    const int nt = blockDim.x, tid = threadIdx.x, v = blockIdx.y;
    const int odd = nu & 1;
    for (int l = 0; l <= L; ++l) acc[l * nt + tid] = 0.0;
    for (int64_t j = blockIdx.x * (int64_t)nt + tid; j < n; j += (int64_t)gridDim.x * nt) {
        const double y = r[j] * invR;
        const double cj = c[j * nvec + v];
        const double u = fma(2.0 * y, y, -1.0);
        const double u2 = 2.0 * u;
        double t0 = odd ? y : 1.0;
        double t1 = odd ? y * (u2 - 1.0) : u;
        acc[tid] += cj * t0;
        if (L >= 1) acc[nt + tid] += cj * t1;
        for (int l = 2; l <= L; ++l) {
            const double t2 = fma(u2, t1, -t0);
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
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
        if (lane == 0) atomicAdd(&mom[(int64_t)v * (L + 1) + l], s);
    }
}

// g[k][v] = sign * sum_l C_l(omega_k R) mu[v][l]: Miller's backward recurrence
// for J_0..J_ntop(omega_k R / 2) in this thread's shared-memory column, then
// the Wimp coefficients C_l and the dot product with each vector's moments.
__global__ void k_noalloc_eval(int nu, int sgn, int L, int ntop, const double* __restrict__ omega,
                               int64_t m, double R, const double* __restrict__ mom, int nvec,
                               double* __restrict__ g)
{
    extern __shared__ double jb[];
    const int nt = blockDim.x, tid = threadIdx.x;
    const int64_t k = blockIdx.x * (int64_t)nt + tid;
    if (k >= m) return;
    const double y = 0.5 * omega[k] * R;
    if (y < 1e-100) {
        for (int v = 0; v < nvec; ++v)
            g[k * nvec + v] = (nu == 0) ? (double)sgn * mom[(int64_t)v * (L + 1)] : 0.0;
        return;
    }
    const int hp = (nu & 1) ? (nu + 1) / 2 : nu / 2;
    const int hm = (nu & 1) ? (nu - 1) / 2 : nu / 2;
    double S = 1.0;
    if (y < 1.0) {
        // power series (DLMF 10.2.2), already normalised: for small y each
        // backward step multiplies by about 2i/y, faster than the rescaling
        // below could follow
        const double h = 0.5 * y, q = -h * h;
        double lead = 1.0;   // (y/2)^i / i!
        for (int i = 0; i <= ntop; ++i) {
            if (i > 0) lead *= h / (double)i;
            double term = lead, sum = lead;
            for (int t = 1; t <= 12; ++t) {
                term *= q / ((double)t * (double)(i + t));
                sum += term;
            }
            jb[i * nt + tid] = sum;
        }
    } else {
        const int ns = miller_start(ntop, y);
        const double inv2y = 2.0 / y;
        double jp1 = 0.0, jc = 1.0;
        S = 2.0;
        if (ns <= ntop) jb[ns * nt + tid] = jc;
        for (int i = ns; i >= 2; i -= 2) {
            const double jm = fma((double)i * inv2y, jc, -jp1);
            const double jmm = fma((double)(i - 1) * inv2y, jm, -jc);
            if (i - 1 <= ntop) jb[(i - 1) * nt + tid] = jm;
            if (i - 2 <= ntop) jb[(i - 2) * nt + tid] = jmm;
            S = fma(2.0, jmm, S);
            jp1 = jm;
            jc = jmm;
            if (too_big(jc)) {
                const double sc = 1e-150;
                jc *= sc; jp1 *= sc; S *= sc;
                const int top = ntop < ns ? ntop : ns;
                for (int q = i - 2; q <= top; ++q) jb[q * nt + tid] *= sc;
            }
        }
        S -= jc;
    }
    const double inv_s2 = 1.0 / (S * S);
    for (int v = 0; v < nvec; ++v) {
        const double* mu = mom + (int64_t)v * (L + 1);
        double sum = 0.0;
        for (int l = 0; l <= L; ++l) {
            const int b = hm - l;
            double jbv = jb[(b >= 0 ? b : -b) * nt + tid];
            if (b < 0 && ((-b) & 1)) jbv = -jbv;
            double cl = jb[(hp + l) * nt + tid] * jbv;
            if (l > 0 || (nu & 1)) cl *= 2.0;
            sum = fma(cl, mu[l], sum);
        }
        g[k * nvec + v] = (double)sgn * sum * inv_s2;
    }
}

}  // namespace

}  // namespace nuht

using namespace nuht;

extern "C" int nuht_local_apply_noalloc(int nu, double eps, const double* r, int64_t n, double r_max,
                                        const double* omega, int64_t m, double omega_max,
                                        const double* c, double* g, int nvec, void* stream)
{
    if (n < 0 || m < 0 || nvec < 1) return NUHT_ERR_INVALID_ARG;
    if ((n > 0 && (!r || !c)) || (m > 0 && (!omega || !g))) return NUHT_ERR_INVALID_ARG;
    if (!(eps >= 1e-15 && eps <= 1e-1)) return NUHT_ERR_INVALID_ARG;
    if (nu > 100 || nu < -100) return NUHT_ERR_UNSUPPORTED;
    if (!(r_max >= 0.0) || !(omega_max >= 0.0) || !(r_max < INFINITY) || !(omega_max < INFINITY))
        return NUHT_ERR_DOMAIN;
    const int anu = nu < 0 ? -nu : nu;
    const int sgn = (nu < 0 && (anu & 1)) ? -1 : 1;
    int M = 0, L = 0;
    double z = 0.0;
    int rc = choose_params(anu, eps, 0, &M, &z, &L);
    if (rc != NUHT_OK) return rc;
    // the whole matrix must be local: every omega_k r_j <= omega_max r_max <= z
    if (omega_max * r_max > z) return NUHT_ERR_DOMAIN;
    const int hp = (anu & 1) ? (anu + 1) / 2 : anu / 2;
    const int ntop = hp + L;
    if (ntop >= kMaxNtop) return NUHT_ERR_UNSUPPORTED;
    if ((int64_t)nvec * (L + 1) > kNoallocMoments) return NUHT_ERR_SCRATCH;
    cudaStream_t s = (cudaStream_t)stream;
    if (m == 0) return NUHT_OK;
    if (n == 0) {
        cudaError_t e = cudaMemsetAsync(g, 0, sizeof(double) * (size_t)m * nvec, s);
        return e == cudaSuccess ? NUHT_OK : NUHT_ERR_CUDA;
    }
    double* mom = nullptr;
    cudaError_t e = noalloc_scratch(&mom);
    if (e != cudaSuccess) return NUHT_ERR_CUDA;
    // the scratch keeps the previous call's moments: clear the part used here
    e = cudaMemsetAsync(mom, 0, sizeof(double) * (size_t)nvec * (L + 1), s);
    if (e != cudaSuccess) return NUHT_ERR_CUDA;
    const double R = r_max > 0.0 ? r_max : 1.0;   // any R >= max r_j with omega_max R <= z
    const double Rm = (r_max > 0.0) ? r_max : 0.0;
    {
        const int threads = local_moment_threads(L);   // (L + 1) doubles per thread
        const size_t smem = sizeof(double) * (size_t)(L + 1) * threads;
        e = cudaFuncSetAttribute(k_noalloc_moments, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return NUHT_ERR_CUDA;
        int dev = 0, sms = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return NUHT_ERR_CUDA;
        int64_t blocks = (n + threads - 1) / threads;
        if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;   // grid-stride beyond 8 CTAs per SM
        dim3 grid((unsigned)blocks, (unsigned)nvec);
        k_noalloc_moments<<<grid, threads, smem, s>>>(anu, L, r, n, Rm > 0.0 ? 1.0 / R : 0.0,
                                                              c, nvec, mom);
        e = cudaGetLastError();
        if (e != cudaSuccess) return NUHT_ERR_CUDA;
        count_launches(1);
    }
    {
        const int threads = local_eval_threads(ntop);
        const size_t smem = sizeof(double) * (size_t)(ntop + 1) * threads;
        e = cudaFuncSetAttribute(k_noalloc_eval, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return NUHT_ERR_CUDA;
        const int64_t blocks = (m + threads - 1) / threads;
        k_noalloc_eval<<<(unsigned)blocks, threads, smem, s>>>(anu, sgn, L, ntop, omega, m, Rm, mom, nvec, g);
        e = cudaGetLastError();
        if (e != cudaSuccess) return NUHT_ERR_CUDA;
        count_launches(1);
    }
    return NUHT_OK;
}
