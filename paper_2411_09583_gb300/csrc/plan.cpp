// C ABI of the NUHT library: plan (sort + subdivision + work lists), execute
// (Algorithm 2 on the device), info and helpers.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <mutex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "nuht_host.h"

using namespace nuht;

namespace {

thread_local std::string g_cuda_msg = "no CUDA error";
std::atomic<int64_t> g_launches{0};

const char* const kStageNames[NUHT_NUM_STAGES] = {
    "gather", "local_moments", "asy_spread", "asy_fft", "asy_interp", "local_eval", "direct", "scatter"};

inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

#define NUHT_CK(call)                                                                   \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            g_cuda_msg = std::string(#call) + ": " + cudaGetErrorString(e_);           \
            return e_ == cudaErrorMemoryAllocation ? NUHT_ERR_NOMEM : NUHT_ERR_CUDA;    \
        }                                                                               \
    } while (0)

// One device allocation carved into aligned pieces.
struct Arena {
    size_t size = 0;
    template <class T>
    size_t reserve(size_t count)
    {
        size_t off = size;
        size += align256(sizeof(T) * (count > 0 ? count : 1));
        return off;
    }
};

// Segments of a tile list plus their exclusive prefix of tile counts; the
// tiles themselves are expanded on the device.
struct SegList {
    std::vector<Seg> segs;
    std::vector<int32_t> prefix{0};
    void add(int32_t blk, int64_t first, int64_t last, int len)
    {
        const int64_t cnt = (last - first + len) / len;
        segs.push_back(Seg{blk, len, first, last});
        prefix.push_back(prefix.back() + (int32_t)cnt);
    }
    void reserve(size_t k)
    {
        segs.reserve(k);
        prefix.reserve(k + 1);
    }
    int nseg() const { return (int)segs.size(); }
    int total() const { return prefix.back(); }
};

}  // namespace

struct nuht_plan_s {
    int nu_user = 0;
    // derivative plan (nuht_plan_deriv): problems nu - 1 and nu + 1 (the
    // second with its sign flipped) over two copies of the base plan's sorted
    // points and frequencies; n_base, m_base are the base plan's sizes
    bool deriv = false;
    int64_t n_base = 0, m_base = 0;
    double eps = 0.0;
    nuht_opts opt{};
    int64_t n = 0, m = 0;
    cudaStream_t stream = nullptr;
    std::vector<ProbParams> probs;   // one per problem of the batch (one for nuht_plan)
    int lmax = 0, qmax = 0;          // largest L and Q = 2M over the problems
    int w = 0;

    // device memory
    char* dmem = nullptr;
    size_t dbytes = 0;
    ProbParams* d_prob = nullptr;
    double *d_r = nullptr, *d_w = nullptr;
    int32_t *d_pr = nullptr, *d_pw = nullptr;
    LocalBlock* d_loc = nullptr;
    Tile *d_tmom = nullptr, *d_teval = nullptr;
    AsyBlock* d_asy = nullptr;
    Tile *d_tspread = nullptr, *d_tinterp = nullptr;
    int32_t* d_smode = nullptr;   // path of each spreading tile (k_spread_modes)
    Tile *d_fblock = nullptr, *d_fsmall = nullptr, *d_fa = nullptr, *d_fb = nullptr;
    DirectBlock* d_dir = nullptr;
    double* d_mom = nullptr;
    double2* d_gb = nullptr;
    float4* d_gtmp = nullptr;   // two-pass FFT intermediate (double-float)
    float4* d_gq = nullptr;   // FFT output, complex values as double-float parts
    double2* d_tg = nullptr;  // adjoint: frequencies spread onto the FFT grid
    float4* d_bq = nullptr;   // adjoint: corrected modes, double-float parts
    double *d_cs = nullptr, *d_gs = nullptr;
    float2 *d_r2 = nullptr, *d_w2 = nullptr, *d_cs2 = nullptr;   // double-float copies
    // the next real component of a pair (complex c, or two vectors), whose
    // local and direct blocks are applied together with the first: its c, local
    // moments and sums
    double *d_csb = nullptr, *d_gsb = nullptr, *d_momb = nullptr;
    float2* d_cs2b = nullptr;
    double *d_es = nullptr, *d_ph = nullptr;
    double2* d_tw = nullptr;
    // per-call input scaling: the bits of the largest input magnitude
    unsigned long long* d_mx = nullptr;
    // persistent local stage: queue head, per-block moment-tile counts and the
    // moment tiles' prefix per block; status word of bounded device waits
    int* d_q = nullptr;
    const int32_t* d_pre_mom = nullptr;
    int* d_status = nullptr;
    // deterministic mode: exact fixed-point (Fx128) accumulators in place of
    // the FP64 targets of the atomics (same element indices)
    bool det = false;
    Fx128 *f_gs = nullptr, *f_gsb = nullptr, *f_cs = nullptr, *f_csb = nullptr;
    Fx128 *f_mom = nullptr, *f_momb = nullptr, *f_gb = nullptr, *f_tg = nullptr;

    int n_loc = 0, n_tmom = 0, n_teval = 0;
    int n_asy = 0, n_tspread = 0, n_tinterp = 0, n_fblock = 0, n_fsmall = 0, n_fa = 0, n_fb = 0;
    int n_dir = 0;
    int64_t mom_len = 0, gb_len = 0, gq_len = 0;
    int max_fblock_pts = 0;   // largest nf2 * Q among the blocks FFT'd whole by one CTA
    int max_nf2_small = 0, max_dir_rows = 0, max_dir_cols = 0, max_dir_area = 0, ntop_max = 0, nu_max = 0, eval_threads = 0;
    int spread_threads = 256;
    // real components per asymptotic launch (forward spreading and
    // interpolation, FP64 path): grids for that many are allocated
    int asy_members = 1;
    int interp_threads = kInterpTileMax;   // frequencies per interpolation tile (one thread each)
    bool has_large_fft = false;
    Tables tab{};
    SubBlk* d_blk = nullptr;          // every block (local, asymptotic, direct), global sorted indices
    int64_t direct_entries = 0, local_rc = 0, asy_rc = 0, fft_points = 0;
    double plan_ms[4] = {0, 0, 0, 0};

    // stage timing (opts.timing): event pairs per (vector component, stage)
    std::vector<cudaEvent_t> ev;
    std::vector<char> ev_used;
    int ev_comps = 0;
};

// Real components applied together by nuht_execute (opts.vec_group; 0 = a
// pair), and the copies of the per-component arrays the plan holds.
static int group_size(const nuht_plan_s* P) { return P->opt.vec_group ? P->opt.vec_group : 2; }
static int group_copies(const nuht_plan_s* P) { return group_size(P) > 2 ? group_size(P) : 2; }
// Device memory the grids of the extra members of an asymptotic launch may take.
constexpr size_t kAsyMemberBytes = (size_t)1 << 30;

namespace nuht {

void count_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

namespace {
constexpr int kMaxDev = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[kMaxDev] = {};
}  // namespace

namespace {
// Host-side fault injection (testing aid): with NUHT_FAULT_ALLOC=k in the
// environment, the k-th device allocation of the library counted from when
// that value was first seen fails as if the device were out of memory.  It
// acts before any CUDA call, so it also runs without a GPU.
std::mutex g_fault_mu;
std::string g_fault_val;
long g_fault_count = 0;

bool injected_alloc_failure()
{
    const char* f = std::getenv("NUHT_FAULT_ALLOC");
    if (!f || !*f) return false;
    std::lock_guard<std::mutex> lock(g_fault_mu);
    if (g_fault_val != f) {
        g_fault_val = f;
        g_fault_count = 0;
    }
    const long k = std::atol(f);
    return k > 0 && ++g_fault_count == k;
}
}  // namespace

// One memory pool per device, owned by the library, whose release threshold
// keeps freed plan memory reserved for the next plan (no re-mapping per plan).
cudaError_t pool_alloc(void** p, size_t bytes, cudaStream_t s)
{
    if (injected_alloc_failure()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDev) return cudaErrorInvalidDevice;
    cudaMemPool_t pool;
    {
        std::lock_guard<std::mutex> lock(g_pool_mu);
        if (!g_pool[dev]) {
            cudaMemPoolProps props = {};
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            e = cudaMemPoolCreate(&g_pool[dev], &props);
            if (e != cudaSuccess) { g_pool[dev] = nullptr; return e; }
            uint64_t thr = ~(uint64_t)0;
            e = cudaMemPoolSetAttribute(g_pool[dev], cudaMemPoolAttrReleaseThreshold, &thr);
            if (e != cudaSuccess) return e;
        }
        pool = g_pool[dev];
    }
    return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

void pool_free(void* p, cudaStream_t s)
{
    if (p) cudaFreeAsync(p, s);
}

}  // namespace nuht

namespace {

// Pinned host staging buffers (grow-only), used by one plan build at a time.
struct Staging {
    char* p = nullptr;
    size_t cap = 0;
    cudaError_t reserve(size_t bytes)
    {
        if (bytes <= cap) return cudaSuccess;
        if (p) cudaFreeHost(p);
        p = nullptr;
        cap = 0;
        size_t want = bytes + bytes / 2 + (1 << 20);
        cudaError_t e = cudaMallocHost((void**)&p, want);
        if (e == cudaSuccess) cap = want;
        return e;
    }
};
std::mutex g_stage_mu;
Staging g_stage_in, g_stage_out;

// Per-device auxiliary stream (and fork / join events) for the independent
// halves of a plan build, used under g_stage_mu.
struct Aux {
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    cudaEvent_t stage_done = nullptr;   // the last upload from g_stage_out on this device
};
cudaEvent_t g_stage_out_event = nullptr;   // set with the last upload; waited on before reuse
Aux g_aux[64];

cudaError_t aux_stream(Aux** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    Aux& a = g_aux[dev];
    if (!a.s) {
        e = cudaStreamCreateWithFlags(&a.s, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&a.fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&a.join, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&a.stage_done, cudaEventDisableTiming);
        if (e != cudaSuccess) return e;
    }
    *out = &a;
    return cudaSuccess;
}

// Per host thread and device: the stream on which the host-buffer entry point
// uploads the coefficients while the plan runs, with its fork and done events.
struct CopyAux {
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, done = nullptr;
};

cudaError_t copy_aux(CopyAux** out)
{
    thread_local CopyAux a[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    CopyAux& x = a[dev];
    if (!x.s) {
        e = cudaStreamCreateWithFlags(&x.s, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&x.fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&x.done, cudaEventDisableTiming);
        if (e != cudaSuccess) return e;
    }
    *out = &x;
    return cudaSuccess;
}

// Per host thread and device: the two streams (and fork / join events) on
// which an execute runs its block classes: the asymptotic pipeline on a
// stream of the greatest priority, the local and direct blocks on one of the
// default priority, so that their CTAs take what the asymptotic kernels'
// CTAs leave free on an SM.  Per thread, so that executes from several host
// threads never share an event.
struct ExecAux {
    cudaStream_t lo = nullptr, hi = nullptr;
    cudaEvent_t fork = nullptr, join_lo = nullptr, join_hi = nullptr;
};
thread_local ExecAux t_exec_aux[64];

// Forks the two streams off s and joins them back into s on close() or when
// it goes out of scope (also on an early error return, so that no work of the
// execute outlives the caller's stream).  Graph capture follows the event
// record / wait pairs.
struct ClassFork {
    ExecAux* ax = nullptr;
    cudaStream_t main = nullptr;
    cudaError_t open(cudaStream_t s)
    {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
        ExecAux& a = t_exec_aux[dev];
        if (!a.lo) {
            int least = 0, greatest = 0;
            e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
            if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&a.hi, cudaStreamNonBlocking, greatest);
            if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&a.lo, cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&a.fork, cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&a.join_lo, cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&a.join_hi, cudaEventDisableTiming);
            if (e != cudaSuccess) return e;
        }
        e = cudaEventRecord(a.fork, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(a.lo, a.fork, 0);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(a.hi, a.fork, 0);
        if (e != cudaSuccess) return e;
        ax = &a;
        main = s;
        return cudaSuccess;
    }
    cudaStream_t local(cudaStream_t s) const { return ax ? ax->lo : s; }
    cudaStream_t asy(cudaStream_t s) const { return ax ? ax->hi : s; }
    cudaError_t close()
    {
        if (!ax) return cudaSuccess;
        cudaError_t e = cudaEventRecord(ax->join_lo, ax->lo);
        if (e == cudaSuccess) e = cudaEventRecord(ax->join_hi, ax->hi);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(main, ax->join_lo, 0);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(main, ax->join_hi, 0);
        ax = nullptr;
        return e;
    }
    ~ClassFork() { close(); }
};

}  // namespace

namespace {

// Records the start / end event of a stage when the plan times its stages.
struct StageTimer {
    nuht_plan_t P;
    int comp;
    int begin(int stage, cudaStream_t s)
    {
        if (!P->opt.timing) return NUHT_OK;
        size_t i = ((size_t)comp * NUHT_NUM_STAGES + stage) * 2;
        P->ev_used[i / 2] = 1;
        NUHT_CK(cudaEventRecord(P->ev[i], s));
        return NUHT_OK;
    }
    int end(int stage, cudaStream_t s)
    {
        if (!P->opt.timing) return NUHT_OK;
        size_t i = ((size_t)comp * NUHT_NUM_STAGES + stage) * 2;
        NUHT_CK(cudaEventRecord(P->ev[i + 1], s));
        return NUHT_OK;
    }
};

int ensure_events(nuht_plan_t P, int comps)
{
    if (!P->opt.timing) return NUHT_OK;
    size_t need = (size_t)comps * NUHT_NUM_STAGES * 2;
    while (P->ev.size() < need) {
        cudaEvent_t e;
        NUHT_CK(cudaEventCreate(&e));
        P->ev.push_back(e);
    }
    P->ev_used.assign(P->ev.size() / 2, 0);
    P->ev_comps = comps;
    return NUHT_OK;
}

}  // namespace

extern "C" {

void nuht_default_opts(nuht_opts* o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = NUHT_PREC_FP64;
    o->min_size = 1024;
    o->n_split_cand = 16;
    o->m_terms = 0;
    o->class_mask = 7;
}

const char* nuht_strerror(int code)
{
    switch (code) {
        case NUHT_OK: return "ok";
        case NUHT_ERR_INVALID_ARG: return "invalid argument";
        case NUHT_ERR_DOMAIN: return "r and omega must be finite and non-negative";
        case NUHT_ERR_NOMEM: return "out of memory";
        case NUHT_ERR_CUDA: return "CUDA error";
        case NUHT_ERR_TIMEOUT: return "device wait timed out";
        case NUHT_ERR_UNSUPPORTED: return "unsupported parameters";
        case NUHT_ERR_SCRATCH: return "request exceeds the no-allocation scratch (nvec * (L + 1) > NUHT_NOALLOC_MAX_MOMENTS)";
        case NUHT_ERR_BAD_BLOCKS: return "a block work list failed its check (cover, classes or sizes)";
        default: return "unknown status";
    }
}

const char* nuht_last_cuda_error(void) { return g_cuda_msg.c_str(); }

int nuht_choose_params(int nu, double eps, int m_terms, int* M, double* z, int* L)
{
    if (!M || !z || !L) return NUHT_ERR_INVALID_ARG;
    if (!(eps >= 1e-15 && eps <= 1e-1)) return NUHT_ERR_INVALID_ARG;
    if (m_terms < 0 || m_terms > kMaxM) return NUHT_ERR_INVALID_ARG;
    if (nu > 100 || nu < -100) return NUHT_ERR_UNSUPPORTED;
    return choose_params(nu, eps, m_terms, M, z, L);
}

int nuht_check_blocks(int nu, double eps, int m_terms, const double* r_sorted, int64_t n,
                      const double* omega_sorted, int64_t m, int min_size, const int64_t* ranges,
                      const int32_t* cls, int64_t count)
{
    if (n < 0 || m < 0 || count < 0 || min_size < 1) return NUHT_ERR_INVALID_ARG;
    if ((n > 0 && !r_sorted) || (m > 0 && !omega_sorted) || (count > 0 && (!ranges || !cls)))
        return NUHT_ERR_INVALID_ARG;
    int M = 0, L = 0;
    double z = 0.0;
    const int rc = nuht_choose_params(nu, eps, m_terms, &M, &z, &L);
    if (rc != NUHT_OK) return rc;
    return check_blocks(r_sorted, n, omega_sorted, m, z, min_size, ranges, cls, count) ? NUHT_OK
                                                                                         : NUHT_ERR_BAD_BLOCKS;
}

void nuht_destroy(nuht_plan_t p)
{
    if (!p) return;
    if (p->dmem) {
        pool_free(p->dmem, p->stream);
        cudaStreamSynchronize(p->stream);
    }
    for (cudaEvent_t e : p->ev) cudaEventDestroy(e);
    delete p;
}

int64_t nuht_kernel_launch_count(void) { return g_launches.load(); }

int nuht_status(nuht_plan_t P, void* stream)
{
    if (!P) return NUHT_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (!P->d_status) return NUHT_OK;
    int h = 0;
    NUHT_CK(cudaMemcpyAsync(&h, P->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    NUHT_CK(cudaMemsetAsync(P->d_status, 0, sizeof(int), s));
    NUHT_CK(cudaStreamSynchronize(s));
    return h;
}

const char* nuht_stage_name(int i) { return (i >= 0 && i < NUHT_NUM_STAGES) ? kStageNames[i] : nullptr; }

int nuht_stage_times(nuht_plan_t P, double* ms, int cap)
{
    if (!P || !ms || cap < 0 || !P->opt.timing || P->ev_comps == 0) return NUHT_ERR_INVALID_ARG;
    for (int st = 0; st < cap; ++st) ms[st] = 0.0;
    for (int comp = 0; comp < P->ev_comps; ++comp) {
        for (int st = 0; st < NUHT_NUM_STAGES && st < cap; ++st) {
            size_t i = (size_t)comp * NUHT_NUM_STAGES + st;
            if (!P->ev_used[i]) continue;
            NUHT_CK(cudaEventSynchronize(P->ev[2 * i + 1]));
            float t = 0.f;
            NUHT_CK(cudaEventElapsedTime(&t, P->ev[2 * i], P->ev[2 * i + 1]));
            ms[st] += t;
        }
    }
    return NUHT_OK;
}

static double ms_since(std::chrono::steady_clock::time_point& t)
{
    auto now = std::chrono::steady_clock::now();
    double ms = std::chrono::duration<double, std::milli>(now - t).count();
    t = now;
    return ms;
}

// Temporaries of the device work-list build (offsets into an arena).
struct BuildTemps {
    size_t loc, asy, dir, fcls, lcnt, acnt, dcnt, tot, maxv, scan;
};

static BuildTemps reserve_build_temps(Arena& a, int64_t cap)
{
    BuildTemps t;
    t.loc = a.reserve<LocalBlock>(cap);
    t.asy = a.reserve<AsyBlock>(cap);
    t.dir = a.reserve<DirectBlock>(cap);
    t.fcls = a.reserve<int8_t>(cap);
    t.lcnt = a.reserve<int64_t>(cap * kLocalCols);
    t.acnt = a.reserve<int64_t>(cap * kAsyCols);
    t.dcnt = a.reserve<int64_t>(cap * kDirCols);
    t.tot = a.reserve<int64_t>(kTotals);
    t.maxv = a.reserve<int64_t>(kMaxv);
    t.scan = a.reserve<int64_t>(block_scan_scratch(cap));
    return t;
}

static void bind_build_temps(BlockBuild& bb, char* base, const BuildTemps& t)
{
    bb.loc = (LocalBlock*)(base + t.loc);
    bb.asy = (AsyBlock*)(base + t.asy);
    bb.dir = (DirectBlock*)(base + t.dir);
    bb.fcls = (int8_t*)(base + t.fcls);
    bb.lcnt = (int64_t*)(base + t.lcnt);
    bb.acnt = (int64_t*)(base + t.acnt);
    bb.dcnt = (int64_t*)(base + t.dcnt);
    bb.totals = (int64_t*)(base + t.tot);
    bb.maxv = (int64_t*)(base + t.maxv);
}

// Checked mode (NUHT_CHECKED set and not "0"): the device-built block lists
// and sorted values go back to the host and each problem's list is checked
// (exact cover, classes, direct-block areas) before the plan is returned.
static int verify_lists(nuht_plan_t P)
{
    const int64_t nb = (int64_t)P->n_loc + P->n_asy + P->n_dir;
    std::vector<SubBlk> blk((size_t)nb);
    std::vector<double> hr((size_t)P->n), hw((size_t)P->m);
    if (nb) NUHT_CK(cudaMemcpyAsync(blk.data(), P->d_blk, sizeof(SubBlk) * nb, cudaMemcpyDeviceToHost, P->stream));
    if (P->n) NUHT_CK(cudaMemcpyAsync(hr.data(), P->d_r, sizeof(double) * P->n, cudaMemcpyDeviceToHost, P->stream));
    if (P->m) NUHT_CK(cudaMemcpyAsync(hw.data(), P->d_w, sizeof(double) * P->m, cudaMemcpyDeviceToHost, P->stream));
    NUHT_CK(cudaStreamSynchronize(P->stream));
    const size_t np = P->probs.size();
    std::vector<std::vector<int64_t>> rg(np);
    std::vector<std::vector<int32_t>> cl(np);
    for (int64_t b = 0; b < nb; ++b) {
        const SubBlk& x = blk[(size_t)b];
        if (x.prob < 0 || (size_t)x.prob >= np) return NUHT_ERR_BAD_BLOCKS;
        const ProbParams& q = P->probs[(size_t)x.prob];
        rg[(size_t)x.prob].insert(rg[(size_t)x.prob].end(),
                                  {x.k0 - q.w_off, x.k1 - q.w_off, x.j0 - q.r_off, x.j1 - q.r_off});
        cl[(size_t)x.prob].push_back(b < P->n_loc ? NUHT_BLOCK_LOCAL
                                                  : (b < (int64_t)P->n_loc + P->n_asy ? NUHT_BLOCK_ASY : NUHT_BLOCK_DIRECT));
    }
    for (size_t i = 0; i < np; ++i) {
        const ProbParams& q = P->probs[i];
        if (!check_blocks(hr.data() + q.r_off, q.n, hw.data() + q.w_off, q.m, q.z, P->opt.min_size, rg[i].data(),
                          cl[i].data(), (int64_t)cl[i].size()))
            return NUHT_ERR_BAD_BLOCKS;
    }
    return NUHT_OK;
}

#define NUHT_TRY_BUILD(x)               \
    do {                                \
        int rc_ = (x);                  \
        if (rc_ != NUHT_OK) return rc_; \
    } while (0)

// src: build from the sorted arrays and permutations of that plan, repeated
// once per problem (derivative plans), instead of checking and sorting r and omega.
static int build_plan(nuht_plan_t P, const double* r, const double* omega, const nuht_plan_s* src = nullptr)
{
    auto clk = std::chrono::steady_clock::now();
    if (P->opt.deterministic)
        for (ProbParams& q : P->probs) q.fxs = kFxScale;
    cudaStream_t s = P->stream;
    const int64_t n = P->n, m = P->m;
    const int nprob = (int)P->probs.size();
    std::vector<ProbParams>& probs = P->probs;
    P->lmax = 0;
    P->qmax = 0;
    P->ntop_max = 0;
    P->nu_max = 0;
    for (const ProbParams& q : probs) {
        P->nu_max = q.nu > P->nu_max ? q.nu : P->nu_max;
        P->lmax = q.L > P->lmax ? q.L : P->lmax;
        P->qmax = q.Q > P->qmax ? q.Q : P->qmax;
        P->ntop_max = q.ntop > P->ntop_max ? q.ntop : P->ntop_max;
    }

    // ---- sort (device) -------------------------------------------------
    Arena sa;
    size_t o_r = sa.reserve<double>(n), o_w = sa.reserve<double>(m);
    size_t o_pr = sa.reserve<int32_t>(n), o_pw = sa.reserve<int32_t>(m);
    size_t o_st = sa.reserve<int32_t>(m);
    size_t o_flag = sa.reserve<int>(2);
    size_t o_prb = sa.reserve<ProbParams>(probs.size());
    size_t o_roff = sa.reserve<int64_t>(probs.size() + 1), o_woff = sa.reserve<int64_t>(probs.size() + 1);
    // device subdivision: two level queues, the three block lists, edge values;
    // work-list build: descriptors, FFT classes, per-block counters, totals
    int64_t qcap = (n + m) / 4 + 4096 + nprob, ocap = (n + m) / 16 + 16384 + nprob;
    if (const char* cap = std::getenv("NUHT_SUBDIVIDE_CAPACITY")) {
        // test knob: smaller device lists exercise the host fallback
        const long long c = std::atoll(cap);
        if (c > 0) {
            qcap = c < qcap ? c : qcap;
            ocap = c < ocap ? c : ocap;
        }
    }
    size_t o_qa = sa.reserve<SubBlk>(qcap), o_qb = sa.reserve<SubBlk>(qcap);
    size_t o_out = sa.reserve<SubBlk>(3 * ocap);
    size_t o_bl = sa.reserve<double>(ocap), o_ba = sa.reserve<double4>(ocap);
    size_t o_res = sa.reserve<int64_t>(4);
    const int sub_ctas = subdivide_grid_ctas();
    size_t o_ctot = sa.reserve<int4>(sub_ctas > 0 ? (size_t)sub_ctas : 1), o_gst = sa.reserve<int64_t>(8);
    BuildTemps bt = reserve_build_temps(sa, ocap);
    size_t o_scr = sa.size;
    const size_t scr = radix_sort_scratch_bytes(n), scr_w = radix_sort_scratch_bytes(m);
    sa.size += align256(scr);
    const size_t o_scr_w = sa.size;
    sa.size += align256(scr_w);
    char* sort_mem = nullptr;
    NUHT_CK(pool_alloc((void**)&sort_mem, sa.size, s));
    struct Free {
        char* p; cudaStream_t s;
        ~Free() { pool_free(p, s); }
    } free_sort{sort_mem, s};
    int* d_flag = (int*)(sort_mem + o_flag);
    NUHT_CK(cudaMemsetAsync(d_flag, 0, sizeof(int) * 2, s));
    std::lock_guard<std::mutex> stage_lock(g_stage_mu);
    // a previous build's upload from the shared staging buffer may still be in flight
    if (g_stage_out_event) NUHT_CK(cudaEventSynchronize(g_stage_out_event));
    // problems and segment offsets (needed by the segmented sort and the staircase)
    ProbParams* d_prb = (ProbParams*)(sort_mem + o_prb);
    int64_t* d_roff = (int64_t*)(sort_mem + o_roff);
    int64_t* d_woff = (int64_t*)(sort_mem + o_woff);
    {
        const size_t pb = sizeof(ProbParams) * probs.size(), ob = sizeof(int64_t) * (probs.size() + 1);
        NUHT_CK(g_stage_out.reserve(pb + 2 * ob));
        std::memcpy(g_stage_out.p, probs.data(), pb);
        int64_t* ro = (int64_t*)(g_stage_out.p + pb);
        int64_t* wo = ro + probs.size() + 1;
        for (int i = 0; i < nprob; ++i) { ro[i] = probs[i].r_off; wo[i] = probs[i].w_off; }
        ro[nprob] = n;
        wo[nprob] = m;
        NUHT_CK(cudaMemcpyAsync(d_prb, g_stage_out.p, pb, cudaMemcpyHostToDevice, s));
        NUHT_CK(cudaMemcpyAsync(d_roff, ro, ob, cudaMemcpyHostToDevice, s));
        NUHT_CK(cudaMemcpyAsync(d_woff, wo, ob, cudaMemcpyHostToDevice, s));
    }
    double* r_s = (double*)(sort_mem + o_r);
    double* w_s = (double*)(sort_mem + o_w);
    int32_t* pr = (int32_t*)(sort_mem + o_pr);
    int32_t* pw = (int32_t*)(sort_mem + o_pw);
    int32_t* stair = (int32_t*)(sort_mem + o_st);
    if (src) {
        // already checked and sorted: one copy of the source's arrays per problem
        for (int ip = 0; ip < nprob; ++ip) {
            const ProbParams& q = probs[ip];
            if (q.n) {
                NUHT_CK(cudaMemcpyAsync(r_s + q.r_off, src->d_r, sizeof(double) * q.n, cudaMemcpyDeviceToDevice, s));
                NUHT_CK(cudaMemcpyAsync(pr + q.r_off, src->d_pr, sizeof(int32_t) * q.n, cudaMemcpyDeviceToDevice, s));
            }
            if (q.m) {
                NUHT_CK(cudaMemcpyAsync(w_s + q.w_off, src->d_w, sizeof(double) * q.m, cudaMemcpyDeviceToDevice, s));
                NUHT_CK(cudaMemcpyAsync(pw + q.w_off, src->d_pw, sizeof(int32_t) * q.m, cudaMemcpyDeviceToDevice, s));
            }
        }
    } else {
    NUHT_CK(launch_check_domain(r, n, d_flag, s));
    NUHT_CK(launch_check_domain(omega, m, d_flag + 1, s));
    // the two sorts are independent: omega on the auxiliary stream
    {
        Aux* ax = nullptr;
        NUHT_CK(aux_stream(&ax));
        NUHT_CK(cudaEventRecord(ax->fork, s));
        NUHT_CK(cudaStreamWaitEvent(ax->s, ax->fork, 0));
        const cudaError_t ew = radix_sort_f64(omega, m, w_s, pw, sort_mem + o_scr_w, scr_w, ax->s, d_woff, nprob);
        const cudaError_t ej = cudaEventRecord(ax->join, ax->s);
        const cudaError_t er = radix_sort_f64(r, n, r_s, pr, sort_mem + o_scr, scr, s, d_roff, nprob);
        // join before anything can free the sort memory
        const cudaError_t ek = ej == cudaSuccess ? cudaStreamWaitEvent(s, ax->join, 0) : cudaStreamSynchronize(ax->s);
        NUHT_CK(ew);
        NUHT_CK(ej);
        NUHT_CK(er);
        NUHT_CK(ek);
    }
    }
    if (nprob == 1) NUHT_CK(launch_staircase(r_s, n, w_s, m, probs[0].z, stair, s));
    else NUHT_CK(launch_staircase_many(r_s, w_s, m, d_prb, nprob, stair, s));
    // ---- subdivision (Algorithm 1) and work lists, on the device ------------
    SubBlk* d_out = (SubBlk*)(sort_mem + o_out);
    int64_t* d_res = (int64_t*)(sort_mem + o_res);
    double* d_bl = (double*)(sort_mem + o_bl);
    double4* d_ba = (double4*)(sort_mem + o_ba);
    NUHT_CK(launch_subdivide(stair, r_s, w_s, d_prb, nprob, P->opt.min_size, P->opt.n_split_cand,
                             (SubBlk*)(sort_mem + o_qa), (SubBlk*)(sort_mem + o_qb), qcap, d_out, ocap, d_res,
                             (int4*)(sort_mem + o_ctot), (int64_t*)(sort_mem + o_gst), sub_ctas, s));
    NUHT_CK(launch_block_bounds(d_out, d_out + ocap, d_res, d_prb, r_s, w_s, d_bl, d_ba, s));
    P->eval_threads = local_eval_threads(P->ntop_max);
    const int sp_tile = P->opt.spread_tile ? P->opt.spread_tile : spread_tile_points(P->qmax);
    P->spread_threads = sp_tile;
    BlockBuild bb{};
    bb.res = d_res;
    bb.sub = d_out;
    bb.ocap = ocap;
    bb.bl = d_bl;
    bb.ba = d_ba;
    bb.probs = d_prb;
    bb.w = P->w;
    bb.mom_tile = kMomentTile;
    bb.eval_tile = P->eval_threads;
    bb.spread_tile = sp_tile;
    P->interp_threads = P->opt.interp_tile ? P->opt.interp_tile : kInterpTileMax;
    bb.interp_tile = P->interp_threads;
    bind_build_temps(bb, sort_mem, bt);
    int64_t* bb_scan = (int64_t*)(sort_mem + bt.scan);
    char* tmp_mem = nullptr;   // temporaries of the host fallback
    struct FreeTmp {
        char** p; cudaStream_t s;
        ~FreeTmp() { pool_free(*p, s); }
    } free_tmp{&tmp_mem, s};
    NUHT_CK(cudaMemsetAsync(bb.totals, 0, sizeof(int64_t) * (kTotals + 0), s));
    NUHT_CK(cudaMemsetAsync(bb.maxv, 0, sizeof(int64_t) * kMaxv, s));
    NUHT_CK(launch_block_build(bb, bb_scan, s));
    // the one wait of the build: flags, counts, totals and maxima to the host
    const size_t o_hf = 0, o_hr = 64, o_ht = o_hr + 64, o_hm = o_ht + align256(sizeof(int64_t) * kTotals);
    NUHT_CK(g_stage_in.reserve(o_hm + 256));
    int* hflag = (int*)(g_stage_in.p + o_hf);
    int64_t* hres = (int64_t*)(g_stage_in.p + o_hr);
    int64_t* htot = (int64_t*)(g_stage_in.p + o_ht);
    int64_t* hmax = (int64_t*)(g_stage_in.p + o_hm);
    auto fetch_results = [&]() -> cudaError_t {
        cudaError_t e = cudaMemcpyAsync(hflag, d_flag, sizeof(int) * 2, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hres, bb.res, sizeof(int64_t) * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(htot, bb.totals, sizeof(int64_t) * kTotals, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hmax, bb.maxv, sizeof(int64_t) * kMaxv, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        return e;
    };
    NUHT_CK(fetch_results());
    if (hflag[0] || hflag[1]) return NUHT_ERR_DOMAIN;
    P->plan_ms[0] = ms_since(clk);
    if (hres[3]) {
        // list capacity exceeded: sorted values and staircase to the host,
        // Algorithm 1 there, the lists back to the device, the build again
        const size_t in_bytes = align256(sizeof(double) * n) + align256(sizeof(double) * m) +
                                align256(sizeof(int32_t) * m);
        std::vector<char> hbuf(in_bytes);
        double* hr = (double*)hbuf.data();
        double* hw = (double*)((char*)hr + align256(sizeof(double) * n));
        int32_t* hst = (int32_t*)((char*)hw + align256(sizeof(double) * m));
        if (n) NUHT_CK(cudaMemcpyAsync(hr, r_s, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
        if (m) NUHT_CK(cudaMemcpyAsync(hw, w_s, sizeof(double) * m, cudaMemcpyDeviceToHost, s));
        if (m) NUHT_CK(cudaMemcpyAsync(hst, stair, sizeof(int32_t) * m, cudaMemcpyDeviceToHost, s));
        NUHT_CK(cudaStreamSynchronize(s));
        std::vector<SubBlk> hl[3];
        std::vector<double> hbl;
        std::vector<double4> hba;
        std::vector<HBlock> lb, ab, db;
        for (int ip = 0; ip < nprob; ++ip) {
            const ProbParams& q = probs[ip];
            subdivide(hst + q.w_off, hr + q.r_off, hw + q.w_off, q.n, q.m, P->opt.min_size, P->opt.n_split_cand,
                      lb, ab, db);
            const std::vector<HBlock>* src[3] = {&lb, &ab, &db};
            {
                // the host walk's lists are checked before they reach the device
                std::vector<int64_t> rg;
                std::vector<int32_t> cl;
                for (int c = 0; c < 3; ++c)
                    for (const HBlock& h : *src[c]) {
                        rg.insert(rg.end(), {h.k0, h.k1, h.j0, h.j1});
                        cl.push_back(c);
                    }
                if (!check_blocks(hr + q.r_off, q.n, hw + q.w_off, q.m, q.z, P->opt.min_size, rg.data(), cl.data(),
                                  (int64_t)cl.size()))
                    return NUHT_ERR_BAD_BLOCKS;
            }
            for (int c = 0; c < 3; ++c)
                for (const HBlock& h : *src[c]) {
                    hl[c].push_back(SubBlk{(int32_t)h.k0, (int32_t)h.k1, (int32_t)h.j0, (int32_t)h.j1, ip});
                    if (c == 0) hbl.push_back(hr[q.r_off + h.j1]);
                    if (c == 1)
                        hba.push_back(make_double4(hr[q.r_off + h.j0], hr[q.r_off + h.j1], hw[q.w_off + h.k0],
                                                   hw[q.w_off + h.k1]));
                }
        }
        int64_t cap = 1;
        for (int c = 0; c < 3; ++c) cap = (int64_t)hl[c].size() > cap ? (int64_t)hl[c].size() : cap;
        Arena ta;
        const size_t t_sub = ta.reserve<SubBlk>(3 * cap), t_bl = ta.reserve<double>(cap);
        const size_t t_ba = ta.reserve<double4>(cap), t_res = ta.reserve<int64_t>(4);
        BuildTemps tt = reserve_build_temps(ta, cap);
        NUHT_CK(pool_alloc((void**)&tmp_mem, ta.size, s));
        std::vector<char> up(t_res + 64, 0);
        for (int c = 0; c < 3; ++c)
            if (!hl[c].empty()) std::memcpy(up.data() + t_sub + sizeof(SubBlk) * c * cap, hl[c].data(),
                                            sizeof(SubBlk) * hl[c].size());
        if (!hbl.empty()) std::memcpy(up.data() + t_bl, hbl.data(), sizeof(double) * hbl.size());
        if (!hba.empty()) std::memcpy(up.data() + t_ba, hba.data(), sizeof(double4) * hba.size());
        int64_t* ures = (int64_t*)(up.data() + t_res);
        ures[0] = (int64_t)hl[0].size(); ures[1] = (int64_t)hl[1].size(); ures[2] = (int64_t)hl[2].size(); ures[3] = 0;
        NUHT_CK(cudaMemcpyAsync(tmp_mem, up.data(), t_res + sizeof(int64_t) * 4, cudaMemcpyHostToDevice, s));
        bb.res = (const int64_t*)(tmp_mem + t_res);
        bb.sub = (const SubBlk*)(tmp_mem + t_sub);
        bb.ocap = cap;
        bb.bl = (const double*)(tmp_mem + t_bl);
        bb.ba = (const double4*)(tmp_mem + t_ba);
        bind_build_temps(bb, tmp_mem, tt);
        bb_scan = (int64_t*)(tmp_mem + tt.scan);
        NUHT_CK(cudaMemsetAsync(bb.totals, 0, sizeof(int64_t) * kTotals, s));
        NUHT_CK(cudaMemsetAsync(bb.maxv, 0, sizeof(int64_t) * kMaxv, s));
        NUHT_CK(launch_block_build(bb, bb_scan, s));
        NUHT_CK(fetch_results());   // (the upload buffer lives until here)
    }
    if (hmax[MX_ERR]) return NUHT_ERR_UNSUPPORTED;
    const int64_t nl = hres[0], na = hres[1], nd = hres[2];
    const int64_t* tl = htot + TOT_LOCAL;
    const int64_t* ta_ = htot + TOT_ASY;
    P->n_loc = (int)nl; P->n_asy = (int)na; P->n_dir = (int)nd;
    P->mom_len = tl[LC_MOM];
    P->n_tmom = (int)tl[LC_TMOM]; P->n_teval = (int)tl[LC_TEVAL];
    P->local_rc = tl[LC_RC];
    P->gb_len = ta_[AC_GB]; P->gq_len = ta_[AC_GQ];
    P->n_tspread = (int)ta_[AC_TSPREAD]; P->n_tinterp = (int)ta_[AC_TINTERP];
    P->n_fblock = (int)ta_[AC_IFK]; P->n_fsmall = (int)ta_[AC_IFS];
    P->n_fa = (int)ta_[AC_IFA]; P->n_fb = (int)ta_[AC_IFB];
    P->asy_rc = ta_[AC_RC]; P->fft_points = ta_[AC_NF2];
    P->direct_entries = htot[TOT_DIR + DC_ENTRIES];
    P->max_dir_rows = (int)hmax[MX_DIR_ROWS]; P->max_dir_cols = (int)hmax[MX_DIR_COLS];
    P->max_dir_area = (int)hmax[MX_DIR_AREA];
    P->max_nf2_small = (int)hmax[MX_NF2_SMALL];
    P->max_fblock_pts = (int)hmax[MX_FBLOCK_PTS];
    P->has_large_fft = hmax[MX_LARGE] != 0;
    const int64_t nseg[kLists] = {nl, nl, na, na, ta_[AC_NFS], ta_[AC_NFL], ta_[AC_NFL], ta_[AC_NFK]};
    const int64_t ntile[kLists] = {tl[LC_TMOM], tl[LC_TEVAL], ta_[AC_TSPREAD], ta_[AC_TINTERP],
                                   ta_[AC_IFS], ta_[AC_IFA], ta_[AC_IFB], ta_[AC_IFK]};
    P->plan_ms[1] = ms_since(clk);

    // ---- one device arena for everything the plan keeps -------------------
    const HostTables& T = kernel_tables(P->w);
    Arena A;
    size_t a_prob = A.reserve<ProbParams>(probs.size());
    size_t a_es = A.reserve<double>(T.es.size()), a_ph = A.reserve<double>(T.ph.size());
    size_t a_es2 = A.reserve<float2>(T.es2.size()), a_ph2 = A.reserve<float2>(T.ph2.size());
    size_t a_ch2 = A.reserve<float2>(T.ch2.size());
    size_t a_tw = A.reserve<double2>(T.tw.size()), a_tw2 = A.reserve<float4>(T.tw2.size());
    size_t host_part = A.size;   // everything above is uploaded from one staging buffer
    size_t a_loc = A.reserve<LocalBlock>(nl);
    size_t a_asy = A.reserve<AsyBlock>(na);
    size_t a_dir = A.reserve<DirectBlock>(nd);
    size_t a_blk = A.reserve<SubBlk>(nl + na + nd);
    size_t a_seg[kLists], a_pre[kLists], a_tile[kLists];
    for (int i = 0; i < kLists; ++i) {
        a_seg[i] = A.reserve<Seg>(nseg[i]);
        a_pre[i] = A.reserve<int32_t>(nseg[i] + 1);
        a_tile[i] = A.reserve<Tile>(ntile[i]);
    }
    size_t a_r = A.reserve<double>(n), a_w = A.reserve<double>(m);
    size_t a_pr = A.reserve<int32_t>(n), a_pw = A.reserve<int32_t>(m);
    // G >= 2 copies (a pair, or a vector group) of the per-component arrays:
    // sorted coefficients, moments and sorted outputs
    const size_t gcopies = (size_t)group_copies(P);
    size_t a_mom = A.reserve<double>(gcopies * (size_t)P->mom_len);
    // Members of one asymptotic launch: up to a group's components share each
    // point's and frequency's cell, basis and phase in the FP64 spreading and
    // interpolation kernels, given their own spreading grid and FFT output,
    // as long as the extra grids stay within kAsyMemberBytes.
    {
        const size_t per = sizeof(double2) * (size_t)P->gb_len + sizeof(float4) * (size_t)P->gq_len;
        int am = P->opt.deterministic ? 1 : group_size(P);
        while (am > 1 && (size_t)(am - 1) * per > kAsyMemberBytes) --am;
        P->asy_members = am;
    }
    size_t a_gb = A.reserve<double2>((size_t)P->asy_members * (size_t)P->gb_len);
    size_t a_gq = A.reserve<float4>((size_t)P->asy_members * (size_t)P->gq_len);
    size_t a_gt = A.reserve<float4>(P->has_large_fft ? (size_t)P->gq_len : 1);
    size_t a_cs = A.reserve<double>(gcopies * (size_t)n), a_gs = A.reserve<double>(gcopies * (size_t)m);
    size_t a_r2 = A.reserve<float2>(n), a_w2 = A.reserve<float2>(m);
    size_t a_cs2 = A.reserve<float2>(gcopies * (size_t)n);
    size_t a_tg = A.reserve<double2>((size_t)P->asy_members * (size_t)P->gq_len);
    size_t a_bq = A.reserve<float4>((size_t)P->asy_members * (size_t)P->gb_len);
    size_t a_sm = A.reserve<int32_t>((size_t)ntile[LIST_SPREAD]);
    const bool det = P->opt.deterministic != 0;
    const size_t f1 = 1;
    size_t a_fgs = A.reserve<Fx128>(det ? (size_t)m : f1), a_fgsb = A.reserve<Fx128>(det ? (size_t)m : f1);
    size_t a_fcs = A.reserve<Fx128>(det ? (size_t)n : f1), a_fcsb = A.reserve<Fx128>(det ? (size_t)n : f1);
    size_t a_fmom = A.reserve<Fx128>(det ? (size_t)P->mom_len : f1);
    size_t a_fmomb = A.reserve<Fx128>(det ? (size_t)P->mom_len : f1);
    size_t a_fgb = A.reserve<Fx128>(det ? 2 * (size_t)P->gb_len : f1);
    size_t a_ftg = A.reserve<Fx128>(det ? 2 * (size_t)P->gq_len : f1);
    size_t a_mx = A.reserve<unsigned long long>(1);
    size_t a_q = A.reserve<int>((size_t)nl + 2), a_status = A.reserve<int>(1);
    NUHT_CK(pool_alloc((void**)&P->dmem, A.size, s));
    P->dbytes = A.size;
    char* D = P->dmem;
    NUHT_CK(g_stage_out.reserve(host_part));
    char* stage = g_stage_out.p;
    auto put = [&](size_t off, const void* src, size_t bytes) {
        if (bytes) std::memcpy(stage + off, src, bytes);
    };
    // Rounding budget of the FP32 tiers.  Each tier below (the taps'
    // polynomial degrees, the spreading moments' degrees, the q-fold's
    // moments, the interpolation's degrees and its per-pair cut) keeps its
    // rounding bound -- a bound relative to the sum of magnitudes, far above
    // the typical rounding -- below kRoundBudget eps.  A point or frequency
    // meets at most four of them, so together they stay below eps / 2, beside
    // the expansions' truncation of at most eps per entry (Lemma 3.1, Sec. 3.2
    // eq. asy-error) and inside the 10 eps ||c||_1 contract.
    constexpr double kRoundBudget = 0.1;
    // Per Hankel pair, the degrees of the interpolation's per-bin and
    // per-frequency sums that need double-float: term q enters g with weight
    // at most |a_q| z^-q, so degree d may round in FP32 once the rounding bound
    // of the degrees from d on (as for tab.dci, whose weight is one) times the
    // pair's larger weight stays below kRoundBudget eps.
    {
        const int nc = T.deg + 1;
        std::vector<double> colsum(nc, 0.0);
        for (int i = 0; i < T.w; ++i)
            for (int d = 0; d < nc; ++d) colsum[d] += std::fabs(T.ch[(size_t)i * nc + d]);
        for (ProbParams& pp : probs)
            for (int pr = 0; pr < kMaxQ / 2; ++pr) {
                double wmax = 0.0;
                for (int q = 2 * pr; q < 2 * pr + 2 && q < pp.Q; ++q)
                    wmax = std::max(wmax, std::fabs(pp.a[q] * std::pow(pp.z, -q)));
                int d = nc;
                double acc = 0.0;
                while (d > 2) {
                    acc += colsum[d - 1] * (d + 2) * 5.9604644775390625e-08;
                    if (acc * wmax <= kRoundBudget * P->eps) --d; else break;
                }
                pp.dcp[pr] = (int8_t)d;
            }
    }
    for (ProbParams& q : probs) q.tw2 = (const float4*)(D + a_tw2);
    put(a_prob, probs.data(), sizeof(ProbParams) * probs.size());
    put(a_es, T.es.data(), sizeof(double) * T.es.size());
    put(a_es2, T.es2.data(), sizeof(float2) * T.es2.size());
    put(a_ch2, T.ch2.data(), sizeof(float2) * T.ch2.size());
    put(a_ph, T.ph.data(), sizeof(double) * T.ph.size());
    put(a_ph2, T.ph2.data(), sizeof(float2) * T.ph2.size());
    put(a_tw, T.tw.data(), sizeof(double2) * T.tw.size());
    put(a_tw2, T.tw2.data(), sizeof(float4) * T.tw2.size());
    P->plan_ms[2] = ms_since(clk);
    NUHT_CK(cudaMemcpyAsync(D, stage, host_part, cudaMemcpyHostToDevice, s));
    {
        Aux* ax = nullptr;
        NUHT_CK(aux_stream(&ax));
        NUHT_CK(cudaEventRecord(ax->stage_done, s));   // the next build waits on it before reusing the buffer
        g_stage_out_event = ax->stage_done;
    }
    BuildLists bl{};
    bl.loc = (LocalBlock*)(D + a_loc);
    bl.asy = (AsyBlock*)(D + a_asy);
    bl.dir = (DirectBlock*)(D + a_dir);
    bl.blk = (SubBlk*)(D + a_blk);
    for (int i = 0; i < kLists; ++i) {
        bl.seg[i] = (Seg*)(D + a_seg[i]);
        bl.pre[i] = (int32_t*)(D + a_pre[i]);
    }
    NUHT_CK(launch_block_fill(bb, bl, s));
    Tile* tiles[kLists];
    for (int i = 0; i < kLists; ++i) {
        tiles[i] = (Tile*)(D + a_tile[i]);
        NUHT_CK(launch_expand_tiles(bl.seg[i], bl.pre[i], (int)nseg[i], (int)ntile[i], tiles[i], s));
    }
    P->d_tmom = tiles[LIST_MOM]; P->d_teval = tiles[LIST_EVAL];
    P->d_tspread = tiles[LIST_SPREAD]; P->d_tinterp = tiles[LIST_INTERP];
    P->d_fsmall = tiles[LIST_FSMALL]; P->d_fa = tiles[LIST_FA]; P->d_fb = tiles[LIST_FB];
    P->d_fblock = tiles[LIST_FBLOCK];
    P->d_pre_mom = bl.pre[LIST_MOM];
    P->d_blk = bl.blk;
    // sorted arrays and permutations stay on the device
    P->d_r = (double*)(D + a_r); P->d_w = (double*)(D + a_w);
    P->d_pr = (int32_t*)(D + a_pr); P->d_pw = (int32_t*)(D + a_pw);
    if (n) {
        NUHT_CK(cudaMemcpyAsync(P->d_r, r_s, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        NUHT_CK(cudaMemcpyAsync(P->d_pr, pr, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
    }
    if (m) {
        NUHT_CK(cudaMemcpyAsync(P->d_w, w_s, sizeof(double) * m, cudaMemcpyDeviceToDevice, s));
        NUHT_CK(cudaMemcpyAsync(P->d_pw, pw, sizeof(int32_t) * m, cudaMemcpyDeviceToDevice, s));
    }
    P->d_prob = (ProbParams*)(D + a_prob);
    P->d_loc = bl.loc;
    P->d_asy = bl.asy;
    P->d_dir = bl.dir;
    P->d_es = (double*)(D + a_es); P->d_ph = (double*)(D + a_ph); P->d_tw = (double2*)(D + a_tw);
    P->d_mom = (double*)(D + a_mom); P->d_momb = P->d_mom + P->mom_len;
    P->d_gb = (double2*)(D + a_gb); P->d_gq = (float4*)(D + a_gq); P->d_gtmp = (float4*)(D + a_gt);
    P->d_cs = (double*)(D + a_cs); P->d_gs = (double*)(D + a_gs);
    P->d_r2 = (float2*)(D + a_r2); P->d_w2 = (float2*)(D + a_w2); P->d_cs2 = (float2*)(D + a_cs2);
    P->d_csb = P->d_cs + n; P->d_gsb = P->d_gs + m; P->d_cs2b = P->d_cs2 + n;
    P->det = det;
    if (det) {
        P->f_gs = (Fx128*)(D + a_fgs); P->f_gsb = (Fx128*)(D + a_fgsb);
        P->f_cs = (Fx128*)(D + a_fcs); P->f_csb = (Fx128*)(D + a_fcsb);
        P->f_mom = (Fx128*)(D + a_fmom); P->f_momb = (Fx128*)(D + a_fmomb);
        P->f_gb = (Fx128*)(D + a_fgb); P->f_tg = (Fx128*)(D + a_ftg);
    }
    P->d_mx = (unsigned long long*)(D + a_mx);
    P->d_q = (int*)(D + a_q);
    P->d_status = (int*)(D + a_status);
    NUHT_CK(cudaMemsetAsync(P->d_status, 0, sizeof(int), s));
    NUHT_CK(launch_split_f64(P->d_r, n, P->d_r2, s));
    NUHT_CK(launch_split_f64(P->d_w, m, P->d_w2, s));
    P->d_tg = (double2*)(D + a_tg); P->d_bq = (float4*)(D + a_bq);
    Tables& tb = P->tab;
    tb.es = P->d_es; tb.es2 = (const float2*)(D + a_es2);
    tb.w = T.w; tb.deg = T.deg; tb.half_w = 0.5 * T.w;
    // plain FP32 for the degrees whose coefficient tail T_k = max_taps sum_{k' > k} |c_k'|
    // keeps the FP32 rounding (2^-23 T_k) below kRoundBudget eps
    tb.deg_comp = T.deg;
    for (int k = T.deg - 1; k >= 0; --k) {
        double tail = 0.0;
        for (int i = 0; i < T.w; ++i) {
            double sum = 0.0;
            for (int kk = k + 1; kk <= T.deg; ++kk) sum += std::fabs(T.es[(size_t)i * (T.deg + 1) + kk]);
            tail = sum > tail ? sum : tail;
        }
        if (tail * 1.1920928955078125e-07 <= kRoundBudget * P->eps) tb.deg_comp = k; else break;
    }
    // Chebyshev form of the taps (moment paths): nb terms, dropping a tail
    // below 1e-3 eps; degrees >= dcs of the spreading moments accumulate in
    // FP32 over at most ceil(tile / 8) points each, degrees >= dci of the
    // interpolation sum in FP32, both with rounding below kRoundBudget eps.
    tb.ch2 = (const float2*)(D + a_ch2);
    {
        const int nc = T.deg + 1;
        std::vector<double> tailmax(nc + 1, 0.0), colsum(nc, 0.0);
        for (int i = 0; i < T.w; ++i) {
            double sum = 0.0;
            for (int d = nc - 1; d >= 0; --d) {
                const double a = std::fabs(T.ch[(size_t)i * nc + d]);
                sum += a;
                colsum[d] += a;
                tailmax[d] = sum > tailmax[d] ? sum : tailmax[d];
            }
        }
        int nb = nc;
        while (nb > 2 && tailmax[nb - 1] <= 1e-3 * P->eps) --nb;
        tb.nb = nb;
        const int nsub = (P->spread_threads + 7) / 8;
        int dcs = nb;
        while (dcs > 2 && tailmax[dcs - 1] * (nsub + nb) * 1.1920928955078125e-07 <= kRoundBudget * P->eps) --dcs;
        tb.dcs = dcs;
        int dci = nb;
        double acc = 0.0;
        while (dci > 2) {
            acc += colsum[dci - 1] * (dci + 2) * 5.9604644775390625e-08;
            if (acc <= kRoundBudget * P->eps) --dci; else break;
        }
        tb.dci = dci;
        // q-folded spreading: the weights' Chebyshev terms are kept down to
        // 1e-3 eps; a term above kRoundBudget eps / ((kMomFold + 2) 2^-23) multiplies
        // moments whose FP32 partial sums (kMomFold points) would show, so
        // those moments stay double-float
        tb.fold_tol = (float)(1e-3 * P->eps);
        tb.fold_df_tol = (float)(kRoundBudget * P->eps / ((kMomFold + 2) * 1.1920928955078125e-07));
    }
    tb.ph = P->d_ph; tb.ph2 = (const float2*)(D + a_ph2);
    tb.ph_pieces = T.ph_pieces; tb.ph_deg = T.ph_deg; tb.ph_comp = T.ph_comp;
    tb.interp_const = std::sqrt(2.0 / M_PI) * 4.0 / ((double)T.w * (double)T.w);
    tb.ic2 = make_float2((float)tb.interp_const, (float)(tb.interp_const - (double)(float)tb.interp_const));
    tb.ph_scale = T.ph_scale; tb.ph_xmax = T.ph_xmax;
    tb.ph_scale2 = make_float2((float)T.ph_scale, (float)(T.ph_scale - (double)(float)T.ph_scale));
    tb.tw = P->d_tw; tb.tw_log2 = T.tw_log2;
    tb.tw2 = (const float4*)(D + a_tw2);
    P->d_smode = (int32_t*)(D + a_sm);
    NUHT_CK(launch_spread_modes(P->d_prob, P->d_asy, P->d_tspread, P->n_tspread, tb, P->d_r, P->d_smode, s));
    P->plan_ms[3] = ms_since(clk);
    if (const char* ck = std::getenv("NUHT_CHECKED"))
        if (*ck && *ck != '0') NUHT_TRY_BUILD(verify_lists(P));
    return NUHT_OK;
}

// Orders, crossover, Hankel coefficients and precision split of one problem.
static int init_problem(ProbParams& pp, int nu, double eps, int m_terms, int64_t n, int64_t m,
                        int64_t r_off, int64_t w_off)
{
    if (nu > 100 || nu < -100) return NUHT_ERR_UNSUPPORTED;
    const int anu = nu < 0 ? -nu : nu;
    pp = ProbParams{};
    pp.nu = anu;
    pp.sgn = (nu < 0 && (anu & 1)) ? -1 : 1;
    pp.fxs = kFxOff;   // FP64 atomics; build_plan sets kFxScale for the deterministic mode
    int rc = choose_params(anu, eps, m_terms, &pp.M, &pp.z, &pp.L);
    if (rc != NUHT_OK) return rc;
    pp.Q = 2 * pp.M;
    const int hp = (anu & 1) ? (anu + 1) / 2 : anu / 2;
    pp.ntop = hp + pp.L;
    if (pp.ntop >= kMaxNtop) return NUHT_ERR_UNSUPPORTED;
    const double phi = -(2.0 * anu + 1.0) * M_PI / 4.0;
    pp.cphi = std::cos(phi);
    pp.sphi = std::sin(phi);
    {
        const float ch = (float)pp.cphi, sh = (float)pp.sphi;
        pp.cphi2 = make_float2(ch, (float)(pp.cphi - (double)ch));
        pp.sphi2 = make_float2(sh, (float)(pp.sphi - (double)sh));
    }
    // Term q of the Hankel sum is at most |a_q| z^-q times the leading one on an
    // asymptotic block (omega r > z).  Summing it in FP32 (relative error well
    // below 1e-6 of the sum of magnitudes) costs at most |a_q| z^-q 1e-6 of
    // ||c||_1; terms from qs on keep that below 1e-2 eps each.
    pp.qs = pp.Q;
    for (int q = pp.Q - 1; q >= 1; --q) {
        if (std::fabs(hankel_coeff(q, anu)) * std::pow(pp.z, -q) * 1e-6 <= 1e-2 * eps) pp.qs = q;
        else break;
    }
    // the kernels sum a_q (omega rho)^-q as (a_q z^-q) (z / (omega rho))^q: the
    // first factor stays in the FP32 range of the double-float parts (a_q alone
    // does not for large orders), the second is at most one
    for (int q = 0; q < kMaxQ; ++q) {
        pp.a[q] = q < pp.Q ? hankel_coeff(q, anu) : 0.0;
        const double as = pp.a[q] * std::pow(pp.z, -q);
        const float hi = (float)as;
        pp.a2[q] = make_float2(hi, (float)(as - (double)hi));
    }
    {
        const float zh = (float)pp.z;
        pp.z2 = make_float2(zh, (float)(pp.z - (double)zh));
    }
    pp.r_off = r_off; pp.w_off = w_off; pp.n = n; pp.m = m; pp.c_off = r_off; pp.g_off = w_off;
    return NUHT_OK;
}

static int check_opts(const nuht_opts* opt, nuht_opts& o)
{
    nuht_default_opts(&o);
    if (opt) o = *opt;
    if (o.min_size < 1 || o.min_size > NUHT_MAX_MIN_SIZE || o.n_split_cand < 2 || o.m_terms < 0 || o.m_terms > kMaxM ||
        (o.precision != NUHT_PREC_FP64 && o.precision != NUHT_PREC_MIXED))
        return NUHT_ERR_INVALID_ARG;
    if (o.reserved) return NUHT_ERR_INVALID_ARG;
    if (o.vec_group < 0 || o.vec_group > NUHT_MAX_VEC_GROUP) return NUHT_ERR_INVALID_ARG;
    if (o.vec_group > 2 && (o.deterministic || o.persistent)) return NUHT_ERR_INVALID_ARG;
    if (o.deterministic != 0 && o.deterministic != 1) return NUHT_ERR_INVALID_ARG;
    if (o.persistent != 0 && o.persistent != 1) return NUHT_ERR_INVALID_ARG;
    if (o.interp_tile != 0 && o.interp_tile != 128 && o.interp_tile != 256) return NUHT_ERR_INVALID_ARG;
    if (o.spread_tile != 0 && (o.spread_tile < 64 || o.spread_tile > 256 || o.spread_tile % 32))
        return NUHT_ERR_INVALID_ARG;
    if (o.timing < NUHT_TIMING_OFF || o.timing > NUHT_TIMING_SERIAL) return NUHT_ERR_INVALID_ARG;
    return NUHT_OK;
}

int nuht_plan(nuht_plan_t* out, int nu, const double* r, int64_t n, const double* omega, int64_t m,
              double eps, const nuht_opts* opt, void* stream)
{
    if (!out) return NUHT_ERR_INVALID_ARG;
    *out = nullptr;
    if (n < 0 || m < 0 || n > 0x7fffffffLL || m > 0x7fffffffLL) return NUHT_ERR_INVALID_ARG;
    if (!(eps >= 1e-15 && eps <= 1e-1)) return NUHT_ERR_INVALID_ARG;
    if ((n > 0 && !r) || (m > 0 && !omega)) return NUHT_ERR_INVALID_ARG;
    if (nu > 100 || nu < -100) return NUHT_ERR_UNSUPPORTED;
    nuht_opts o;
    int rc = check_opts(opt, o);
    if (rc != NUHT_OK) return rc;
    if (o.precision == NUHT_PREC_MIXED && eps < 1e-6) return NUHT_ERR_UNSUPPORTED;
    nuht_plan_t P = new (std::nothrow) nuht_plan_s();
    if (!P) return NUHT_ERR_NOMEM;
    P->nu_user = nu;
    P->eps = eps;
    P->opt = o;
    P->n = n;
    P->m = m;
    P->stream = (cudaStream_t)stream;
    P->probs.resize(1);
    rc = init_problem(P->probs[0], nu, eps, o.m_terms, n, m, 0, 0);
    if (rc != NUHT_OK) { delete P; return rc; }
    P->w = nufft_width(eps);
    rc = build_plan(P, r, omega);
    if (rc != NUHT_OK) { nuht_destroy(P); return rc; }
    *out = P;
    return NUHT_OK;
}

int nuht_plan_many(nuht_plan_t* out, int nprob, const int* nu, const double* r, const int64_t* n,
                   const double* omega, const int64_t* m, double eps, const nuht_opts* opt, void* stream)
{
    if (!out) return NUHT_ERR_INVALID_ARG;
    *out = nullptr;
    if (nprob < 1 || nprob > 65536 || !nu || !n || !m) return NUHT_ERR_INVALID_ARG;
    if (!(eps >= 1e-15 && eps <= 1e-1)) return NUHT_ERR_INVALID_ARG;
    int64_t nt = 0, mt = 0;
    for (int i = 0; i < nprob; ++i) {
        if (n[i] < 0 || m[i] < 0) return NUHT_ERR_INVALID_ARG;
        if (nu[i] > 100 || nu[i] < -100) return NUHT_ERR_UNSUPPORTED;
        nt += n[i];
        mt += m[i];
    }
    if (nt > 0x7fffffffLL || mt > 0x7fffffffLL) return NUHT_ERR_INVALID_ARG;
    if ((nt > 0 && !r) || (mt > 0 && !omega)) return NUHT_ERR_INVALID_ARG;
    nuht_opts o;
    int rc = check_opts(opt, o);
    if (rc != NUHT_OK) return rc;
    if (o.precision == NUHT_PREC_MIXED && eps < 1e-6) return NUHT_ERR_UNSUPPORTED;
    nuht_plan_t P = new (std::nothrow) nuht_plan_s();
    if (!P) return NUHT_ERR_NOMEM;
    P->nu_user = nu[0];
    P->eps = eps;
    P->opt = o;
    P->n = nt;
    P->m = mt;
    P->stream = (cudaStream_t)stream;
    P->probs.resize(nprob);
    int64_t ro = 0, wo = 0;
    for (int i = 0; i < nprob; ++i) {
        rc = init_problem(P->probs[i], nu[i], eps, o.m_terms, n[i], m[i], ro, wo);
        if (rc != NUHT_OK) { delete P; return rc; }
        ro += n[i];
        wo += m[i];
    }
    P->w = nufft_width(eps);
    rc = build_plan(P, r, omega);
    if (rc != NUHT_OK) { nuht_destroy(P); return rc; }
    *out = P;
    return NUHT_OK;
}

#define NUHT_TRY(x)                   \
    do {                              \
        int rc_ = (x);                \
        if (rc_ != NUHT_OK) return rc_; \
    } while (0)

// Accumulation targets of the kernels: the FP64 array, or in the
// deterministic mode its exact fixed-point twin (passed under the same
// pointer type; the kernels index it by element through Accum).
static double* acc_target(nuht_plan_t P, double* f64, Fx128* fx) { return P->det ? (double*)fx : f64; }
static size_t acc_bytes(nuht_plan_t P, int64_t count) { return (size_t)count * (P->det ? sizeof(Fx128) : sizeof(double)); }

// Sorted coefficients and sums of member v of a group (the accumulation
// target of the sums: d_gs + v m, or in the deterministic mode, where groups
// are pairs, f_gs / f_gsb).
static float2* member_c2(nuht_plan_t P, int v) { return P->d_cs2 + (int64_t)v * P->n; }
static double* member_c(nuht_plan_t P, int v) { return P->d_cs + (int64_t)v * P->n; }
static double* member_g(nuht_plan_t P, int v) { return P->d_gs + (int64_t)v * P->m; }
static double* member_g_acc(nuht_plan_t P, int v)
{
    if (P->det) return (double*)(v == 0 ? P->f_gs : P->f_gsb);
    return member_g(P, v);
}

// Algorithm 2 on the device for the ng real components c0 .. c0 + ng - 1 of a
// group (sorted, scaled coefficients in member_c / member_c2): every block
// class adds into the members' sums (sorted order, FP64 atomics).  The local
// and direct blocks are applied to the whole group at once, with one Bessel
// evaluation for all members (the pair kernels for ng <= 2, the group
// kernels above); the asymptotic type-3 pipeline runs per member.
static int apply_forward(nuht_plan_t P, int c0, int ng, cudaStream_t s)
{
    const int mask = P->opt.class_mask;
    StageTimer T{P, c0};
    double* gs = member_g_acc(P, 0);
    double* gsb = ng == 2 ? member_g_acc(P, 1) : nullptr;
    double* mom_acc = acc_target(P, P->d_mom, P->f_mom);
    double* momb_acc = acc_target(P, P->d_momb, P->f_momb);
    double2* gb_acc = (double2*)acc_target(P, (double*)P->d_gb, P->f_gb);
    const bool loc = (mask & 1) && P->n_loc, dir = (mask & 4) && P->n_dir;
    const bool asy = (mask & 2) && P->n_asy;
    const bool group = ng > 2;
    // The block classes share no scratch and only add into g (FP64 atomics):
    // the local and direct blocks run beside the asymptotic pipeline (ClassFork),
    // each stage's events on its own stream.  NUHT_TIMING_SERIAL keeps every
    // stage in order on s, so that each stage's time is its own.
    ClassFork fk;
    if (P->opt.timing != NUHT_TIMING_SERIAL && asy && (loc || dir)) NUHT_CK(fk.open(s));
    const cudaStream_t ls = fk.local(s), as = fk.asy(s);
    if (loc && group) {
        NUHT_TRY(T.begin(NUHT_STAGE_LOCAL_MOMENTS, ls));
        NUHT_CK(cudaMemsetAsync(P->d_mom, 0, sizeof(double) * P->mom_len * ng, ls));
        NUHT_CK(launch_local_moments_group(P->d_prob, P->d_loc, P->d_tmom, P->n_tmom, P->lmax, P->d_r2,
                                           P->d_cs2, P->n, ng, P->d_mom, P->mom_len, ls));
        NUHT_TRY(T.end(NUHT_STAGE_LOCAL_MOMENTS, ls));
        NUHT_TRY(T.begin(NUHT_STAGE_LOCAL_EVAL, ls));
        NUHT_CK(launch_local_eval_group(P->d_prob, P->d_loc, P->d_teval, P->n_teval, P->ntop_max,
                                        P->eval_threads, P->d_w2, P->d_mom, P->mom_len, ng, P->d_gs, P->m, ls));
        NUHT_TRY(T.end(NUHT_STAGE_LOCAL_EVAL, ls));
    } else if (loc && P->opt.persistent && !P->det) {
        // moments and evaluation in one persistent launch (per-block waits)
        NUHT_TRY(T.begin(NUHT_STAGE_LOCAL_MOMENTS, ls));
        double* momb = ng == 2 ? P->d_momb : nullptr;
        NUHT_CK(cudaMemsetAsync(P->d_mom, 0, sizeof(double) * P->mom_len, ls));
        if (momb) NUHT_CK(cudaMemsetAsync(momb, 0, sizeof(double) * P->mom_len, ls));
        const char* st = std::getenv("NUHT_QUEUE_STALL");
        const bool stall = st && *st && *st != '0';
        NUHT_CK(launch_local_persistent(P->d_prob, P->d_loc, P->d_tmom, P->n_tmom, P->d_teval, P->n_teval,
                                        P->d_pre_mom, P->lmax, P->ntop_max, P->eval_threads, P->d_r2, P->d_cs2,
                                        P->d_cs2b, P->d_w2, P->d_mom, momb, gs, gsb, P->d_q,
                                        P->n_loc, P->d_status, stall ? 4096 : (1 << 22), stall ? 1 : 0, ls));
        NUHT_TRY(T.end(NUHT_STAGE_LOCAL_MOMENTS, ls));
    } else if (loc) {
        NUHT_TRY(T.begin(NUHT_STAGE_LOCAL_MOMENTS, ls));
        NUHT_CK(cudaMemsetAsync(mom_acc, 0, acc_bytes(P, P->mom_len), ls));
        // a pair's moments in one pass (one Chebyshev recurrence per point for
        // both components) when its accumulators fit, else a second launch (the
        // group kernel at G = 2 was measured slower on the complex n = m = 4e6
        // workload: 5.68 against 5.38 ms per execute)
        double* momb = ng == 2 ? P->d_momb : nullptr;
        if (momb) NUHT_CK(cudaMemsetAsync(momb_acc, 0, acc_bytes(P, P->mom_len), ls));
        if (momb && local_moments2_fits(P->lmax)) {
            NUHT_CK(launch_local_moments2(P->d_prob, P->d_loc, P->d_tmom, P->n_tmom, P->lmax, P->d_r2,
                                          P->d_cs2, P->d_cs2b, mom_acc, momb_acc, ls));
        } else {
            NUHT_CK(launch_local_moments(P->d_prob, P->d_loc, P->d_tmom, P->n_tmom, P->lmax, P->d_r2,
                                         P->d_cs2, mom_acc, ls));
            if (momb)
                NUHT_CK(launch_local_moments(P->d_prob, P->d_loc, P->d_tmom, P->n_tmom, P->lmax, P->d_r2,
                                             P->d_cs2b, momb_acc, ls));
        }
        if (P->det) NUHT_CK(launch_fx_decode(P->f_mom, P->d_mom, P->mom_len, P->d_prob, ls));
        if (momb && P->det) NUHT_CK(launch_fx_decode(P->f_momb, P->d_momb, P->mom_len, P->d_prob, ls));
        NUHT_TRY(T.end(NUHT_STAGE_LOCAL_MOMENTS, ls));
        NUHT_TRY(T.begin(NUHT_STAGE_LOCAL_EVAL, ls));
        if (P->opt.precision == NUHT_PREC_MIXED)
            NUHT_CK(launch_local_eval_f32(P->d_prob, P->d_loc, P->d_teval, P->n_teval, P->ntop_max,
                                          P->eval_threads, P->d_w2, P->d_mom, gs, momb, gsb, ls));
        else
            NUHT_CK(launch_local_eval(P->d_prob, P->d_loc, P->d_teval, P->n_teval, P->ntop_max,
                                      P->nu_max > 0, P->eval_threads, P->d_w2, P->d_mom, gs, momb, gsb, ls));
        NUHT_TRY(T.end(NUHT_STAGE_LOCAL_EVAL, ls));
    }
    if (dir) {
        NUHT_TRY(T.begin(NUHT_STAGE_DIRECT, ls));
        const int mode = direct_sum_mode(P->eps, P->max_dir_rows, P->max_dir_cols);
        if (group)
            NUHT_CK(launch_direct_group(P->d_prob, P->d_dir, P->n_dir, P->max_dir_area, mode >= 1 ? 1 : 0, P->d_r,
                                        P->d_w, P->d_r2, P->d_w2, P->d_cs2, P->n, ng, P->d_gs, P->m, ls));
        else
            NUHT_CK(launch_direct(P->d_prob, P->d_dir, P->n_dir, P->max_dir_rows, P->max_dir_area, mode, P->d_r,
                                  P->d_w, P->d_r2, P->d_w2, P->d_cs, P->d_cs2, gs, gsb ? P->d_csb : nullptr,
                                  gsb ? P->d_cs2b : nullptr, gsb, P->det ? 1 : 0, ls));
        NUHT_TRY(T.end(NUHT_STAGE_DIRECT, ls));
    }
    // the asymptotic pipeline, asy_members components per spreading and
    // interpolation launch (their FFTs one after the other)
    const bool lowp = P->opt.precision == NUHT_PREC_MIXED;   // FP32 kernels and butterflies
    const int am = P->asy_members;
    for (int v0 = 0; asy && v0 < ng; v0 += am) {
        const int nv = ng - v0 < am ? ng - v0 : am;
        StageTimer Tv{P, c0 + v0};
        const float2* c2 = member_c2(P, v0);
        double* gv = member_g_acc(P, v0);
        NUHT_TRY(Tv.begin(NUHT_STAGE_ASY_SPREAD, as));
        NUHT_CK(cudaMemsetAsync(gb_acc, 0, acc_bytes(P, 2 * P->gb_len * nv), as));
        if (lowp)
            NUHT_CK(launch_asy_spread_f32(P->d_prob, P->d_asy, P->d_tspread, P->d_smode, P->n_tspread, P->qmax,
                                          P->spread_threads, P->tab, P->d_r, P->d_r2, c2, P->n, nv, gb_acc,
                                          P->gb_len, as));
        else
            NUHT_CK(launch_asy_spread(P->d_prob, P->d_asy, P->d_tspread, P->d_smode, P->n_tspread, P->qmax,
                                      P->spread_threads, P->tab, P->d_r, P->d_r2, c2, P->n, nv, gb_acc,
                                      P->gb_len, P->det ? 1 : 0, as));
        if (P->det) NUHT_CK(launch_fx_decode(P->f_gb, (double*)P->d_gb, 2 * P->gb_len, P->d_prob, as));
        NUHT_TRY(Tv.end(NUHT_STAGE_ASY_SPREAD, as));
        NUHT_TRY(Tv.begin(NUHT_STAGE_ASY_FFT, as));
        // the members' FFTs of whole blocks in one launch each; the two-pass
        // FFTs of large blocks per member (one temporary)
        NUHT_CK(launch_asy_fft_block(P->d_prob, P->d_asy, P->d_fblock, P->n_fblock, P->max_fblock_pts, P->tab,
                                     P->d_gb, P->d_gq, as, false, lowp, nv, P->gb_len, P->gq_len));
        NUHT_CK(launch_asy_fft_small(P->d_prob, P->d_asy, P->d_fsmall, P->n_fsmall, P->max_nf2_small,
                                     P->tab, P->d_gb, P->d_gq, as, false, lowp, nv, P->gb_len, P->gq_len));
        for (int u = 0; P->has_large_fft && u < nv; ++u)
            NUHT_CK(launch_asy_fft_large(P->d_prob, P->d_asy, P->d_fa, P->n_fa, P->d_fb, P->n_fb, P->tab,
                                         P->d_gb + (int64_t)u * P->gb_len, P->d_gtmp,
                                         P->d_gq + (int64_t)u * P->gq_len, as, false, lowp));
        NUHT_TRY(Tv.end(NUHT_STAGE_ASY_FFT, as));
        NUHT_TRY(Tv.begin(NUHT_STAGE_ASY_INTERP, as));
        if (lowp)
            NUHT_CK(launch_asy_interp_f32(P->d_prob, P->d_asy, P->d_tinterp, P->n_tinterp, P->qmax,
                                          P->interp_threads, P->tab, P->d_w, P->d_w2, P->d_gq, P->gq_len, nv,
                                          gv, P->m, as));
        else
            NUHT_CK(launch_asy_interp(P->d_prob, P->d_asy, P->d_tinterp, P->n_tinterp, P->qmax,
                                      P->interp_threads, P->tab, P->d_w, P->d_w2, P->d_gq, P->gq_len, nv, gv,
                                      P->m, as));
        NUHT_TRY(Tv.end(NUHT_STAGE_ASY_INTERP, as));
    }
    NUHT_CK(fk.close());
    return NUHT_OK;
}

// The component loop of a forward transform, in groups of G real components
// (opts.vec_group; 1 when the plan has no local or direct blocks to share):
// gather(comp, c, c2) writes a component's sorted, scaled input into its
// member's arrays, apply_forward adds every block class into the members'
// sums, scatter(comp, g) writes a member's sums out.
extern "C++" {
template <class Gather, class Scatter>
static int drive_forward(nuht_plan_t P, int comps, cudaStream_t s, Gather&& gather, Scatter&& scatter)
{
    NUHT_TRY(ensure_events(P, comps));
    const bool share = ((P->opt.class_mask & 4) && P->n_dir > 0) || ((P->opt.class_mask & 1) && P->n_loc > 0);
    int G = share ? group_size(P) : 1;
    // groups whose moment outputs or shared memory would not fit one CTA: pairs
    if (G > 2 && !local_group_fits(P->lmax, P->ntop_max, P->eval_threads, G)) G = 2;
    for (int c0 = 0; c0 < comps; c0 += G) {
        const int ng = comps - c0 < G ? comps - c0 : G;
        StageTimer T{P, c0};
        NUHT_TRY(T.begin(NUHT_STAGE_GATHER, s));
        for (int v = 0; v < ng; ++v) {
            NUHT_CK(cudaMemsetAsync(member_g_acc(P, v), 0, acc_bytes(P, P->m), s));
            NUHT_CK(gather(c0 + v, member_c(P, v), member_c2(P, v)));
        }
        NUHT_TRY(T.end(NUHT_STAGE_GATHER, s));
        NUHT_TRY(apply_forward(P, c0, ng, s));
        for (int v = 0; v < ng; ++v) {
            StageTimer Tv{P, c0 + v};
            NUHT_TRY(Tv.begin(NUHT_STAGE_SCATTER, s));
            if (P->det) NUHT_CK(launch_fx_decode(member_g_acc(P, v), member_g(P, v), P->m, P->d_prob, s));
            NUHT_CK(scatter(c0 + v, member_g(P, v)));
            NUHT_TRY(Tv.end(NUHT_STAGE_SCATTER, s));
        }
    }
    return NUHT_OK;
}
}  // extern "C++"

int nuht_execute(nuht_plan_t P, const double* c, double* g, int nvec, int is_complex, void* stream)
{
    if (!P || nvec < 1 || P->deriv) return NUHT_ERR_INVALID_ARG;
    if ((P->n > 0 && !c) || (P->m > 0 && !g)) return NUHT_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int comps = nvec * (is_complex ? 2 : 1);
    if (P->m == 0) return NUHT_OK;
    if (P->n == 0) {
        NUHT_CK(cudaMemsetAsync(g, 0, sizeof(double) * P->m * comps, s));
        return NUHT_OK;
    }
    // c is scaled by a power of two from its largest magnitude
    NUHT_CK(launch_input_scale(c, P->n * comps, P->d_mx, s));
    return drive_forward(
        P, comps, s,
        [&](int cp, double* o, float2* o2) { return launch_gather(c, P->d_pr, P->n, comps, cp, P->d_mx, o, o2, s); },
        [&](int cp, const double* src) { return launch_scatter(src, P->d_pw, P->m, comps, cp, P->d_mx, g, s); });
}

// The accumulation target of member v's adjoint sums (d_cs + v n, or f_cs /
// f_csb in the deterministic mode, where groups are pairs).
static double* member_c_acc(nuht_plan_t P, int v)
{
    if (P->det) return (double*)(v == 0 ? P->f_cs : P->f_csb);
    return member_c(P, v);
}

// Transpose of apply_forward for the ng real components c0 .. c0 + ng - 1 of
// a group: sorted g of member v in member_g -> sorted c in member_c.  Each
// block class runs its transposed pipeline; column contributions of blocks at
// different levels meet in c with FP64 atomics.  The local blocks take a
// group of more than two members in the group kernels (one Miller sweep per
// row and one basis per point for all), else pairs (one Miller sweep per row
// for both); the direct blocks run per member; the asymptotic pipeline takes
// asy_members members per spreading and interpolation launch.
static int apply_adjoint(nuht_plan_t P, int c0, int ng, bool pairs, cudaStream_t s)
{
    const int mask = P->opt.class_mask;
    StageTimer T{P, c0};
    const bool loc = (mask & 1) && P->n_loc, dir = (mask & 4) && P->n_dir;
    const bool asy = (mask & 2) && P->n_asy;
    // local and direct blocks beside the asymptotic pipeline, as in apply_forward
    ClassFork fk;
    if (P->opt.timing != NUHT_TIMING_SERIAL && asy && (loc || dir)) NUHT_CK(fk.open(s));
    const cudaStream_t ls = fk.local(s), as = fk.asy(s);
    if (loc) {
        // member v's adjoint moments in d_mom + v mom_len (f_mom / f_momb in the
        // deterministic mode, decoded there)
        const int thr = local_adj_threads(P->ntop_max);
        auto mom_of = [&](int v) { return P->d_mom + (int64_t)v * P->mom_len; };
        auto mom_acc = [&](int v) { return P->det ? (double*)(v == 0 ? P->f_mom : P->f_momb) : mom_of(v); };
        NUHT_TRY(T.begin(NUHT_STAGE_LOCAL_MOMENTS, ls));
        if (ng > 2) {
            // a group: one Miller sweep per row and one basis per point for all members
            NUHT_CK(cudaMemsetAsync(P->d_mom, 0, sizeof(double) * P->mom_len * ng, ls));
            NUHT_CK(launch_local_adj_group(P->d_prob, P->d_loc, P->d_teval, P->n_teval, P->d_tmom, P->n_tmom,
                                           P->lmax, P->ntop_max, local_adj_group_threads(P->ntop_max), P->d_w2,
                                           P->d_r2, P->d_gs, P->m, ng, P->d_mom, P->mom_len, P->d_cs, P->n, true,
                                           ls));
            NUHT_TRY(T.end(NUHT_STAGE_LOCAL_MOMENTS, ls));
            NUHT_TRY(T.begin(NUHT_STAGE_LOCAL_EVAL, ls));
            NUHT_CK(launch_local_adj_group(P->d_prob, P->d_loc, P->d_teval, P->n_teval, P->d_tmom, P->n_tmom,
                                           P->lmax, P->ntop_max, 0, P->d_w2, P->d_r2, P->d_gs, P->m, ng, P->d_mom,
                                           P->mom_len, P->d_cs, P->n, false, ls));
            NUHT_TRY(T.end(NUHT_STAGE_LOCAL_EVAL, ls));
        }
        for (int v = 0; ng <= 2 && v < ng; v += pairs ? 2 : 1) {
            const bool two = pairs && v + 1 < ng;
            NUHT_CK(cudaMemsetAsync(mom_acc(v), 0, acc_bytes(P, P->mom_len * (two && !P->det ? 2 : 1)), ls));
            if (two && P->det) NUHT_CK(cudaMemsetAsync(mom_acc(v + 1), 0, acc_bytes(P, P->mom_len), ls));
            NUHT_CK(launch_local_adj_moments(P->d_prob, P->d_loc, P->d_teval, P->n_teval, P->ntop_max, thr,
                                             P->d_w2, member_g(P, v), mom_acc(v),
                                             two ? member_g(P, v + 1) : nullptr, two ? mom_acc(v + 1) : nullptr,
                                             ls));
            if (P->det) {
                NUHT_CK(launch_fx_decode(P->f_mom, mom_of(0), P->mom_len, P->d_prob, ls));
                if (two) NUHT_CK(launch_fx_decode(P->f_momb, mom_of(1), P->mom_len, P->d_prob, ls));
            }
        }
        if (ng <= 2) {
            NUHT_TRY(T.end(NUHT_STAGE_LOCAL_MOMENTS, ls));
            NUHT_TRY(T.begin(NUHT_STAGE_LOCAL_EVAL, ls));
            for (int v = 0; v < ng; ++v)
                NUHT_CK(launch_local_adj_eval(P->d_prob, P->d_loc, P->d_tmom, P->n_tmom, P->lmax, P->d_r2,
                                              mom_of(v), member_c_acc(P, v), ls));
            NUHT_TRY(T.end(NUHT_STAGE_LOCAL_EVAL, ls));
        }
    }
    if (dir) {
        NUHT_TRY(T.begin(NUHT_STAGE_DIRECT, ls));
        for (int v = 0; v < ng; ++v)
            NUHT_CK(launch_direct_adj(P->d_prob, P->d_dir, P->n_dir, P->max_dir_cols, P->max_dir_area,
                                      P->eps >= 1e-6 ? 1 : 0, P->d_r, P->d_w, P->d_r2, P->d_w2, member_g(P, v),
                                      member_c_acc(P, v), P->det ? 1 : 0, ls));
        NUHT_TRY(T.end(NUHT_STAGE_DIRECT, ls));
    }
    double2* tg_acc = (double2*)acc_target(P, (double*)P->d_tg, P->f_tg);
    const int am = P->asy_members;
    for (int v0 = 0; asy && v0 < ng; v0 += am) {
        const int nv = ng - v0 < am ? ng - v0 : am;
        StageTimer Tv{P, c0 + v0};
        NUHT_TRY(Tv.begin(NUHT_STAGE_ASY_SPREAD, as));
        NUHT_CK(cudaMemsetAsync(tg_acc, 0, acc_bytes(P, 2 * P->gq_len * nv), as));
        NUHT_CK(launch_asy_adj_spread(P->d_prob, P->d_asy, P->d_tinterp, P->n_tinterp, P->qmax, P->interp_threads,
                                      P->tab, P->d_w, member_g(P, v0), P->m, nv, tg_acc, P->gq_len, as));
        if (P->det) NUHT_CK(launch_fx_decode(P->f_tg, (double*)P->d_tg, 2 * P->gq_len, P->d_prob, as));
        NUHT_TRY(Tv.end(NUHT_STAGE_ASY_SPREAD, as));
        NUHT_TRY(Tv.begin(NUHT_STAGE_ASY_FFT, as));
        NUHT_CK(launch_asy_fft_block(P->d_prob, P->d_asy, P->d_fblock, P->n_fblock, P->max_fblock_pts, P->tab,
                                     P->d_tg, P->d_bq, as, true, false, nv, P->gq_len, P->gb_len));
        NUHT_CK(launch_asy_fft_small(P->d_prob, P->d_asy, P->d_fsmall, P->n_fsmall, P->max_nf2_small, P->tab,
                                     P->d_tg, P->d_bq, as, true, false, nv, P->gq_len, P->gb_len));
        for (int u = 0; P->has_large_fft && u < nv; ++u)
            NUHT_CK(launch_asy_fft_large(P->d_prob, P->d_asy, P->d_fa, P->n_fa, P->d_fb, P->n_fb, P->tab,
                                         P->d_tg + (int64_t)u * P->gq_len, P->d_gtmp,
                                         P->d_bq + (int64_t)u * P->gb_len, as, true));
        NUHT_TRY(Tv.end(NUHT_STAGE_ASY_FFT, as));
        NUHT_TRY(Tv.begin(NUHT_STAGE_ASY_INTERP, as));
        NUHT_CK(launch_asy_adj_interp(P->d_prob, P->d_asy, P->d_tspread, P->n_tspread, P->qmax, P->tab, P->d_r,
                                      P->d_bq, P->gb_len, nv, member_c_acc(P, v0), P->n, as));
        NUHT_TRY(Tv.end(NUHT_STAGE_ASY_INTERP, as));
    }
    NUHT_CK(fk.close());
    return NUHT_OK;
}

// The component loop of an adjoint transform (drive_forward transposed), in
// groups as in drive_forward: gather(comp, g) writes a component's sorted,
// scaled input into its member's array, apply_adjoint adds every block class
// into the members' sums, scatter(comp, c) writes a member's sums out.
extern "C++" {
template <class Gather, class Scatter>
static int drive_adjoint(nuht_plan_t P, int comps, cudaStream_t s, Gather&& gather, Scatter&& scatter)
{
    NUHT_TRY(ensure_events(P, comps));
    const bool share = (P->opt.class_mask & 1) && P->n_loc > 0;
    const bool pairs = share && group_size(P) != 1;
    // members per group: the group size when there are asymptotic launches to
    // share, else a pair of the local blocks
    int G = group_size(P);
    if (G > 2 && !local_group_fits(P->lmax, P->ntop_max, P->eval_threads, G)) G = 2;
    if (!pairs && !(P->n_asy && (P->opt.class_mask & 2))) G = 1;
    for (int c0 = 0; c0 < comps; c0 += G) {
        const int ng = comps - c0 < G ? comps - c0 : G;
        StageTimer T{P, c0};
        NUHT_TRY(T.begin(NUHT_STAGE_GATHER, s));
        for (int v = 0; v < ng; ++v) {
            NUHT_CK(cudaMemsetAsync(member_c_acc(P, v), 0, acc_bytes(P, P->n), s));
            NUHT_CK(gather(c0 + v, member_g(P, v)));
        }
        NUHT_TRY(T.end(NUHT_STAGE_GATHER, s));
        NUHT_TRY(apply_adjoint(P, c0, ng, pairs, s));
        for (int v = 0; v < ng; ++v) {
            StageTimer Tv{P, c0 + v};
            NUHT_TRY(Tv.begin(NUHT_STAGE_SCATTER, s));
            if (P->det) NUHT_CK(launch_fx_decode(member_c_acc(P, v), member_c(P, v), P->n, P->d_prob, s));
            NUHT_CK(scatter(c0 + v, member_c(P, v)));
            NUHT_TRY(Tv.end(NUHT_STAGE_SCATTER, s));
        }
    }
    return NUHT_OK;
}
}  // extern "C++"

int nuht_adjoint(nuht_plan_t P, const double* g, double* c, int nvec, int is_complex, void* stream)
{
    if (!P || nvec < 1 || P->deriv) return NUHT_ERR_INVALID_ARG;
    if ((P->m > 0 && !g) || (P->n > 0 && !c)) return NUHT_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int comps = nvec * (is_complex ? 2 : 1);
    if (P->n == 0) return NUHT_OK;
    if (P->m == 0) {
        NUHT_CK(cudaMemsetAsync(c, 0, sizeof(double) * P->n * comps, s));
        return NUHT_OK;
    }
    // g is scaled by a power of two from its largest magnitude
    NUHT_CK(launch_input_scale(g, P->m * comps, P->d_mx, s));
    return drive_adjoint(
        P, comps, s,
        [&](int cp, double* o) { return launch_gather(g, P->d_pw, P->m, comps, cp, P->d_mx, o, nullptr, s); },
        [&](int cp, const double* src) { return launch_scatter(src, P->d_pr, P->n, comps, cp, P->d_mx, c, s); });
}

int nuht_plan_deriv(nuht_plan_t* out, nuht_plan_t base, void* stream)
{
    if (!out) return NUHT_ERR_INVALID_ARG;
    *out = nullptr;
    if (!base || base->deriv || base->probs.size() != 1) return NUHT_ERR_INVALID_ARG;
    const int nu = base->nu_user;
    if (nu - 1 < -100 || nu + 1 > 100) return NUHT_ERR_UNSUPPORTED;
    nuht_plan_t P = new (std::nothrow) nuht_plan_s();
    if (!P) return NUHT_ERR_NOMEM;
    P->deriv = true;
    P->n_base = base->n;
    P->m_base = base->m;
    P->nu_user = nu;
    P->eps = base->eps;
    P->opt = base->opt;
    P->n = 2 * base->n;
    P->m = 2 * base->m;
    P->stream = (cudaStream_t)stream;
    P->probs.resize(2);
    int rc = init_problem(P->probs[0], nu - 1, P->eps, P->opt.m_terms, base->n, base->m, 0, 0);
    if (rc == NUHT_OK)
        rc = init_problem(P->probs[1], nu + 1, P->eps, P->opt.m_terms, base->n, base->m, base->n, base->m);
    if (rc != NUHT_OK) { delete P; return rc; }
    P->probs[1].sgn = -P->probs[1].sgn;   // its sums enter with -J_{nu+1}
    P->w = nufft_width(P->eps);
    rc = build_plan(P, nullptr, nullptr, base);
    if (rc != NUHT_OK) { nuht_destroy(P); return rc; }
    *out = P;
    return NUHT_OK;
}

int nuht_grad_omega(nuht_plan_t D, const double* c, const double* e, double* grad_omega, int nvec, void* stream)
{
    if (!D || !D->deriv || nvec < 1) return NUHT_ERR_INVALID_ARG;
    const int64_t nb = D->n_base, mb = D->m_base;
    if ((nb > 0 && !c) || (mb > 0 && (!e || !grad_omega))) return NUHT_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (mb == 0) return NUHT_OK;
    if (nb == 0) {
        NUHT_CK(cudaMemsetAsync(grad_omega, 0, sizeof(double) * mb, s));
        return NUHT_OK;
    }
    // the forward transform of r c, scaled by a power of two from its largest magnitude
    NUHT_CK(launch_absmax_weighted(c, D->d_pr, D->d_r, nb, nvec, D->d_mx, s));
    return drive_forward(
        D, nvec, s,
        [&](int cp, double* o, float2* o2) {
            return launch_gather_deriv(c, D->d_pr, D->d_r, nb, nvec, cp, D->d_mx, o, o2, s);
        },
        [&](int cp, const double* src) {
            return launch_scatter_deriv(src, D->d_pw, mb, nvec, cp, D->d_mx, e, grad_omega, s);
        });
}

int nuht_grad_r(nuht_plan_t D, const double* c, const double* e, double* grad_r, int nvec, void* stream)
{
    if (!D || !D->deriv || nvec < 1) return NUHT_ERR_INVALID_ARG;
    const int64_t nb = D->n_base, mb = D->m_base;
    if ((nb > 0 && (!c || !grad_r)) || (mb > 0 && !e)) return NUHT_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (nb == 0) return NUHT_OK;
    if (mb == 0) {
        NUHT_CK(cudaMemsetAsync(grad_r, 0, sizeof(double) * nb, s));
        return NUHT_OK;
    }
    // the adjoint transform of omega e, scaled by a power of two from its largest magnitude
    NUHT_CK(launch_absmax_weighted(e, D->d_pw, D->d_w, mb, nvec, D->d_mx, s));
    return drive_adjoint(
        D, nvec, s,
        [&](int cp, double* o) { return launch_gather_deriv(e, D->d_pw, D->d_w, mb, nvec, cp, D->d_mx, o, nullptr, s); },
        [&](int cp, const double* src) {
            return launch_scatter_deriv(src, D->d_pr, nb, nvec, cp, D->d_mx, c, grad_r, s);
        });
}

int nuht_transform_host(int nu, const double* r, int64_t n, const double* omega, int64_t m, double eps,
                        const double* c, double* g, int nvec, const nuht_opts* opt, void* stream)
{
    if (n < 0 || m < 0 || nvec < 1) return NUHT_ERR_INVALID_ARG;
    if ((n > 0 && (!r || !c)) || (m > 0 && (!omega || !g))) return NUHT_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    Arena A;
    size_t o_r = A.reserve<double>(n), o_w = A.reserve<double>(m);
    size_t o_c = A.reserve<double>((size_t)n * nvec), o_g = A.reserve<double>((size_t)m * nvec);
    // the coefficients' upload runs on a stream of its own beside the plan's
    // device work (the plan never reads c); execute waits for it
    char* D = nullptr;
    NUHT_CK(pool_alloc((void**)&D, A.size, s));
    int rc = NUHT_OK;
    nuht_plan_t P = nullptr;
    CopyAux* cx = nullptr;
    bool c_issued = false;
    do {
        cudaError_t e = cudaSuccess;
        if (n) e = cudaMemcpyAsync(D + o_r, r, sizeof(double) * n, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && m) e = cudaMemcpyAsync(D + o_w, omega, sizeof(double) * m, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && n) {
            // forked after the point uploads so that it does not share the
            // link with them: the plan starts as early as before
            e = copy_aux(&cx);
            if (e == cudaSuccess) e = cudaEventRecord(cx->fork, s);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(cx->s, cx->fork, 0);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(D + o_c, c, sizeof(double) * n * nvec, cudaMemcpyHostToDevice, cx->s);
            if (e == cudaSuccess) e = cudaEventRecord(cx->done, cx->s);
            c_issued = e == cudaSuccess;
        }
        if (e != cudaSuccess) { g_cuda_msg = cudaGetErrorString(e); rc = NUHT_ERR_CUDA; break; }
        rc = nuht_plan(&P, nu, (const double*)(D + o_r), n, (const double*)(D + o_w), m, eps, opt, stream);
        if (rc != NUHT_OK) break;
        if (c_issued) {
            e = cudaStreamWaitEvent(s, cx->done, 0);
            if (e != cudaSuccess) { g_cuda_msg = cudaGetErrorString(e); rc = NUHT_ERR_CUDA; break; }
        }
        rc = nuht_execute(P, (const double*)(D + o_c), (double*)(D + o_g), nvec, 0, stream);
        if (rc != NUHT_OK) break;
        if (m) e = cudaMemcpyAsync(g, D + o_g, sizeof(double) * m * nvec, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { g_cuda_msg = cudaGetErrorString(e); rc = NUHT_ERR_CUDA; break; }
    } while (0);
    nuht_destroy(P);
    // the upload finishes before the arena goes back to the pool (also on the
    // paths that left the loop early)
    if (cx) cudaStreamSynchronize(cx->s);
    pool_free(D, s);
    cudaStreamSynchronize(s);
    return rc;
}

int nuht_info(nuht_plan_t P, nuht_plan_info* out)
{
    if (!P || !out) return NUHT_ERR_INVALID_ARG;
    std::memset(out, 0, sizeof(*out));
    out->nu = P->nu_user;
    out->M = P->probs[0].M;
    out->L = P->probs[0].L;
    out->nufft_width = P->w;
    out->nufft_degree = P->tab.deg;
    out->asy_members = P->asy_members;
    out->z = P->probs[0].z;
    out->eps = P->eps;
    out->n = P->n;
    out->m = P->m;
    out->n_local = P->n_loc;
    out->n_asy = P->n_asy;
    out->n_direct = P->n_dir;
    out->direct_entries = P->direct_entries;
    out->local_rows_cols = P->local_rc;
    out->asy_rows_cols = P->asy_rc;
    out->fft_points = P->fft_points;
    out->device_bytes = (int64_t)P->dbytes;
    for (int i = 0; i < 4; ++i) out->plan_ms[i] = P->plan_ms[i];
    return NUHT_OK;
}

int nuht_get_blocks(nuht_plan_t P, int cls, int64_t* ranges, int64_t cap, int64_t* count)
{
    if (!P || cls < 0 || cls > 2 || !count || cap < 0 || (cap > 0 && !ranges)) return NUHT_ERR_INVALID_ARG;
    const int64_t first = cls == 0 ? 0 : (cls == 1 ? P->n_loc : (int64_t)P->n_loc + P->n_asy);
    *count = cls == 0 ? P->n_loc : (cls == 1 ? P->n_asy : P->n_dir);
    const int64_t nc = cap < *count ? cap : *count;
    if (nc <= 0) return NUHT_OK;
    std::vector<SubBlk> v((size_t)nc);
    NUHT_CK(cudaMemcpyAsync(v.data(), P->d_blk + first, sizeof(SubBlk) * nc, cudaMemcpyDeviceToHost, P->stream));
    NUHT_CK(cudaStreamSynchronize(P->stream));
    for (int64_t i = 0; i < nc; ++i) {
        ranges[4 * i + 0] = v[(size_t)i].k0;
        ranges[4 * i + 1] = v[(size_t)i].k1;
        ranges[4 * i + 2] = v[(size_t)i].j0;
        ranges[4 * i + 3] = v[(size_t)i].j1;
    }
    return NUHT_OK;
}

int nuht_get_permutations(nuht_plan_t P, int32_t* perm_r, int32_t* perm_omega)
{
    if (!P) return NUHT_ERR_INVALID_ARG;
    if (perm_r && P->n)
        NUHT_CK(cudaMemcpyAsync(perm_r, P->d_pr, sizeof(int32_t) * P->n, cudaMemcpyDeviceToHost, P->stream));
    if (perm_omega && P->m)
        NUHT_CK(cudaMemcpyAsync(perm_omega, P->d_pw, sizeof(int32_t) * P->m, cudaMemcpyDeviceToHost, P->stream));
    NUHT_CK(cudaStreamSynchronize(P->stream));
    return NUHT_OK;
}

}  // extern "C"
