/*
 * nuht.h -- C ABI of the GB300 (sm_103a) nonuniform fast Hankel transform.
 *
 * The transform (the discrete Hankel transform, Sec. 1, eq. DHT; matrix
 * form A(k, j) = J_nu(omega_k r_j) of Sec. 2):
 *
 *     g_k = sum_{j=0}^{n-1} c_j J_nu(omega_k r_j),   k = 0..m-1,
 *
 * from n nonuniform points r_j >= 0 to m nonuniform frequencies omega_k >= 0,
 * to a requested precision eps, by the paper's method (Algorithm 2): the
 * matrix is subdivided along omega r = z (Algorithm 1); blocks with
 * omega r <= z use the Wimp expansion (Sec. 3.1), blocks with omega r > z use
 * Hankel's expansion through 2M type-3 NUFFTs (Sec. 3.2), and small
 * mixed blocks are summed directly.  The orders L, M and the crossover z come
 * from the error bounds of Lemma 3.1 and Sec. 3.2 (eq. asy-error), as
 * described in Sec. 3.3.
 *
 * Index convention: points are indexed by j (length n), frequencies by k
 * (length m).  The paper uses the opposite letters.
 *
 * Accuracy contract (per coefficient vector):
 *     max_k |g_k - g_k^exact| <= 10 eps ||c||_1.
 *
 * Memory: unless stated otherwise every array argument is a DEVICE pointer
 * (cudaMalloc'd or managed memory of the current device).  All FP64 arrays are
 * contiguous.  The caller owns every array it passes.  Calls are ordered on
 * the given CUDA stream (a cudaStream_t passed as void*; NULL = the legacy
 * default stream) and may return before the GPU work finishes, except
 * nuht_plan, nuht_plan_many and nuht_plan_deriv, which wait once for the
 * sizes of the block lists (the sort, the subdivision and the list build run
 * on the device; only lists beyond the device capacity are built on the
 * host), and the *_host entry points, which synchronise before returning.
 *
 * Errors: every int-returning call returns NUHT_OK (0) or one of the
 * NUHT_ERR_* codes below; nuht_strerror() gives a message.  On error no
 * output array is written (plan: *out is set to NULL).
 */
#ifndef NUHT_H
#define NUHT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
#define NUHT_OK              0
#define NUHT_ERR_INVALID_ARG 1   /* n or m < 0, eps outside [1e-15, 1e-1], nvec < 1, NULL plan ... */
#define NUHT_ERR_DOMAIN      2   /* some r_j or omega_k is negative, NaN or infinite */
#define NUHT_ERR_NOMEM       3   /* a device or host allocation failed */
#define NUHT_ERR_CUDA        4   /* a CUDA runtime call failed (see nuht_last_cuda_error) */
#define NUHT_ERR_TIMEOUT     5   /* a bounded device wait gave up (reported by nuht_status) */
#define NUHT_ERR_UNSUPPORTED 6   /* option combination not built (e.g. order |nu| > 100) */
#define NUHT_ERR_SCRATCH     7   /* request exceeds the fixed scratch of nuht_local_apply_noalloc */
#define NUHT_ERR_BAD_BLOCKS  8   /* a block work list failed its check (nuht_check_blocks) */

/* --------------------------------------------------------------- options */
#define NUHT_PREC_FP64  0   /* every stage in FP64 (or FP64-accurate arithmetic) */
#define NUHT_PREC_MIXED 1   /* FP32 spreading / interpolation (FP32 accumulation), FFT
                               butterflies, local evaluation and direct entries; fixed-point /
                               double-float positions, phase reduction, Hankel coefficients and
                               moments; needs eps >= 1e-6 (else NUHT_ERR_UNSUPPORTED) */

/* Block classes (Sec. 4.1). */
#define NUHT_BLOCK_LOCAL  0
#define NUHT_BLOCK_ASY    1
#define NUHT_BLOCK_DIRECT 2

/* Upper limit of nuht_opts.min_size: a direct block's row (or column) sums
   and its entry list stay in one CTA's shared memory. */
#define NUHT_MAX_MIN_SIZE 16384

/* Upper limit of nuht_opts.vec_group. */
#define NUHT_MAX_VEC_GROUP 16

/* opts.timing: NUHT_TIMING_OFF records nothing; NUHT_TIMING_LIVE records a
 * CUDA event pair around each stage on the stream the stage runs on (the
 * block classes run concurrently as in an untimed execute, so the stage times
 * of different classes overlap); NUHT_TIMING_SERIAL runs every stage in order
 * on the caller's stream, so each time is that stage alone. */
#define NUHT_TIMING_OFF    0
#define NUHT_TIMING_LIVE   1
#define NUHT_TIMING_SERIAL 2

typedef struct {
    int precision;     /* NUHT_PREC_FP64 (default) or NUHT_PREC_MIXED */
    int min_size;      /* largest area (rows*cols) of a mixed block summed directly;
                          default 1024, at most NUHT_MAX_MIN_SIZE (Sec. 4.1) */
    int n_split_cand;  /* candidate rows tried by SplitIndices (Sec. 4.1); default 16 */
    int m_terms;       /* asymptotic terms M; 0 = the heuristic of Sec. 3.3 */
    int class_mask;    /* bit c set = apply blocks of class c (testing aid); default 7 */
    int timing;        /* NUHT_TIMING_*: stage events (see nuht_stage_times); default 0 */
    int spread_tile;   /* points per spreading CTA: 0 = automatic (256, or 128 when
                          2M > 16); else 64..256, a multiple of 32 */
    int deterministic; /* 1 = bitwise reproducible results: every block class adds its
                          contributions to g (c for the adjoint), to the spreading grids and
                          to the moments as exact 128-bit fixed-point integers (scaled per
                          call by the largest input magnitude, rounded once per
                          contribution at about 2^-54 of it), so the order of the additions
                          does not matter; the same inputs on the same GPU then give the same
                          bits on every run.  Slower (more atomics, no FP32 row sums in the
                          direct blocks, extra device memory).  Default 0 (FP64 atomics). */
    int persistent;    /* 1 = the local blocks' moments and evaluation in one persistent
                          launch: resident CTAs take moment tiles, then evaluation tiles,
                          from a device queue, and an evaluation tile waits (a bounded
                          poll) until its block's moments are complete.  A wait that gives
                          up records NUHT_ERR_TIMEOUT for nuht_status.  Not used with
                          deterministic = 1.  Default 0 (two launches). */
    int interp_tile;   /* frequencies per interpolation CTA (also the adjoint's spreading of
                          frequencies): 0 = 256, or 128 (better when the asymptotic blocks
                          hold few frequencies each) */
    int vec_group;     /* real components (vectors, or the parts of complex c) whose local
                          and direct blocks nuht_execute applies together, sharing their
                          Bessel work (the moment basis, the Miller sweeps, the direct
                          entries; the moments become one dense (L+1) x n_b by n_b x G
                          product per block): 1..NUHT_MAX_VEC_GROUP, 0 = 2.  The plan
                          holds G copies of the sorted coefficient, moment and output
                          arrays.  Above 2 not with deterministic = 1 or persistent = 1.
                          The adjoint shares in pairs whenever this is not 1. */
    int reserved;      /* must be zero */
} nuht_opts;

/* Execute stages, in launch order (nuht_stage_times / nuht_stage_name). */
#define NUHT_STAGE_GATHER        0   /* c to sorted order */
#define NUHT_STAGE_LOCAL_MOMENTS 1   /* Wimp moments of the local blocks */
#define NUHT_STAGE_ASY_SPREAD    2   /* type-3 spreading of the asymptotic blocks */
#define NUHT_STAGE_ASY_FFT       3   /* deconvolution + FFT of the spread grids */
#define NUHT_STAGE_ASY_INTERP    4   /* interpolation + Hankel combination */
#define NUHT_STAGE_LOCAL_EVAL    5   /* Wimp evaluation of the local blocks */
#define NUHT_STAGE_DIRECT        6   /* direct blocks */
#define NUHT_STAGE_SCATTER       7   /* g back to user order */
#define NUHT_NUM_STAGES          8

typedef struct {
    int     nu;            /* order */
    int     M;             /* Hankel terms (pairs), Sec. 3.3 */
    int     L;             /* Wimp order (terms l = 0..L), Lemma 3.1 */
    int     nufft_width;   /* ES kernel width w of the type-3 NUFFTs */
    int     nufft_degree;  /* degree of the kernel's piecewise polynomials */
    int     asy_members;   /* real components per asymptotic spreading / interpolation launch */
    double  z;             /* crossover point, B^asy_{nu,M}(z) = eps */
    double  eps;
    int64_t n, m;
    int64_t n_local, n_asy, n_direct;     /* block counts per class */
    int64_t direct_entries;               /* sum of direct block areas */
    int64_t local_rows_cols;              /* sum over local blocks of rows + cols */
    int64_t asy_rows_cols;                /* sum over asymptotic blocks of rows + cols */
    int64_t fft_points;                   /* sum over asymptotic blocks of FFT sizes */
    int64_t device_bytes;                 /* device memory held by the plan */
    double  plan_ms[4];                   /* host wall time of the plan phases: [0] checks, sort
                                             and copies back, [1] subdivision, [2] work lists,
                                             [3] upload */
} nuht_plan_info;

typedef struct nuht_plan_s *nuht_plan_t;

/* Fill *opt with the defaults listed above. */
void nuht_default_opts(nuht_opts *opt);

/* Host-only: the expansion orders and crossover of Sec. 3.3 for (nu, eps).
 * m_terms = 0 uses the heuristic of Sec. 3.3 (eq. num-asy-terms) for M.  Outputs: *M, *z (root of
 * B^asy_{nu,M}(z) = eps, Sec. 3.2 eq. asy-error) and *L (smallest L with
 * B^loc_{nu,L}(z) < eps, Lemma 3.1).  No GPU needed. */
int nuht_choose_params(int nu, double eps, int m_terms, int *M, double *z, int *L);

/* Build a plan for order nu, points r[0..n), frequencies omega[0..m) (device
 * FP64, any order, values >= 0), tolerance eps in [1e-15, 1e-1].  Sorts r and
 * omega, subdivides the matrix (Algorithm 1) and builds the block work lists,
 * all on the device; the host waits once for the list sizes.  The call
 * returns with the rest of the build queued on the stream (stream-ordered
 * like every call).  The plan copies what it needs; r and omega are consumed
 * before that wait and may be freed after return.  opt may be NULL (defaults).  Negative
 * nu is mapped through J_{-nu} = (-1)^nu J_nu.  n = 0 or m = 0 is allowed.
 * Block lists beyond the device capacity ((n+m)/16 + 16384 per class; the
 * environment variable NUHT_SUBDIVIDE_CAPACITY lowers it, for testing) are
 * built by a host walk of Algorithm 1 instead, with the same result. */
int nuht_plan(nuht_plan_t *out, int nu, const double *r, int64_t n,
              const double *omega, int64_t m, double eps, const nuht_opts *opt,
              void *stream);

/* A batch of nprob independent problems in one plan (the same eps): problem
 * i has order nu[i] (host array), n[i] points and m[i] frequencies (host
 * arrays); the points of all problems are concatenated in r (device, sum n[i]
 * entries, problem 0 first) and the frequencies in omega (device, sum m[i]).
 * One execute then applies every problem's transform with one launch per
 * stage over the whole batch: c and g are the concatenations of the
 * problems' vectors in the same order (c: sum n[i] rows, g: sum m[i] rows).
 * nprob <= 65536.  nuht_get_blocks reports indices into the concatenated
 * sorted arrays; nuht_info reports the first problem's orders. */
int nuht_plan_many(nuht_plan_t *out, int nprob, const int *nu, const double *r, const int64_t *n,
                   const double *omega, const int64_t *m, double eps, const nuht_opts *opt,
                   void *stream);

/* Forward transform g = A c.  c: n x nvec (row-major, c[j*nvec + v]) FP64,
 * or n x nvec complex (interleaved re,im: c[2*(j*nvec+v)+{0,1}]) when
 * is_complex != 0.  g: m x nvec of the same kind, OVERWRITTEN, in the
 * caller's original omega order.  The operator is real, so a complex c is
 * transformed as its real and imaginary parts. */
int nuht_execute(nuht_plan_t p, const double *c, double *g, int nvec, int is_complex,
                 void *stream);

/* Adjoint (transposed) transform c = A^T g with the same conventions (g has
 * m rows, c has n rows, c is overwritten, in the caller's original r order).
 * A is real, so the adjoint is the transpose. */
int nuht_adjoint(nuht_plan_t p, const double *g, double *c, int nvec, int is_complex,
                 void *stream);

/* Derivative plan of a plan built by nuht_plan (not a batch): the transforms
 * of orders nu - 1 and nu + 1 on the base plan's points and frequencies, for
 * the gradients with respect to r and omega.  With J_nu' = (J_{nu-1} -
 * J_{nu+1}) / 2 (DLMF 10.6.1; J_{-1} = -J_1 as for any negative order):
 *
 *   d/dr_j     sum_k e_k g_k = c_j sum_k e_k omega_k J_nu'(omega_k r_j)
 *   d/domega_k sum_k e_k g_k = e_k sum_j c_j r_j J_nu'(omega_k r_j)
 *
 * The two orders run as two problems of one plan whose sums are added with
 * opposite signs, so each gradient is one pass of the pipeline.  The plan
 * reuses the base plan's sorted values and permutations (no second sort or
 * domain check); it needs |nu| + 1 <= 100 (else NUHT_ERR_UNSUPPORTED) and uses
 * the base plan's eps and options.  The base plan may be destroyed afterwards.
 * nuht_execute / nuht_adjoint reject a derivative plan (NUHT_ERR_INVALID_ARG);
 * nuht_info reports its two problems' combined sizes (2n, 2m) and the orders
 * of nu - 1. */
int nuht_plan_deriv(nuht_plan_t *out, nuht_plan_t base, void *stream);

/* Gradient with respect to r through a derivative plan d:
 *   grad_r[j] = sum_v c[j][v] sum_k e[k][v] omega_k J_nu'(omega_k r_j)
 * for nvec real vectors (c: n x nvec, e: m x nvec, row-major as in
 * nuht_execute); grad_r has n entries (caller's r order), overwritten.  The
 * weighting by omega and by c and the half difference of the two orders run
 * in the gather and scatter kernels.  Accuracy: within 10 eps |c_j| ||omega e||_1
 * per vector. */
int nuht_grad_r(nuht_plan_t d, const double *c, const double *e, double *grad_r, int nvec, void *stream);

/* Gradient with respect to omega through a derivative plan d:
 *   grad_omega[k] = sum_v e[k][v] sum_j c[j][v] r_j J_nu'(omega_k r_j)
 * (same conventions; grad_omega has m entries, caller's omega order).
 * Accuracy: within 10 eps |e_k| ||r c||_1 per vector. */
int nuht_grad_omega(nuht_plan_t d, const double *c, const double *e, double *grad_omega, int nvec, void *stream);

/* Whole transform from HOST arrays: copies r, omega, c to the device, plans,
 * executes, copies g (m x nvec real) back to the host array g, and frees the
 * plan.  r, omega, c, g are host pointers (pinned memory is fastest).
 * Synchronises the stream before returning. */
int nuht_transform_host(int nu, const double *r, int64_t n, const double *omega,
                        int64_t m, double eps, const double *c, double *g, int nvec,
                        const nuht_opts *opt, void *stream);

/* Host-only check of a work list: the subdivision (Algorithm 1, Sec. 4.1) of
 * one problem with order nu, tolerance eps and m_terms as in the plan
 * options; the crossover z is the one nuht_choose_params gives.  r_sorted (n) and omega_sorted
 * (m) are HOST arrays in ascending order; ranges holds count blocks as
 * (k0, k1, j0, j1) (inclusive indices into omega_sorted / r_sorted, the
 * layout of nuht_get_blocks) and cls their classes (NUHT_BLOCK_*), both host
 * arrays.  Returns NUHT_OK when the blocks cover every entry of the m x n
 * matrix exactly once, every local block has omega_k1 r_j1 <= z, every
 * asymptotic block omega_k0 r_j0 > z, and every direct block an area of at
 * most min_size; NUHT_ERR_BAD_BLOCKS otherwise (or when the arrays are not
 * sorted); NUHT_ERR_INVALID_ARG / NUHT_ERR_UNSUPPORTED for bad arguments.
 * The plan runs the same check on the host subdivision's lists before using
 * them, and on its device-built lists when the environment variable
 * NUHT_CHECKED is set (and not "0"); nuht_plan then fails with
 * NUHT_ERR_BAD_BLOCKS instead of executing an invalid list.  No GPU needed. */
int nuht_check_blocks(int nu, double eps, int m_terms, const double *r_sorted, int64_t n,
                      const double *omega_sorted, int64_t m, int min_size, const int64_t *ranges,
                      const int32_t *cls, int64_t count);

/* Plan summary (orders, block counts, work sizes). */
int nuht_info(nuht_plan_t p, nuht_plan_info *out);

/* Copy the blocks of class cls (NUHT_BLOCK_*) into ranges, 4 int64 per block
 * (k0, k1, j0, j1; inclusive; indices into the SORTED omega / r), host
 * memory, at most cap blocks.  *count receives the number of blocks of that
 * class (call with cap = 0 to size the buffer). */
int nuht_get_blocks(nuht_plan_t p, int cls, int64_t *ranges, int64_t cap, int64_t *count);

/* Copy the sorting permutations to HOST arrays: perm_r[i] = user index of
 * the i-th smallest r (n entries), perm_omega likewise (m entries).  Either
 * pointer may be NULL. */
int nuht_get_permutations(nuht_plan_t p, int32_t *perm_r, int32_t *perm_omega);

/* Device time (milliseconds) of each stage of the most recent nuht_execute
 * of a plan built with opts.timing != NUHT_TIMING_OFF, summed over the vectors
 * of that call (with NUHT_TIMING_LIVE the stages of different block classes
 * overlap);
 * ms has room for cap doubles (NUHT_NUM_STAGES suffices); stages that did not
 * run report 0.  Waits for the events of that call.  NUHT_ERR_INVALID_ARG if
 * timing is off or nothing ran yet. */
int nuht_stage_times(nuht_plan_t p, double *ms, int cap);

/* Static name of stage i ("gather", "local_moments", ...), or NULL. */
const char *nuht_stage_name(int i);

/* Errors found on the device since the last call for this plan: waits for
 * the stream, then returns NUHT_OK or the recorded status (NUHT_ERR_TIMEOUT
 * when a bounded device wait of a persistent launch gave up; that launch
 * skipped the work behind the wait, so its output is invalid) and clears it.
 * The execute and adjoint calls return before their kernels run, so a device
 * error surfaces here. */
int nuht_status(nuht_plan_t p, void *stream);

/* Number of CUDA kernels this library has launched in this process so far
 * (a diagnostic counter). */
int64_t nuht_kernel_launch_count(void);

/* Throughput probe (the paper has no counterpart; a measurement aid).  Times,
 * with CUDA events on the given stream, one launch of kind 0 = FP32 fused
 * multiply-adds, 1 = FP64 fused multiply-adds, 2 = the double-float
 * compensated multiply-add the execute kernels accumulate with (a product of
 * two double-float numbers added to a compensated FP32 sum), iters iterations
 * of 8 independent chains per thread on 4 CTAs of 256 threads per SM.
 * *ms receives the launch time, *ops the number of operations (multiply-adds)
 * it ran; 2 * ops / ms gives FLOP/ms (for kind 2, FP64-equivalent FLOPs).
 * Synchronises the stream.  iters in [1, 2^32]. */
int nuht_probe_alu(int kind, int64_t iters, double *ms, double *ops, void *stream);

/* ------------------------------------------------- no-allocation entry point
 * The paper has no counterpart to this call; it is a service for callers that
 * cannot let a library call cudaMalloc -- frameworks that reserve nearly all
 * device memory for their own pool up front, and latency-critical loops in
 * which cudaMalloc / cudaFree would stall on an implicit device
 * synchronisation.
 *
 * nuht_local_apply_noalloc computes g = A c (same definition and accuracy
 * contract as nuht_execute) for a transform whose whole matrix is local:
 * the caller gives bounds r_max >= every r_j and omega_max >= every omega_k
 * with omega_max * r_max <= z(nu, eps) (z from nuht_choose_params), and the
 * Wimp expansion of Sec. 3.1 is applied to the whole matrix as one block.
 * r (n), omega (m), c (n x nvec, c[j*nvec+v]) and g (m x nvec, overwritten)
 * are device FP64 arrays in any order.  Values outside the stated bounds give
 * unspecified (but memory-safe) results.
 *
 * It allocates nothing.  Its scratch (the nvec x (L+1) Wimp moments) is a
 * fixed device array of NUHT_NOALLOC_MAX_MOMENTS doubles (256 KiB) that every
 * GPU which loads the library holds until the process exits; requests with
 * nvec * (L + 1) > NUHT_NOALLOC_MAX_MOMENTS return NUHT_ERR_SCRATCH.  All calls
 * on a device share that array (each call clears what it uses), so calls that
 * overlap on the GPU -- e.g. on two streams -- race.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress, with
 * that device current) and caches it; make that first call before any stream
 * capture, and do not use the call across a cudaDeviceReset (the array may
 * move when the module is loaded again).  Errors: NUHT_ERR_INVALID_ARG (sizes, pointers, eps),
 * NUHT_ERR_DOMAIN (omega_max * r_max > z, or a bound negative / not finite),
 * NUHT_ERR_UNSUPPORTED (|nu| > 100), NUHT_ERR_SCRATCH, NUHT_ERR_CUDA. */
#define NUHT_NOALLOC_MAX_MOMENTS 32768
int nuht_local_apply_noalloc(int nu, double eps, const double *r, int64_t n, double r_max,
                             const double *omega, int64_t m, double omega_max,
                             const double *c, double *g, int nvec, void *stream);

/* Release a plan (NULL is ignored).  Waits for the plan's stream. */
void nuht_destroy(nuht_plan_t p);

/* Static message for a status code. */
const char *nuht_strerror(int code);

/* Message of the last CUDA error seen by this library in this thread. */
const char *nuht_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* NUHT_H */
