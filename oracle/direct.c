/*
 * Oracle (test infrastructure only; never part of the product path).
 *
 * Plain FP64 CPU evaluation of the discrete Hankel transform (Sec. 1,
 * eq. DHT):
 *
 *     g_k = sum_j c_j J_nu(omega_k r_j)
 *
 * with its own Bessel evaluator:
 *   - power series (DLMF 10.2.2) for small arguments,
 *   - Miller backward recurrence normalised by 1 = J_0 + 2 sum_k J_2k
 *     (DLMF 10.74(iv), 10.12.4) for moderate arguments,
 *   - Hankel's asymptotic expansion (Sec. 3.2, DLMF 10.17.3) for large
 *     arguments, summed until the terms fall below 1e-17.
 * The sum over j uses Neumaier compensated summation; rows are split over
 * POSIX threads.  Nothing here is shared with the CUDA path.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <unistd.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ---------------------------------------------------------------- series */
/* J_nu(x) = (x/2)^nu sum_k (-x^2/4)^k / (k! Gamma(nu+k+1)), DLMF 10.2.2. */
double oracle_jv_series(double nu, double x)
{
    if (x == 0.0) return nu == 0.0 ? 1.0 : 0.0;
    double h = 0.5 * x;
    double lead;
    if (nu == floor(nu)) {
        /* integer order: exact factorial by product */
        lead = 1.0;
        for (int i = 1; i <= (int)nu; ++i) lead *= h / (double)i;
    } else {
        lead = pow(h, nu) / tgamma(nu + 1.0);
    }
    double term = lead, sum = lead, q = -h * h;
    for (int k = 1; k < 1000; ++k) {
        term *= q / ((double)k * (nu + (double)k));
        sum += term;
        if (fabs(term) <= 1e-18 * fabs(sum)) break;
    }
    return sum;
}

/* ---------------------------------------------------------------- Hankel */
/* Hankel's expansion (Sec. 3.2; DLMF 10.17.3) at x = x_hi + x_lo (the exact
 * product of two doubles), with a_k(nu) from DLMF 10.17.1:
 *   a_k(nu) = prod_{i=1..k} (4nu^2 - (2i-1)^2) / (k! 8^k).
 * Sums until a term drops below 1e-17; *ok = 0 if the series starts to grow
 * before that (argument too small for this order). */
double oracle_jv_hankel2(double nu, double x_hi, double x_lo, int *ok)
{
    double mu = 4.0 * nu * nu;
    double P = 1.0, Q = 0.0, term = 1.0, prev = INFINITY;
    int conv = 0;
    for (int k = 1; k < 200; ++k) {
        double f = (mu - (double)(2 * k - 1) * (double)(2 * k - 1)) / ((double)k * 8.0 * x_hi);
        term *= f;
        double at = fabs(term);
        if (term == 0.0) { conv = 1; break; }        /* half-integer order: exact */
        if (at > prev) break;                          /* divergent tail */
        if (k & 1) Q += ((((k - 1) / 2) & 1) ? -term : term);
        else       P += (((k / 2) & 1) ? -term : term);
        if (at < 1e-17) { conv = 1; break; }
        prev = at;
    }
    if (ok) *ok = conv;
    double ph = (2.0 * nu + 1.0) * M_PI / 4.0;
    double cp = cos(ph), sp = sin(ph);
    double cx = cos(x_hi), sx = sin(x_hi);
    /* first-order correction for the low part of the argument */
    double cx2 = cx - x_lo * sx, sx2 = sx + x_lo * cx;
    double cchi = cx2 * cp + sx2 * sp;   /* cos(x - ph) */
    double schi = sx2 * cp - cx2 * sp;   /* sin(x - ph) */
    return sqrt(2.0 / (M_PI * x_hi)) * (P * cchi - Q * schi);
}

double oracle_jv_hankel(double nu, double x, int *ok)
{
    return oracle_jv_hankel2(nu, x, 0.0, ok);
}

/* ---------------------------------------------------------------- Miller */
/* Backward recurrence J_{k-1} = (2k/x) J_k - J_{k+1} from a start index well
 * beyond max(n, x), normalised with J_0 + 2 sum_{k>=1} J_{2k} = 1. */
double oracle_jn_miller(int n, double x)
{
    if (x == 0.0) return n == 0 ? 1.0 : 0.0;
    double mx = x > (double)n ? x : (double)n;
    int ns = 2 * ((int)(mx + 40.0 + sqrt(80.0 * mx)) / 2 + 1);
    double jip1 = 0.0, ji = 1.0;
    double S = 2.0 * ji;                 /* ns is even and > 0 */
    double res = (n == ns) ? ji : 0.0;
    for (int i = ns; i >= 1; --i) {
        double jim1 = (2.0 * (double)i / x) * ji - jip1;
        jip1 = ji;
        ji = jim1;
        int idx = i - 1;
        if (idx == n) res = ji;
        if (idx == 0) S += ji;
        else if ((idx & 1) == 0) S += 2.0 * ji;
        if (fabs(ji) > 1e250) { ji *= 1e-250; jip1 *= 1e-250; S *= 1e-250; res *= 1e-250; }
    }
    return res / S;
}

/* ------------------------------------------------------------ dispatcher */
/* Integer order n (any sign; J_{-n} = (-1)^n J_n), argument x = hi + lo >= 0. */
static double jn2(int n, double hi, double lo)
{
    double sgn = 1.0;
    if (n < 0) { n = -n; if (n & 1) sgn = -1.0; }
    if (hi == 0.0) return n == 0 ? sgn : 0.0;
    double x = hi;
    if (x <= 2.0 || 0.25 * x * x < 0.25 * (double)(n + 1))
        return sgn * oracle_jv_series((double)n, x);
    if (x >= 25.0 + 0.5 * (double)n * (double)n) {
        int ok = 0;
        double v = oracle_jv_hankel2((double)n, hi, lo, &ok);
        if (ok) return sgn * v;
    }
    return sgn * oracle_jn_miller(n, x);
}

double oracle_jn(int n, double x) { return jn2(n, x, 0.0); }

/* J_n at the exact product a*b of two non-negative doubles. */
double oracle_jn_prod(int n, double a, double b)
{
    double hi = a * b;
    double lo = fma(a, b, -hi);
    return jn2(n, hi, lo);
}

/* ------------------------------------------------------------ direct sum */
typedef struct {
    int nu;
    const double *r; int64_t n;
    const double *omega;
    const int64_t *rows; int64_t nrows;
    const double *c; int nvec;
    double *g;
    int64_t row_begin, row_end;
} job_t;

static void *direct_worker(void *arg)
{
    job_t *J = (job_t *)arg;
    int nv = J->nvec;
    double *sum = (double *)calloc((size_t)nv * 2, sizeof(double));
    double *comp = sum + nv;
    for (int64_t i = J->row_begin; i < J->row_end; ++i) {
        int64_t k = J->rows ? J->rows[i] : i;
        double w = J->omega[k];
        for (int v = 0; v < nv; ++v) { sum[v] = 0.0; comp[v] = 0.0; }
        for (int64_t j = 0; j < J->n; ++j) {
            double a = oracle_jn_prod(J->nu, w, J->r[j]);
            for (int v = 0; v < nv; ++v) {
                double x = J->c[j * nv + v] * a;
                double t = sum[v] + x;          /* Neumaier compensated sum */
                if (fabs(sum[v]) >= fabs(x)) comp[v] += (sum[v] - t) + x;
                else                          comp[v] += (x - t) + sum[v];
                sum[v] = t;
            }
        }
        for (int v = 0; v < nv; ++v) J->g[i * nv + v] = sum[v] + comp[v];
    }
    free(sum);
    return NULL;
}

/* g[i*nvec + v] = sum_j c[j*nvec + v] J_nu(omega[row_i] r_j) for i < nrows,
 * row_i = rows[i] (or i when rows == NULL).  nthreads <= 0: all cores. */
int oracle_direct(int nu, const double *r, int64_t n, const double *omega,
                  const int64_t *rows, int64_t nrows, const double *c, int nvec,
                  double *g, int nthreads)
{
    if (nthreads <= 0) nthreads = (int)sysconf(_SC_NPROCESSORS_ONLN);
    if (nthreads < 1) nthreads = 1;
    if (nthreads > nrows) nthreads = nrows > 0 ? (int)nrows : 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    job_t *jobs = (job_t *)malloc(sizeof(job_t) * (size_t)nthreads);
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = (job_t){nu, r, n, omega, rows, nrows, c, nvec, g,
                          nrows * t / nthreads, nrows * (t + 1) / nthreads};
        pthread_create(&th[t], NULL, direct_worker, &jobs[t]);
    }
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(th);
    free(jobs);
    return nthreads;
}

/* Elementwise J_n(x) over an array (single thread). */
void oracle_jn_array(int n, const double *x, double *out, int64_t len)
{
    for (int64_t i = 0; i < len; ++i) out[i] = oracle_jn(n, x[i]);
}
