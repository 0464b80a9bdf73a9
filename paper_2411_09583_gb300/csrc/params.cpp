// Host-side numerics of the plan: expansion orders and crossover (Sec. 3.3),
// and the tables of the type-3 NUFFT kernel (exponential of semicircle).
#include <cmath>
#include <cstdint>
#include <map>
#include <mutex>
#include <vector>

#include "nuht_host.h"

namespace nuht {

// a_k(nu) = prod_{i=1..k} (4 nu^2 - (2i-1)^2) / (k! 8^k)   (Hankel's expansion, Sec. 3.2;
// the printed product is garbled and is read as DLMF 10.17.1)
double hankel_coeff(int k, double nu)
{
    const double mu = 4.0 * nu * nu;
    double v = 1.0;
    for (int i = 1; i <= k; ++i) v *= (mu - (double)(2 * i - 1) * (double)(2 * i - 1)) / (8.0 * i);
    return v;
}

// psi(p) = log p + sqrt(1 - p^2) - log(1 + sqrt(1 - p^2)), 0 < p < 1 (Lemma 3.1)
static double siegel_psi(double p)
{
    const double s = std::sqrt(1.0 - p * p);
    return std::log(p) + s - std::log1p(s);
}

// Lemma 3.1: bound on the Wimp expansion truncated after l = L, at Omega R = x.
// Odd orders repeat the lemma's argument for the odd expansion (orders
// (nu+1)/2 + l and l - (nu-1)/2); the gamma term needs L + 1 > (nu or nu-1)/2
// strictly; outside Siegel's range the bound is infinite.
double bound_local(int nu, int L, double x)
{
    if (x <= 0.0) return 0.0;
    double d_beta, d_gamma, a_beta, a_gamma;
    bool use_gamma;
    if ((nu & 1) == 0) {
        d_beta = 2.0 * L + 2 + nu;
        d_gamma = 2.0 * L + 2 - nu;
        use_gamma = (L + 1) > nu / 2.0;
        a_beta = a_gamma = nu / 2.0;
    } else {
        d_beta = 2.0 * L + 3 + nu;
        d_gamma = 2.0 * L + 3 - nu;
        use_gamma = (L + 1) > (nu - 1) / 2.0;
        a_beta = (nu + 1) / 2.0;
        a_gamma = (nu - 1) / 2.0;
    }
    const double p = x / d_beta;
    if (p >= 1.0) return INFINITY;
    const double beta = siegel_psi(p);
    double gamma = 0.0;
    if (use_gamma) {
        const double pg = x / d_gamma;
        if (pg >= 1.0) return INFINITY;
        gamma = siegel_psi(pg);
    }
    if (beta + gamma >= 0.0) return INFINITY;
    return 2.0 * std::exp(a_beta * beta - a_gamma * gamma + (L + 1) * (beta + gamma)) /
           (1.0 - std::exp(beta + gamma));
}

// Remainder bound of the M-pair Hankel expansion at z (Sec. 3.2, eq. asy-error).
double bound_asy(int nu, int M, double z)
{
    return std::sqrt(2.0 / M_PI) * (std::fabs(hankel_coeff(2 * M, nu)) / std::pow(z, 2 * M + 0.5) +
                                    std::fabs(hankel_coeff(2 * M + 1, nu)) / std::pow(z, 2 * M + 1.5));
}

int heuristic_m(int nu, double eps)
{
    int M = (int)std::floor(1.0 + nu / 5.0 - std::log10(eps) / 4.0);
    return M > kMaxM ? kMaxM : (M < 1 ? 1 : M);
}

// z with B^asy(z) = eps: B^asy decreases in z; bisection on log z to full precision.
double crossover(int nu, int M, double eps)
{
    double lo = 1e-3, hi = 1.0;
    while (bound_asy(nu, M, hi) > eps) hi *= 2.0;
    while (bound_asy(nu, M, lo) < eps) lo *= 0.5;
    for (int it = 0; it < 200; ++it) {
        const double mid = std::sqrt(lo * hi);
        if (mid <= lo || mid >= hi) break;
        if (bound_asy(nu, M, mid) > eps) lo = mid; else hi = mid;
    }
    return hi;
}

int local_order(int nu, double z, double eps)
{
    for (int L = 0; L <= 4 * kMaxNtop; ++L)
        if (bound_local(nu, L, z) < eps) return L;
    return -1;
}

int choose_params(int nu, double eps, int m_terms, int* M, double* z, int* L)
{
    nu = nu < 0 ? -nu : nu;
    // a pure function of (nu, eps, m_terms) whose bisections take microseconds:
    // remembered, so that a batch of many problems of few orders pays once per order
    struct Key {
        int nu, m_terms;
        double eps;
        bool operator<(const Key& o) const
        {
            if (nu != o.nu) return nu < o.nu;
            if (m_terms != o.m_terms) return m_terms < o.m_terms;
            return eps < o.eps;
        }
    };
    struct Val {
        int M, L;
        double z;
    };
    static std::mutex mu;
    static std::map<Key, Val> cache;
    const Key key{nu, m_terms, eps};
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = cache.find(key);
        if (it != cache.end()) {
            *M = it->second.M;
            *z = it->second.z;
            *L = it->second.L;
            return *L < 0 ? NUHT_ERR_UNSUPPORTED : NUHT_OK;
        }
    }
    *M = m_terms > 0 ? m_terms : heuristic_m(nu, eps);
    *z = crossover(nu, *M, eps);
    *L = local_order(nu, *z, eps);
    {
        std::lock_guard<std::mutex> lock(mu);
        if (cache.size() < 4096) cache.emplace(key, Val{*M, *L, *z});
    }
    return *L < 0 ? NUHT_ERR_UNSUPPORTED : NUHT_OK;
}

// ----------------------------------------------------------- kernel tables
static double es_kernel(double t, double beta)
{
    if (std::fabs(t) > 1.0) return 0.0;
    return std::exp(beta * (std::sqrt(1.0 - t * t) - 1.0));
}

// Chebyshev interpolant of f on [-1, 1] (deg + 1 first-kind nodes), returned
// as monomial coefficients in v (and, if cheb is given, as the coefficients of
// T_0..T_deg).
template <class F>
static void cheb_monomial(F f, int deg, double* out, double* cheb = nullptr)
{
    const int n = deg + 1;
    std::vector<double> fv(n), c(n, 0.0);
    for (int k = 0; k < n; ++k) fv[k] = f(std::cos(M_PI * (k + 0.5) / n));
    for (int j = 0; j < n; ++j) {
        double s = 0.0;
        for (int k = 0; k < n; ++k) s += fv[k] * std::cos(j * M_PI * (k + 0.5) / n);
        c[j] = 2.0 * s / n;
    }
    c[0] *= 0.5;
    if (cheb)
        for (int j = 0; j < n; ++j) cheb[j] = c[j];
    // monomial coefficients of T_j by T_j = 2 v T_{j-1} - T_{j-2}
    std::vector<double> tm2(n, 0.0), tm1(n, 0.0), tj(n, 0.0);
    for (int i = 0; i < n; ++i) out[i] = 0.0;
    tm2[0] = 1.0;
    out[0] += c[0];
    if (n > 1) {
        tm1[1] = 1.0;
        out[1] += c[1];
    }
    for (int j = 2; j < n; ++j) {
        for (int i = 0; i < n; ++i) tj[i] = -tm2[i] + (i > 0 ? 2.0 * tm1[i - 1] : 0.0);
        for (int i = 0; i < n; ++i) out[i] += c[j] * tj[i];
        tm2.swap(tm1);
        tm1.swap(tj);
    }
}

// Gauss-Legendre nodes and weights on [-1, 1] (Newton on P_n).
static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w)
{
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        double pp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p1 = 1.0, p2 = 0.0;
            for (int j = 1; j <= n; ++j) {
                const double p3 = p2;
                p2 = p1;
                p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
            }
            pp = n * (z * p1 - p2) / (z * z - 1.0);
            const double dz = p1 / pp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = -z;
        x[n - 1 - i] = z;
        w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * pp * pp);
    }
}

// psi^(xi) = int_{-1}^{1} psi(t) cos(xi t) dt = 2 int_0^{pi/2} e^{beta(sin th - 1)} cos(xi cos th) sin th dth
static double es_fourier(double xi, double beta, const std::vector<double>& gx,
                         const std::vector<double>& gw)
{
    double s = 0.0;
    for (size_t i = 0; i < gx.size(); ++i) {
        const double th = (gx[i] + 1.0) * (M_PI / 4.0);
        s += gw[i] * std::exp(beta * (std::sin(th) - 1.0)) * std::cos(xi * std::cos(th)) * std::sin(th);
    }
    return 2.0 * s * (M_PI / 4.0);
}

const HostTables& kernel_tables(int w)
{
    static std::mutex mu;
    static std::map<int, HostTables> cache;
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(w);
    if (it != cache.end()) return it->second;
    HostTables T;
    T.w = w;
    T.beta = 2.30 * w;
    T.deg = w + 1 > kMaxDeg ? kMaxDeg : w + 1;
    T.es.assign((size_t)w * (T.deg + 1), 0.0);
    T.ch.assign((size_t)w * (T.deg + 1), 0.0);
    for (int i = 0; i < w; ++i) {
        auto f = [&](double v) { return es_kernel(-1.0 + ((v + 1.0) * 0.5 + i) * 2.0 / w, T.beta); };
        cheb_monomial(f, T.deg, &T.es[(size_t)i * (T.deg + 1)], &T.ch[(size_t)i * (T.deg + 1)]);
    }
    T.es2.resize(T.es.size());
    T.ch2.resize(T.ch.size());
    for (size_t i = 0; i < T.es.size(); ++i) {
        const float hi = (float)T.es[i];
        T.es2[i] = make_float2(hi, (float)(T.es[i] - (double)hi));
        const float ch = (float)T.ch[i];
        T.ch2[i] = make_float2(ch, (float)(T.ch[i] - (double)ch));
    }
    // psi^ on [0, xmax], xmax slightly above w pi / 4 (the largest argument used)
    std::vector<double> gx, gw;
    gauss_legendre(160, gx, gw);
    T.ph_xmax = w * M_PI / 4.0 * 1.02;
    T.ph_pieces = (int)std::ceil(T.ph_xmax / 0.5);
    T.ph_deg = 12;
    T.ph_scale = T.ph_pieces / T.ph_xmax;
    T.ph.assign((size_t)T.ph_pieces * (T.ph_deg + 1), 0.0);
    const double width = T.ph_xmax / T.ph_pieces;
    for (int p = 0; p < T.ph_pieces; ++p) {
        auto f = [&](double v) { return es_fourier((p + (v + 1.0) * 0.5) * width, T.beta, gx, gw); };
        cheb_monomial(f, T.ph_deg, &T.ph[(size_t)p * (T.ph_deg + 1)]);
    }
    T.ph2.resize(T.ph.size());
    for (size_t i = 0; i < T.ph.size(); ++i) {
        const float hi = (float)T.ph[i];
        T.ph2[i] = make_float2(hi, (float)(T.ph[i] - (double)hi));
    }
    // Degrees whose coefficient tail, rounded in FP32 (2^-23 relative), stays
    // below 1e-3 eps_w of the smallest psi^ on the piece, for the smallest
    // tolerance of this width, eps_w = 10^-(w - 1): the deconvolution factor's
    // relative error stays below 1e-3 eps.  The largest such degree over the
    // pieces bounds the compensated part of the Horner sums.
    {
        const int nc = T.ph_deg + 1;
        const double eps_w = std::pow(10.0, -(double)(w - 1));
        T.ph_comp = 0;
        for (int p = 0; p < T.ph_pieces; ++p) {
            const double* c = &T.ph[(size_t)p * nc];
            double mn = 1e300;
            for (int t = 0; t <= 64; ++t) {
                const double v = -1.0 + 2.0 * t / 64.0;
                double y = 0.0;
                for (int k = nc - 1; k >= 0; --k) y = y * v + c[k];
                mn = std::fmin(mn, std::fabs(y));
            }
            double tail = 0.0;
            int kc = -1;
            for (int k = nc - 1; k >= 0; --k) {
                tail += std::fabs(c[k]);
                if (tail * 1.1920928955078125e-07 > 1e-3 * eps_w * mn) { kc = k; break; }
            }
            T.ph_comp = kc > T.ph_comp ? kc : T.ph_comp;
        }
    }
    // twiddles e^{2 pi i k / 8192}, k < 4096 (single-CTA FFTs up to 8192 points)
    T.tw_log2 = 13;
    T.tw.assign((size_t)1 << (T.tw_log2 - 1), make_double2(0.0, 0.0));
    for (int k = 0; k < (1 << (T.tw_log2 - 1)); ++k) {
        const double a = 2.0 * M_PI * k / (double)(1 << T.tw_log2);
        T.tw[k] = make_double2(std::cos(a), std::sin(a));
    }
    T.tw2.resize(T.tw.size());
    for (size_t k = 0; k < T.tw.size(); ++k) {
        const float ch = (float)T.tw[k].x, sh = (float)T.tw[k].y;
        T.tw2[k] = make_float4(ch, (float)(T.tw[k].x - (double)ch), sh, (float)(T.tw[k].y - (double)sh));
    }
    return cache.emplace(w, std::move(T)).first->second;
}

int nufft_width(double eps)
{
    int w = (int)std::ceil(-std::log10(eps)) + 1;
    if (w < 2) w = 2;
    if (w > kMaxW) w = kMaxW;
    return w;
}

}  // namespace nuht
