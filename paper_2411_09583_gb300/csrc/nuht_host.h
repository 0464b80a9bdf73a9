// Host-only internals: parameter choice, kernel tables, subdivision, plan.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "nuht_internal.h"

namespace nuht {

double hankel_coeff(int k, double nu);
double bound_local(int nu, int L, double x);
double bound_asy(int nu, int M, double z);
int heuristic_m(int nu, double eps);
double crossover(int nu, int M, double eps);
int local_order(int nu, double z, double eps);
int choose_params(int nu, double eps, int m_terms, int* M, double* z, int* L);
int nufft_width(double eps);

struct HostTables {
    int w = 0, deg = 0;
    double beta = 0.0;
    std::vector<double> es;     // [w][deg + 1]
    std::vector<float2> es2;    // the same split into (hi, lo) floats
    std::vector<double> ch;     // [w][deg + 1] the same pieces as coefficients of T_0..T_deg(v)
    std::vector<float2> ch2;    // the same split into (hi, lo) floats
    int ph_pieces = 0, ph_deg = 0;
    int ph_comp = 0;            // psi-hat degrees above this one may be summed in plain FP32
    double ph_scale = 0.0, ph_xmax = 0.0;
    std::vector<double> ph;     // [ph_pieces][ph_deg + 1]
    std::vector<float2> ph2;    // the same split into (hi, lo) floats
    int tw_log2 = 0;
    std::vector<double2> tw;
    std::vector<float4> tw2;    // the same as double-float (cos.h, cos.l, sin.h, sin.l)
};
const HostTables& kernel_tables(int w);

// Block of the subdivision: rows k0..k1 (sorted omega), columns j0..j1 (sorted r).
struct HBlock {
    int64_t k0, k1, j0, j1;
    int32_t prob = 0;   // problem of a batch
    // sorted values at the edges (r_j0, r_j1, omega_k0, omega_k1), filled by the plan
    double b[4] = {0.0, 0.0, 0.0, 0.0};
};

// Algorithm 1 with SplitIndices on the sorted matrix, from the staircase
// stair[k] = max{j : omega_k r_j <= z} (or -1) of every row.
// r, omega: the problem's sorted values (for the size limit of asymptotic blocks).
void subdivide(const int32_t* stair, const double* r, const double* omega, int64_t n, int64_t m,
               int64_t min_size, int n_cand, std::vector<HBlock>& loc, std::vector<HBlock>& asy,
               std::vector<HBlock>& dir);

// Host check of a work list (exact cover, block classes, direct-block area);
// ranges holds (k0, k1, j0, j1) per block in sorted indices, cls its class.
bool check_blocks(const double* r, int64_t n, const double* omega, int64_t m, double z, int64_t min_size,
                  const int64_t* ranges, const int32_t* cls, int64_t count);

// Device memory from the library's pool (kept reserved between plans) and
// pinned host staging buffers (grow-only, used under stage_lock()).
cudaError_t pool_alloc(void** p, size_t bytes, cudaStream_t s);
void pool_free(void* p, cudaStream_t s);

inline int spread_tile_points(int qmax) { return qmax > 16 ? 128 : 256; }
constexpr int kInterpTileMax = 256;   // frequencies per interpolation tile: 256 (default) or 128
constexpr int kMomentTile = 2048;

}  // namespace nuht
