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
    int ph_pieces = 0, ph_deg = 0;
    double ph_scale = 0.0, ph_xmax = 0.0;
    std::vector<double> ph;     // [ph_pieces][ph_deg + 1]
    int tw_log2 = 0;
    std::vector<double2> tw;
};
const HostTables& kernel_tables(int w);

// Block of the subdivision: rows k0..k1 (sorted omega), columns j0..j1 (sorted r).
struct HBlock {
    int64_t k0, k1, j0, j1;
};

// Algorithm 1 with SplitIndices; r, w sorted ascending (local indices).
void subdivide(const double* r, int64_t n, const double* w, int64_t m, double z, int64_t min_size,
               int n_cand, std::vector<HBlock>& loc, std::vector<HBlock>& asy,
               std::vector<HBlock>& dir);

inline int spread_tile_points(int qmax) { return qmax > 16 ? 128 : 256; }
constexpr int kInterpTile = 128;
constexpr int kMomentTile = 2048;

}  // namespace nuht
