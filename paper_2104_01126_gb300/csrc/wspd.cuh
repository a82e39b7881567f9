// wspd.cuh -- arguments of the WSPD traversal and BCCP kernels (see wspd.cu).
#pragma once

#include "wm_internal.cuh"

namespace wm {

struct TravArgs {
    int N = 0, n = 0, d = 0;
    const float *lo = nullptr, *hi = nullptr, *diam2 = nullptr;
    const int *begin = nullptr, *end = nullptr, *left = nullptr, *right = nullptr;
    const int *comp = nullptr;
    const float *cdmin = nullptr, *cdmax = nullptr;   // HDBSCAN* node bounds (null for EMST)
    const float *x32 = nullptr;
    const double *x64 = nullptr;
    const int *pid = nullptr;
    const float *cd32 = nullptr;                       // HDBSCAN* cd2 per tree position
    const double *cd64 = nullptr;
    double eta = 0.0;          // absolute distance error of the FP32 copy (FP64 input), else 0
    int fp64 = 0;              // plain FP64 form
    int beta = 2;
    double rho_lo = 0.0, rho_hi = 0.0;
    double *rho_out = nullptr; // GetRho result (WriteMin target)
    long long inline_max = 64; // pairs with |A||B| <= this are evaluated inside the traversal
    int frontier_cap = 0;
    int2 *big = nullptr;
    int *big_count = nullptr;
    int big_cap = 0;
    EdgeK *edges = nullptr;
    int *edge_count = nullptr;
    int edge_cap = 0;
    unsigned *overflow = nullptr;      // bit 0 frontier, bit 1 edges, bit 2 big pairs
    unsigned long long *stat = nullptr; // [0] pairs, [1] evals, [2] fp64 rechecks, [3] tile evals
};

void launch_comp_labels(const Tree &T, const Points &P, int *uf, cudaStream_t st);
int run_traversal(int mode, TravArgs &a, int2 *fa, int2 *fb, int *counters, cudaStream_t st, int *pinned,
                  unsigned *overflow_out, int *levels_out);
int run_bccp_tiles(TravArgs &a, int m, int *jobs, int *total, cudaStream_t st, Arena &ar, bool hdb, bool fp64);

}  // namespace wm
