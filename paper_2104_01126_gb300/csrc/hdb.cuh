// hdb.cuh -- HDBSCAN* state and the k-NN / dendrogram entry points (knn.cu, dendro.cu).
#pragma once

#include "wm_internal.cuh"

namespace wm {

constexpr int kMaxMinPts = 256;   // largest minPts of the k-NN pass

struct HdbState {
    double *cd64 = nullptr;   // cd2 per tree position (FP64, the exact squared core distance)
    float *cd32 = nullptr;    // cd2 per tree position rounded to nearest FP32 (screen copy)
    float *cdmin = nullptr;   // per node: min cd2 rounded down
    float *cdmax = nullptr;   // per node: max cd2 rounded up
    EdgeK *rep = nullptr;     // repair edges {(p,q): w2(p,q) <= cd2(p)} with mutual-reachability
    int nrep = 0;             //   weights, each pair once, in no particular order
};

int core_distances(Points &P, Tree &T, int min_pts, bool fp64, HdbState &H, Arena &ar, cudaStream_t st, int *pin,
                   wm_stats *stats);
int write_core_distances(const Points &P, const HdbState &H, double *out, Arena &ar, cudaStream_t st);
int dendrogram(const EdgeK *E, int n, int start, wm_dnode *out_dendro, int *out_order, double *out_reach, Arena &ar,
               cudaStream_t st, int *pin);
int dendrogram_impl(const EdgeK *E, int n, int start, int key_squared, wm_dnode *out_dendro, int *out_order,
                    double *out_reach, Arena &ar, cudaStream_t st, int *pin);
int edges_from_wm(const wm_edge *src, int n, EdgeK *out, int *bad, cudaStream_t st);

}  // namespace wm
