// batch.cuh -- device steps of wm_batch (see batch.cu).
#pragma once

#include <algorithm>

#include "wm_internal.cuh"

namespace wm {

// raw[c * total + t] (SoA, d + 1 coordinates) from the instances' inputs src[j] (device, dims[j]
// <= d coordinates each, the rest 0), base[j] = first combined index of instance j (base[k] =
// total); coordinate d = j; *maxabs = max |x| bits
void batch_gather(const void *const *src, const int *dims, const long long *base, int k, long long total, int d,
                  int dtype, int layout, double *raw, unsigned *maxabs, cudaStream_t st);
void batch_scale(double *x, long long total, double L, cudaStream_t st);
void batch_edge_inst(const EdgeK *E, int m, const long long *base, int k, EdgeK *keys, cudaStream_t st);
void batch_edge_place(const EdgeK *keys, const EdgeK *E, int m, const long long *base, int *local, wm_edge *stage,
                      int *bad, cudaStream_t st);
void batch_totals(const wm_edge *stage, const long long *base, int k, double *tot, cudaStream_t st);
void batch_cd(const double *cd64, const int *pid, int total, double *stage, cudaStream_t st);
void batch_bridges(const int *starts, int k, EdgeK *out, cudaStream_t st);
void batch_dendro(const wm_dnode *dn, const EdgeK *E, int m, long long total, const long long *base, int k,
                  const int *local, wm_dnode *stage, int *bad, cudaStream_t st);
void batch_order(const int *order, const double *reach, long long total, const long long *base, int k, int *ostage,
                 double *rstage, int *bad, cudaStream_t st);
// dst[j][t - off[j]] = stage[t] for t in [off[j], off[j+1]) where dst[j] is not null
template <typename T>
void batch_scatter(const T *stage, long long cnt, const long long *off, int k, T *const *dst, cudaStream_t st);

}  // namespace wm
