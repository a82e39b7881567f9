// batch.cu -- kernels of wm_batch: several independent instances solved as one point set.
//
// The instances of a group (same minPts) are concatenated, with the coordinates an instance does
// not have set to 0 (they add exactly 0 to every distance); coordinate d (an extra one) holds
// j * L for instance j, with L a power of two larger than twice the diameter bound of every
// instance.  Two points of one instance differ by exactly 0 in that coordinate, so every FP32
// screen value and every FP64 key of a pair inside an instance is bit for bit the instance's own;
// two points of different instances are at least L apart, and the rounds cap rho_hi below L^2,
// so no pair of nodes from different instances is ever retrieved.  The tree edges found are the
// union of the instances' own K-minimum spanning trees.  For the ordered dendrogram the
// instances are chained by bridge edges of infinite weight between consecutive start points, so
// each instance's dendrogram is a subtree ordered from its own start point, and its plot a block.
#include "batch.cuh"

namespace wm {

namespace {

// instance of item t: the largest j with off[j] <= t (off ascending, off[0] = 0)
__device__ inline int inst_of(const long long *__restrict__ off, int k, long long t)
{
    int lo = 0, hi = k - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// instance j has dims[j] <= d coordinates; the others are 0 (they add exactly 0 to every distance)
__global__ void gather_kernel(const void *const *__restrict__ src, const int *__restrict__ dims,
                              const long long *__restrict__ base, int k, long long total, int d, int dtype, int layout,
                              double *__restrict__ raw, unsigned *__restrict__ maxabs)
{
    float mx = 0.f;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int j = inst_of(base, k, t);
        const long long i = t - base[j], nj = base[j + 1] - base[j];
        const int dj = dims[j];
        for (int c = 0; c < d; ++c) {
            double v = 0.0;
            if (c < dj) {
                const size_t s = layout == WM_SOA ? (size_t)c * nj + i : (size_t)i * dj + c;
                v = dtype == WM_F32 ? (double)((const float *)src[j])[s] : ((const double *)src[j])[s];
            }
            raw[(size_t)c * total + t] = v;
            const float a = (float)fabs(v);
            if (a > mx) mx = a;   // NaN never raises it; ingest rejects non-finite input
        }
        raw[(size_t)d * total + t] = (double)j;
    }
    for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx > 0.f) atomicMax(maxabs, __float_as_uint(mx));
}

__global__ void scale_kernel(double *__restrict__ x, long long total, double L)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x)
        x[t] *= L;   // j * L is exact: L is a power of two
}

// keys[g] = {hi = instance of tree edge g, lo = g}: sorted, they group the edges by instance in K order
__global__ void edge_inst_kernel(const EdgeK *__restrict__ E, int m, const long long *__restrict__ base, int k,
                                 EdgeK *__restrict__ keys)
{
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < m; g += gridDim.x * blockDim.x) {
        EdgeK key;
        key.hi = (unsigned long long)inst_of(base, k, edge_u(E[g]));
        key.lo = (unsigned long long)g;
        keys[g] = key;
    }
}

// position t of the grouped list: instance j, local index t - eoff[j]; stage the instance-local edge
__global__ void edge_place_kernel(const EdgeK *__restrict__ keys, const EdgeK *__restrict__ E, int m,
                                  const long long *__restrict__ base, int *__restrict__ local,
                                  wm_edge *__restrict__ stage, int *bad)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m; t += gridDim.x * blockDim.x) {
        const int g = (int)keys[t].lo, j = (int)keys[t].hi;
        const long long eo = base[j] - j;   // edges of the instances before j
        local[g] = (int)(t - eo);
        const EdgeK x = E[g];
        const long long u = edge_u(x) - base[j], v = edge_v(x) - base[j];
        if (u < 0 || v >= base[j + 1] - base[j]) atomicOr(bad, 1);
        wm_edge o;
        o.u = (int)u;
        o.v = (int)v;
        o.w = sqrt(edge_w2(x));
        stage[t] = o;
    }
}

// total weight of every instance: one block per instance, a fixed summation order
__global__ void inst_total_kernel(const wm_edge *__restrict__ stage, const long long *__restrict__ base, int k,
                                  double *__restrict__ tot)
{
    __shared__ double part[256];
    for (int j = blockIdx.x; j < k; j += gridDim.x) {
        const long long b = base[j] - j, e = base[j + 1] - (j + 1);
        double s = 0.0;
        for (long long t = b + threadIdx.x; t < e; t += blockDim.x) s += stage[t].w;
        part[threadIdx.x] = s;
        __syncthreads();
        for (int h = blockDim.x / 2; h; h >>= 1) {
            if ((int)threadIdx.x < h) part[threadIdx.x] += part[threadIdx.x + h];
            __syncthreads();
        }
        if (threadIdx.x == 0) tot[j] = part[0];
        __syncthreads();
    }
}

__global__ void cd_stage_kernel(const double *__restrict__ cd64, const int *__restrict__ pid, int total,
                                double *__restrict__ stage)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < total; p += gridDim.x * blockDim.x)
        stage[pid[p]] = sqrt(cd64[p]);
}

// tree edges followed by the bridges (s_j, s_{j+1}) of infinite weight: K order is kept
__global__ void bridge_kernel(const int *__restrict__ starts, int k, EdgeK *__restrict__ out)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j + 1 < k; j += gridDim.x * blockDim.x)
        out[j] = make_edge(INFINITY, starts[j], starts[j + 1]);
}

// merge g of the joint dendrogram (an instance's tree edge) -> node local[g] of that instance
__global__ void dendro_extract_kernel(const wm_dnode *__restrict__ dn, const EdgeK *__restrict__ E, int m,
                                      long long total, const long long *__restrict__ base, int k,
                                      const int *__restrict__ local, wm_dnode *__restrict__ stage, int *bad)
{
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < m; g += gridDim.x * blockDim.x) {
        const int j = inst_of(base, k, edge_u(E[g]));
        const long long nj = base[j + 1] - base[j];
        wm_dnode o = dn[g];
        long long c[2] = {o.left, o.right};
        for (int s = 0; s < 2; ++s) {
            if (c[s] < total) {
                c[s] -= base[j];
                if (c[s] < 0 || c[s] >= nj) atomicOr(bad, 1);
            } else {
                const long long h = c[s] - total;
                if (h >= m) { atomicOr(bad, 1); c[s] = 0; }
                else c[s] = nj + local[h];
            }
        }
        o.left = (int)c[0];
        o.right = (int)c[1];
        stage[(base[j] - j) + local[g]] = o;
    }
}

// the joint plot is the instances' plots one after another, instance 0 first; each block starts
// at its instance's start point, after an infinite bar
__global__ void order_extract_kernel(const int *__restrict__ order, const double *__restrict__ reach, long long total,
                                     const long long *__restrict__ base, int k, int *__restrict__ ostage,
                                     double *__restrict__ rstage, int *bad)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int p = order[t];
        const int j = inst_of(base, k, p);
        if (inst_of(base, k, t) != j) atomicOr(bad, 2);
        ostage[t] = (int)(p - base[j]);
        rstage[t] = t == base[j] ? (double)INFINITY : reach[t];
    }
}

template <typename T>
__global__ void scatter_out_kernel(const T *__restrict__ stage, long long cnt, const long long *__restrict__ off, int k,
                                   T *const *__restrict__ dst)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < cnt;
         t += (long long)gridDim.x * blockDim.x) {
        const int j = inst_of(off, k, t);
        if (dst[j]) dst[j][t - off[j]] = stage[t];
    }
}

}  // namespace

void batch_gather(const void *const *src, const int *dims, const long long *base, int k, long long total, int d,
                  int dtype, int layout, double *raw, unsigned *maxabs, cudaStream_t st)
{
    launch(gather_kernel, grid_for(total, 256), 256, 0, st, src, dims, base, k, total, d, dtype, layout, raw, maxabs);
}

void batch_scale(double *x, long long total, double L, cudaStream_t st)
{
    launch(scale_kernel, grid_for(total, 256), 256, 0, st, x, total, L);
}

void batch_edge_inst(const EdgeK *E, int m, const long long *base, int k, EdgeK *keys, cudaStream_t st)
{
    if (m > 0) launch(edge_inst_kernel, grid_for(m, 256), 256, 0, st, E, m, base, k, keys);
}

void batch_edge_place(const EdgeK *keys, const EdgeK *E, int m, const long long *base, int *local, wm_edge *stage,
                      int *bad, cudaStream_t st)
{
    if (m > 0) launch(edge_place_kernel, grid_for(m, 256), 256, 0, st, keys, E, m, base, local, stage, bad);
}

void batch_totals(const wm_edge *stage, const long long *base, int k, double *tot, cudaStream_t st)
{
    launch(inst_total_kernel, std::min(k, num_sms() * 16), 256, 0, st, stage, base, k, tot);
}

void batch_cd(const double *cd64, const int *pid, int total, double *stage, cudaStream_t st)
{
    launch(cd_stage_kernel, grid_for(total, 256), 256, 0, st, cd64, pid, total, stage);
}

void batch_bridges(const int *starts, int k, EdgeK *out, cudaStream_t st)
{
    if (k > 1) launch(bridge_kernel, grid_for(k, 256), 256, 0, st, starts, k, out);
}

void batch_dendro(const wm_dnode *dn, const EdgeK *E, int m, long long total, const long long *base, int k,
                  const int *local, wm_dnode *stage, int *bad, cudaStream_t st)
{
    if (m > 0) launch(dendro_extract_kernel, grid_for(m, 256), 256, 0, st, dn, E, m, total, base, k, local, stage, bad);
}

void batch_order(const int *order, const double *reach, long long total, const long long *base, int k, int *ostage,
                 double *rstage, int *bad, cudaStream_t st)
{
    launch(order_extract_kernel, grid_for(total, 256), 256, 0, st, order, reach, total, base, k, ostage, rstage, bad);
}

template <typename T>
void batch_scatter(const T *stage, long long cnt, const long long *off, int k, T *const *dst, cudaStream_t st)
{
    if (cnt > 0) launch(scatter_out_kernel<T>, grid_for(cnt, 256), 256, 0, st, stage, cnt, off, k, dst);
}

template void batch_scatter<wm_edge>(const wm_edge *, long long, const long long *, int, wm_edge *const *, cudaStream_t);
template void batch_scatter<double>(const double *, long long, const long long *, int, double *const *, cudaStream_t);
template void batch_scatter<wm_dnode>(const wm_dnode *, long long, const long long *, int, wm_dnode *const *,
                                      cudaStream_t);
template void batch_scatter<int>(const int *, long long, const long long *, int, int *const *, cudaStream_t);

}  // namespace wm
