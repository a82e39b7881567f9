// gfk.cu -- the list steps of the GFK and EMST-Naive forms (Sec. 3.2.2, Algorithm 2; Sec. 5's
// EMST-Naive): the well-separated pairs of the full WSPD are materialised once, and every round
// works on the lists:
//   split      pairs of at most beta points go to the BCCP size-class lists (their BCCP is
//              computed once; its edge joins the edge pool, which caches it), the rest are kept;
//   min bound  rho_hi = the smallest lower bound d(A,B) of the kept pairs;
//   partition  pool edges lighter than rho_hi form the round's Kruskal batch, the rest stay;
//   filter     pairs whose points are all connected, and pool edges whose endpoints are, go.
// All steps are stream compactions with warp-aggregated appends.
#include "wspd.cuh"

namespace wm {

namespace {

// appends the lanes with `take` to out at one counter increment per warp; returns the slot
__device__ inline int warp_slot(int *counter, bool take)
{
    const unsigned b = __ballot_sync(0xffffffffu, take);
    const int lane = threadIdx.x & 31;
    int base = 0;
    if (lane == 0 && b) base = atomicAdd(counter, __popc(b));
    base = __shfl_sync(0xffffffffu, base, 0);
    return base + __popc(b & lanemask_lt());
}

// size classes as in the traversal (by |A||B|)
__device__ inline int size_class(long long prod, int medium_max, long long big_max)
{
    return prod <= 8 ? 0 : prod <= 64 ? 1 : prod <= medium_max ? 2 : prod <= big_max ? 3 : 4;
}

__global__ void gfk_split_kernel(TravArgs a, const int2 *__restrict__ S, const float *__restrict__ lb, int m,
                                 long long beta, int2 *__restrict__ keep, float *__restrict__ keep_lb, int *keep_count)
{
    const int limit = (m + 31) & ~31;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < limit; t += gridDim.x * blockDim.x) {
        int2 p = make_int2(0, 0);
        float l = 0.f;
        long long sz = 0, prod = 0;
        if (t < m) {
            p = S[t];
            l = lb[t];
            const int4 u = a.rec[p.x].l, v = a.rec[p.y].l;
            sz = (long long)(u.y - u.x) + (v.y - v.x);
            prod = (long long)(u.y - u.x) * (v.y - v.x);
        }
        const bool small = t < m && sz <= beta;
        const int s = warp_slot(keep_count, t < m && !small);
        if (t < m && !small) { keep[s] = p; keep_lb[s] = l; }
        const int c = small ? size_class(prod, a.medium_max, a.big_max) : -1;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const int q = warp_slot(a.list_count + k, c == k);
            if (c == k) {
                if (q < a.list_cap[k]) { a.list[k][q] = p; a.list_lb[k][q] = l; }
                else atomicOr(a.overflow, 4u);
            }
        }
    }
}

__global__ void gfk_min_lb_kernel(const float *__restrict__ lb, int m, unsigned *rho_bits)
{
    float v = INFINITY;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m; t += gridDim.x * blockDim.x) v = fminf(v, lb[t]);
    for (int o = 16; o; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0 && v < INFINITY) atomicMin(rho_bits, __float_as_uint(v));   // non-negative floats
}

// pool edges with w2 < hi go to the batch, the others to rest (both compacted)
__global__ void gfk_partition_kernel(const EdgeK *__restrict__ pool, int m, double hi, EdgeK *__restrict__ batch,
                                     int *batch_count, int batch_cap, EdgeK *__restrict__ rest, int *rest_count,
                                     unsigned *overflow)
{
    const unsigned long long hb = (unsigned long long)__double_as_longlong(hi);
    const int limit = (m + 31) & ~31;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < limit; t += gridDim.x * blockDim.x) {
        EdgeK e;
        e.lo = e.hi = 0;
        if (t < m) e = pool[t];
        const bool now = t < m && e.hi < hb;
        const int sb = warp_slot(batch_count, now);
        if (now) {
            if (sb < batch_cap) batch[sb] = e;
            else atomicOr(overflow, 2u);
        }
        const int sr = warp_slot(rest_count, t < m && !now);
        if (t < m && !now) rest[sr] = e;
    }
}

// drops the pairs whose points all lie in one component (node labels in rec[x].l.w)
__global__ void gfk_filter_pairs_kernel(const int2 *__restrict__ S, const float *__restrict__ lb, int m,
                                        const NodeRec *__restrict__ rec, int2 *__restrict__ out, float *__restrict__ out_lb,
                                        int *count)
{
    const int limit = (m + 31) & ~31;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < limit; t += gridDim.x * blockDim.x) {
        bool keep = false;
        int2 p = make_int2(0, 0);
        float l = 0.f;
        if (t < m) {
            p = S[t];
            l = lb[t];
            const int ca = rec[p.x].l.w, cb = rec[p.y].l.w;
            keep = !(ca >= 0 && ca == cb);
        }
        const int s = warp_slot(count, keep);
        if (keep) { out[s] = p; out_lb[s] = l; }
    }
}

// drops the pool edges whose endpoints are already connected (uf flattened: roots)
__global__ void gfk_filter_edges_kernel(const EdgeK *__restrict__ pool, int m, const int *__restrict__ uf,
                                        EdgeK *__restrict__ out, int *count)
{
    const int limit = (m + 31) & ~31;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < limit; t += gridDim.x * blockDim.x) {
        bool keep = false;
        EdgeK e;
        e.lo = e.hi = 0;
        if (t < m) {
            e = pool[t];
            keep = uf[edge_u(e)] != uf[edge_v(e)];
        }
        const int s = warp_slot(count, keep);
        if (keep) out[s] = e;
    }
}

}  // namespace

void gfk_split(const TravArgs &a, const int2 *S, const float *lb, int m, long long beta, int2 *keep, float *keep_lb,
               int *keep_count, cudaStream_t st)
{
    if (m <= 0) return;
    launch(gfk_split_kernel, grid_for(m, 256), 256, 0, st, a, S, lb, m, beta, keep, keep_lb, keep_count);
}

void gfk_min_lb(const float *lb, int m, unsigned *rho_bits, cudaStream_t st)
{
    fill_i32((int *)rho_bits, 0x7f800000, 1, st);   // +inf
    if (m > 0) launch(gfk_min_lb_kernel, grid_for(m, 256), 256, 0, st, lb, m, rho_bits);
}

void gfk_partition(const EdgeK *pool, int m, double hi, EdgeK *batch, int *batch_count, int batch_cap, EdgeK *rest,
                   int *rest_count, unsigned *overflow, cudaStream_t st)
{
    if (m > 0)
        launch(gfk_partition_kernel, grid_for(m, 256), 256, 0, st, pool, m, hi, batch, batch_count, batch_cap, rest,
               rest_count, overflow);
}

void gfk_filter_pairs(const int2 *S, const float *lb, int m, const NodeRec *rec, int2 *out, float *out_lb, int *count,
                      cudaStream_t st)
{
    if (m > 0) launch(gfk_filter_pairs_kernel, grid_for(m, 256), 256, 0, st, S, lb, m, rec, out, out_lb, count);
}

void gfk_filter_edges(const EdgeK *pool, int m, const int *uf, EdgeK *out, int *count, cudaStream_t st)
{
    if (m > 0) launch(gfk_filter_edges_kernel, grid_for(m, 256), 256, 0, st, pool, m, uf, out, count);
}

}  // namespace wm
