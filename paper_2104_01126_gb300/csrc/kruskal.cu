// kruskal.cu -- batched Kruskal over a union-find shared across rounds (Sec. 3.1.2
// "ParallelKruskal", Algorithms 2 and 3), made deterministic with reservations.
//
// A batch of edges is accepted exactly as sequential Kruskal would accept it in the order of the
// key K = (w2, min id, max id), without sorting the batch: every pending edge finds the roots of
// its endpoints; equal roots reject it.  Otherwise it reserves both roots with a WriteMin of its
// key (two 64-bit WriteMins: the w2 bits, then, among the edges with the winning w2, the id
// pair).  An edge that holds the reservation of a root links that root under the other root and
// is accepted; edges that hold neither retry in the next step.  The K-smallest pending edge
// touching a root always wins it, so every step accepts or rejects at least one edge, and an
// edge is accepted only when no K-smaller pending edge touches the component it links, which is
// the sequential condition.  Exact copies of an edge (the same key twice in a batch) all win the
// same root; the link is a compare-and-swap, so one copy links and the others are rejected in
// the next step.
#include <cstdio>

#include "wm_internal.cuh"

namespace wm {

namespace {

constexpr int kPending = 0, kAccept = 1, kReject = 2;

// Every loop that follows union-find pointers is bounded: a valid forest over n < 2^30 vertices
// has no path longer than n, so the bound is never reached unless the structure is corrupt.
constexpr int kChaseLimit = 1 << 30;

__device__ inline int uf_find_halving(int *uf, int x)
{
    for (int it = 0; it < kChaseLimit; ++it) {
        int p = uf[x];
        if (p == x) return x;
        int g = uf[p];
        if (g == p) return p;
        uf[x] = g;   // path halving: g is an ancestor of x in the current (static) forest
        x = g;
    }
    return x;
}

__device__ inline int uf_find_ro(const int *uf, int x)
{
    for (int it = 0; it < kChaseLimit; ++it) {
        int p = uf[x];
        if (p == x) return x;
        x = p;
    }
    return x;
}

// Drops edges whose endpoints are already connected (the union-find is flat here).
__global__ void filter_connected_kernel(const EdgeK *__restrict__ in, int m, const int *__restrict__ uf,
                                        EdgeK *__restrict__ out, int *count)
{
    __shared__ int sh[32];
    for (int b0 = blockIdx.x * blockDim.x; b0 < m; b0 += gridDim.x * blockDim.x) {
        const int t = b0 + threadIdx.x;
        bool keep = false;
        EdgeK e;
        if (t < m) {
            e = in[t];
            keep = uf_find_ro(uf, edge_u(e)) != uf_find_ro(uf, edge_v(e));
        }
        const int slot = block_append(count, keep ? 1 : 0, sh);
        if (keep) out[slot] = e;
    }
}

__global__ void init_list_kernel(int *list, int m, int *status)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        list[i] = i;
        status[i] = kPending;
    }
}

// Finds the roots; rejects edges inside one component (and invalid edges, flagged in *bad: every
// edge must have 0 <= u < v < n); WriteMin of the w2 bits on both roots.
__global__ void reserve_hi_kernel(const EdgeK *__restrict__ e, const int *__restrict__ list, const int *__restrict__ cnt,
                                  int n, int *uf, unsigned long long *Rhi, int2 *__restrict__ roots,
                                  int *__restrict__ status, int *bad)
{
    const int m = *cnt;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
        const int i = list[j];
        const EdgeK x = e[i];
        const int u = edge_u(x), v = edge_v(x);
        if (u < 0 || u >= v || v >= n) {
            atomicOr(bad, 1);
            status[i] = kReject;
            roots[j] = make_int2(-1, -1);
            continue;
        }
        const int ru = uf_find_halving(uf, u), rv = uf_find_halving(uf, v);
        if (ru == rv) {
            status[i] = kReject;
            roots[j] = make_int2(-1, -1);
        } else {
            roots[j] = make_int2(ru, rv);
            // a WriteMin that cannot lower the value is skipped (many edges share a big root)
            if (x.hi < *(volatile unsigned long long *)&Rhi[ru]) atomicMin(&Rhi[ru], x.hi);
            if (x.hi < *(volatile unsigned long long *)&Rhi[rv]) atomicMin(&Rhi[rv], x.hi);
        }
    }
}

// Among the edges that won the w2 WriteMin of a root: WriteMin of the id pair.
__global__ void reserve_lo_kernel(const EdgeK *__restrict__ e, const int *__restrict__ list, const int *__restrict__ cnt,
                                  const unsigned long long *__restrict__ Rhi, unsigned long long *Rlo,
                                  const int2 *__restrict__ roots)
{
    const int m = *cnt;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
        const int2 r = roots[j];
        if (r.x < 0) continue;
        const EdgeK x = e[list[j]];
        if (Rhi[r.x] == x.hi && x.lo < *(volatile unsigned long long *)&Rlo[r.x]) atomicMin(&Rlo[r.x], x.lo);
        if (Rhi[r.y] == x.hi && x.lo < *(volatile unsigned long long *)&Rlo[r.y]) atomicMin(&Rlo[r.y], x.lo);
    }
}

__device__ inline void append_edge(const EdgeK &x, bool has, EdgeK *out, int *out_count, int out_cap, int *bad)
{
    const int lane = threadIdx.x & 31;
    const unsigned b = __ballot_sync(0xffffffffu, has);
    int base = 0;
    if (lane == 0 && b) base = atomicAdd(out_count, __popc(b));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (has) {
        const int k = base + __popc(b & lanemask_lt());
        if (k < out_cap) out[k] = x;
        else atomicOr(bad, 2);
    }
}

// The holder of a root's reservation links that root under the other root and is accepted.
// Accepted edges are appended to the output (in no particular order).
__global__ void commit_kernel(const EdgeK *__restrict__ e, const int *__restrict__ list, const int *__restrict__ cnt,
                              int *uf, const unsigned long long *__restrict__ Rhi,
                              const unsigned long long *__restrict__ Rlo, const int2 *__restrict__ roots,
                              int *__restrict__ status, EdgeK *__restrict__ out, int *out_count, int out_cap, int *bad)
{
    const int m = *cnt;
    const int lane = threadIdx.x & 31;
    const int limit = (m + 31) & ~31;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j - lane < limit; j += gridDim.x * blockDim.x) {
        bool acc = false;
        EdgeK x;
        x.hi = 0; x.lo = 0;
        if (j < m) {
            const int2 r = roots[j];
            if (r.x >= 0) {
                const int i = list[j];
                x = e[i];
                if (Rhi[r.y] == x.hi && Rlo[r.y] == x.lo) acc = atomicCAS(&uf[r.y], r.y, r.x) == r.y;
                else if (Rhi[r.x] == x.hi && Rlo[r.x] == x.lo) acc = atomicCAS(&uf[r.x], r.x, r.y) == r.x;
                if (acc) status[i] = kAccept;
            }
        }
        append_edge(x, acc, out, out_count, out_cap, bad);
    }
}

// Clears the reservations that were made and compacts the pending edges.
__global__ void reset_compact_kernel(const int *__restrict__ list, const int *__restrict__ cnt, unsigned long long *Rhi,
                                     unsigned long long *Rlo, const int2 *__restrict__ roots,
                                     const int *__restrict__ status, int *__restrict__ next, int *next_cnt)
{
    __shared__ int sh[32];
    const int m = *cnt;
    for (int b0 = blockIdx.x * blockDim.x; b0 < m; b0 += gridDim.x * blockDim.x) {
        const int j = b0 + threadIdx.x;
        bool keep = false;
        int i = 0;
        if (j < m) {
            const int2 r = roots[j];
            if (r.x >= 0) {
                Rhi[r.x] = ~0ull; Rhi[r.y] = ~0ull;
                Rlo[r.x] = ~0ull; Rlo[r.y] = ~0ull;
            }
            i = list[j];
            keep = status[i] == kPending;
        }
        const int slot = block_append(next_cnt, keep ? 1 : 0, sh);
        if (keep) next[slot] = i;
    }
}

}  // namespace

int filter_connected(const EdgeK *in, int m, const int *uf, EdgeK *out, int *count_dev, cudaStream_t st)
{
    cudaMemsetAsync(count_dev, 0, sizeof(int), st);
    if (m > 0) launch(filter_connected_kernel, grid_for(m, 256), 256, 0, st, in, m, uf, out, count_dev);
    return 0;
}

// Kruskal over the batch e[0..m) (any order).  R holds 2 n 64-bit reservation words, all ~0 on
// entry (kept so).  Accepted edges are appended to out at out_base (in no particular order);
// *accepted receives their number.
int batch_kruskal(const EdgeK *e, int m, int n, int *uf, unsigned long long *R, EdgeK *out, int out_base, int *accepted,
                  Arena &ar, cudaStream_t st, int *pinned)
{
    *accepted = 0;
    if (m <= 0) return 0;
    size_t mark = ar.off;
    int *listA = ar.get<int>(m), *listB = ar.get<int>(m), *status = ar.get<int>(m);
    int2 *roots = ar.get<int2>(m);
    int *cnt = ar.get<int>(4);   // [0] / [1] pending counts, [2] accepted, [3] bad
    if (ar.failed) return WM_ENOMEM;
    unsigned long long *Rhi = R, *Rlo = R + n;
    launch(init_list_kernel, grid_for(m, 256), 256, 0, st, listA, m, status);
    const int init[4] = {m, 0, 0, 0};   // pageable source: copied out before the call returns
    cudaMemcpyAsync(cnt, init, sizeof init, cudaMemcpyHostToDevice, st);
    int step = 0;
    const int grid = grid_for(m, 256);
    while (true) {
        for (int b = 0; b < 4; ++b, ++step) {
            int *lin = (step & 1) ? listB : listA, *lout = (step & 1) ? listA : listB;
            int *cin = cnt + (step & 1), *cout = cnt + ((step + 1) & 1);
            launch(reserve_hi_kernel, grid, 256, 0, st, e, lin, cin, n, uf, Rhi, roots, status, cnt + 3);
            launch(reserve_lo_kernel, grid, 256, 0, st, e, lin, cin, Rhi, Rlo, roots);
            launch(commit_kernel, grid, 256, 0, st, e, lin, cin, uf, Rhi, Rlo, roots, status, out + out_base,
                   cnt + 2, n - 1 - out_base, cnt + 3);
            // cout must be zero before this kernel appends into it: it was consumed two steps ago
            launch(reset_compact_kernel, grid, 256, 0, st, lin, cin, Rhi, Rlo, roots, status, lout, cout);
            // the consumed input counter becomes the next output counter: zero it now
            cudaMemsetAsync(cin, 0, sizeof(int), st);
        }
        cudaMemcpyAsync(pinned, cnt, 4 * sizeof(int), cudaMemcpyDeviceToHost, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) return WM_ECUDA;
        if (pinned[3] & 1) {
            set_error_detail("a candidate edge handed to Kruskal has an endpoint outside [0, n) or u >= v");
            return WM_EINTERNAL;
        }
        if (pinned[3] & 2) {
            set_error_detail("Kruskal accepted more than n-1 edges in total");
            return WM_EINTERNAL;
        }
        if (pinned[step & 1] == 0) break;
        if (step > 4 * (m + 8)) {
            char msg[160];
            snprintf(msg, sizeof msg, "batched Kruskal made no progress (reservations): %d of %d edges pending",
                     pinned[step & 1], m);
            set_error_detail(msg);
            return WM_EINTERNAL;
        }
    }
    *accepted = pinned[2];
    ar.off = mark;
    return 0;
}

}  // namespace wm
