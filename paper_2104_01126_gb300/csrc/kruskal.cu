// kruskal.cu -- batched Kruskal over a union-find shared across rounds (Sec. 3.1.2
// "ParallelKruskal", Algorithms 2 and 3), made deterministic with reservations.
//
// A batch of edges sorted by K is accepted exactly as sequential Kruskal would accept it: edge i
// (its index in the sorted batch is its priority) finds the roots of its endpoints; equal roots
// reject it.  Otherwise it reserves both roots with a WriteMin of its priority.  An edge that
// holds the reservation of a root links that root under the other root and is accepted; edges
// that hold neither retry in the next step.  The lowest-priority edge touching a root always
// wins it, so every step accepts or rejects at least one edge, and an edge is accepted only when
// no earlier pending edge touches the component it links, which is the sequential condition.
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
    const int lane = threadIdx.x & 31;
    const int limit = (m + 31) & ~31;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t - lane < limit; t += gridDim.x * blockDim.x) {
        bool keep = false;
        EdgeK e;
        if (t < m) {
            e = in[t];
            keep = uf_find_ro(uf, edge_u(e)) != uf_find_ro(uf, edge_v(e));
        }
        unsigned b = __ballot_sync(0xffffffffu, keep);
        int base = 0;
        if (lane == 0 && b) base = atomicAdd(count, __popc(b));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (keep) out[base + __popc(b & lanemask_lt())] = e;
    }
}

// Every edge handed to Kruskal must have 0 <= u < v < n.
__global__ void validate_edges_kernel(const EdgeK *__restrict__ e, int m, int n, int *bad)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        int u = edge_u(e[i]), v = edge_v(e[i]);
        if (u < 0 || u >= v || v >= n) atomicOr(bad, 1);
    }
}

__global__ void init_list_kernel(int *list, int m, int *status)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        list[i] = i;
        status[i] = kPending;
    }
}

__global__ void reserve_kernel(const EdgeK *__restrict__ e, const int *__restrict__ list, const int *__restrict__ cnt,
                               int *uf, int *R, int2 *__restrict__ roots, int *__restrict__ status)
{
    const int m = *cnt;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
        int i = list[j];
        EdgeK x = e[i];
        int ru = uf_find_halving(uf, edge_u(x)), rv = uf_find_halving(uf, edge_v(x));
        if (ru == rv) {
            status[i] = kReject;
            roots[j] = make_int2(-1, -1);
        } else {
            roots[j] = make_int2(ru, rv);
            atomicMin(&R[ru], i);
            atomicMin(&R[rv], i);
        }
    }
}

__global__ void commit_kernel(const int *__restrict__ list, const int *__restrict__ cnt, int *uf, const int *__restrict__ R,
                              const int2 *__restrict__ roots, int *__restrict__ status)
{
    const int m = *cnt;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
        int2 r = roots[j];
        if (r.x < 0) continue;
        int i = list[j];
        if (R[r.y] == i) { uf[r.y] = r.x; status[i] = kAccept; }
        else if (R[r.x] == i) { uf[r.x] = r.y; status[i] = kAccept; }
    }
}

__global__ void reset_compact_kernel(const int *__restrict__ list, const int *__restrict__ cnt, int *R,
                                     const int2 *__restrict__ roots, const int *__restrict__ status,
                                     int *__restrict__ next, int *next_cnt, int *zero_me)
{
    const int m = *cnt;
    const int lane = threadIdx.x & 31;
    const int limit = (m + 31) & ~31;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j - lane < limit; j += gridDim.x * blockDim.x) {
        bool keep = false;
        int i = 0;
        if (j < m) {
            int2 r = roots[j];
            if (r.x >= 0) { R[r.x] = 0x7fffffff; R[r.y] = 0x7fffffff; }
            i = list[j];
            keep = status[i] == kPending;
        }
        unsigned b = __ballot_sync(0xffffffffu, keep);
        int base = 0;
        if (lane == 0 && b) base = atomicAdd(next_cnt, __popc(b));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (keep) next[base + __popc(b & lanemask_lt())] = i;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && zero_me) *zero_me = 0;
}

// Appends the accepted edges of the batch, in batch (K) order, to the output tree.
__global__ void flag_accept_kernel(const int *__restrict__ status, int m, int *__restrict__ flag)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) flag[i] = status[i] == kAccept;
}

__global__ void append_accept_kernel(const EdgeK *__restrict__ e, const int *__restrict__ status,
                                     const int *__restrict__ pre, int m, EdgeK *__restrict__ out, int out_base,
                                     int out_cap, int *bad)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
        if (status[i] == kAccept) {
            int k = out_base + pre[i];
            if (k < out_cap) out[k] = e[i];
            else atomicOr(bad, 2);
        }
}

}  // namespace

int filter_connected(const EdgeK *in, int m, const int *uf, EdgeK *out, int *count_dev, cudaStream_t st)
{
    cudaMemsetAsync(count_dev, 0, sizeof(int), st);
    if (m > 0) launch(filter_connected_kernel, grid_for(m, 256), 256, 0, st, in, m, uf, out, count_dev);
    return 0;
}

// Kruskal over a K-sorted batch e[0..m).  R[n] must hold INT_MAX everywhere on entry (kept so).
// Accepted edges are appended to out at out_base; *accepted receives their number.
int batch_kruskal(const EdgeK *e, int m, int n, int *uf, int *R, EdgeK *out, int out_base, int *accepted, Arena &ar,
                  cudaStream_t st, int *pinned)
{
    *accepted = 0;
    if (m <= 0) return 0;
    size_t mark = ar.off;
    int *listA = ar.get<int>(m), *listB = ar.get<int>(m), *status = ar.get<int>(m + 1), *pre = ar.get<int>(m + 1);
    int2 *roots = ar.get<int2>(m);
    int *cnt = ar.get<int>(4);
    int *bad = ar.get<int>(1);
    if (ar.failed) return WM_ENOMEM;
    cudaMemsetAsync(bad, 0, sizeof(int), st);
    launch(validate_edges_kernel, grid_for(m, 256), 256, 0, st, e, m, n, bad);
    cudaMemcpyAsync(pinned, bad, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return WM_ECUDA;
    if (pinned[0]) {
        set_error_detail("a candidate edge handed to Kruskal has an endpoint outside [0, n) or u >= v");
        return WM_EINTERNAL;
    }
    launch(init_list_kernel, grid_for(m, 256), 256, 0, st, listA, m, status);
    int hm = m;
    cudaMemcpyAsync(cnt, &hm, sizeof(int), cudaMemcpyHostToDevice, st);
    cudaMemsetAsync(cnt + 1, 0, sizeof(int), st);
    int step = 0;
    const int grid = grid_for(m, 256);
    while (true) {
        for (int b = 0; b < 4; ++b, ++step) {
            int *lin = (step & 1) ? listB : listA, *lout = (step & 1) ? listA : listB;
            int *cin = cnt + (step & 1), *cout = cnt + ((step + 1) & 1);
            launch(reserve_kernel, grid, 256, 0, st, e, lin, cin, uf, R, roots, status);
            launch(commit_kernel, grid, 256, 0, st, lin, cin, uf, R, roots, status);
            // cout must be zero before this kernel appends into it: it was consumed two steps ago
            launch(reset_compact_kernel, grid, 256, 0, st, lin, cin, R, roots, status, lout, cout, nullptr);
            // the consumed input counter becomes the next output counter: zero it now
            cudaMemsetAsync(cin, 0, sizeof(int), st);
        }
        cudaMemcpyAsync(pinned, cnt + (step & 1), sizeof(int), cudaMemcpyDeviceToHost, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) return WM_ECUDA;
        if (pinned[0] == 0) break;
        if (step > 4 * (m + 8)) {
            char msg[160];
            snprintf(msg, sizeof msg, "batched Kruskal made no progress (reservations): %d of %d edges pending",
                     pinned[0], m);
            set_error_detail(msg);
            return WM_EINTERNAL;
        }
    }
    launch(flag_accept_kernel, grid, 256, 0, st, status, m, pre);
    int rc = scan_exclusive_i32(pre, pre, m, cnt + 2, st, ar);
    if (rc) return rc;
    launch(append_accept_kernel, grid, 256, 0, st, e, status, pre, m, out, out_base, n - 1, bad);
    cudaMemcpyAsync(pinned, cnt + 2, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(pinned + 1, bad, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return WM_ECUDA;
    *accepted = pinned[0];
    if (pinned[1]) {
        set_error_detail("Kruskal accepted more than n-1 edges in total");
        return WM_EINTERNAL;
    }
    ar.off = mark;
    return 0;
}

}  // namespace wm
