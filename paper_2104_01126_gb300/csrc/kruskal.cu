// kruskal.cu -- batched Kruskal over a union-find shared across rounds (Sec. 3.2.2
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
#include <algorithm>
#include <cstdio>

#include "wm_internal.cuh"

namespace wm {

namespace {

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

__global__ void init_list_kernel(int *list, int m)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) list[i] = i;
}

// The reservations of step s live in set s & 1; set (s - 1) & 1, written by the previous step, is
// cleared here (its roots list and count are intact until the next step), so a step needs no
// separate reset pass.
__device__ inline void clear_reservations(const int2 *__restrict__ roots, int m, unsigned long long *Rhi,
                                          unsigned long long *Rlo)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
        const int2 r = roots[j];
        if (r.x >= 0) {
            Rhi[r.x] = ~0ull; Rhi[r.y] = ~0ull;
            Rlo[r.x] = ~0ull; Rlo[r.y] = ~0ull;
        }
    }
}

struct StepArgs {
    const EdgeK *e;
    const int *list;          // pending edges of this step
    const int *cnt;           // their number
    int2 *roots;              // roots of each pending edge (-1: rejected)
    unsigned long long *Rhi, *Rlo;   // reservation set of this step
    const int2 *prev_roots;   // previous step: roots, count, reservation set (cleared here)
    const int *prev_cnt;
    unsigned long long *prev_hi, *prev_lo;
    int *zero_cnt;            // the counter the next step appends into: zeroed here
    int *next;                // pending edges after this step, and their counter
    int *next_cnt;
};

// Finds the roots; rejects edges inside one component (and invalid edges, flagged in *bad: every
// edge must have 0 <= u < v < n); WriteMin of the w2 bits on both roots.
__global__ void reserve_hi_kernel(StepArgs a, int n, int *uf, int *bad)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) *a.zero_cnt = 0;
    clear_reservations(a.prev_roots, *a.prev_cnt, a.prev_hi, a.prev_lo);
    const int m = *a.cnt;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
        const EdgeK x = a.e[a.list[j]];
        const int u = edge_u(x), v = edge_v(x);
        if (u < 0 || u >= v || v >= n) {
            atomicOr(bad, 1);
            a.roots[j] = make_int2(-1, -1);
            continue;
        }
        const int ru = uf_find_halving(uf, u), rv = uf_find_halving(uf, v);
        if (ru == rv) {
            a.roots[j] = make_int2(-1, -1);
        } else {
            a.roots[j] = make_int2(ru, rv);
            // a WriteMin that cannot lower the value is skipped (many edges share a big root)
            if (x.hi < *(volatile unsigned long long *)&a.Rhi[ru]) atomicMin(&a.Rhi[ru], x.hi);
            if (x.hi < *(volatile unsigned long long *)&a.Rhi[rv]) atomicMin(&a.Rhi[rv], x.hi);
        }
    }
}

// Among the edges that won the w2 WriteMin of a root: WriteMin of the id pair.
__global__ void reserve_lo_kernel(StepArgs a)
{
    const int m = *a.cnt;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
        const int2 r = a.roots[j];
        if (r.x < 0) continue;
        const EdgeK x = a.e[a.list[j]];
        if (a.Rhi[r.x] == x.hi && x.lo < *(volatile unsigned long long *)&a.Rlo[r.x]) atomicMin(&a.Rlo[r.x], x.lo);
        if (a.Rhi[r.y] == x.hi && x.lo < *(volatile unsigned long long *)&a.Rlo[r.y]) atomicMin(&a.Rlo[r.y], x.lo);
    }
}

// warp-aggregated append of the lanes with has set
template <typename T>
__device__ inline void warp_append(const T &x, bool has, T *out, int *out_count, int out_cap, int *bad)
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

// The holder of a root's reservation links that root under the other root and is accepted
// (appended to the output, in no particular order); edges that hold neither stay pending and
// are appended to the next list.
__global__ void commit_kernel(StepArgs a, int *uf, EdgeK *__restrict__ out, int *out_count, int out_cap, int *bad)
{
    __shared__ int sh[32];
    const int m = *a.cnt;
    // block-uniform loop: the appends take one counter atomic per block (a batch of millions of
    // edges would otherwise serialise tens of thousands of warps on two counters)
    for (int b0 = blockIdx.x * blockDim.x; b0 < m; b0 += gridDim.x * blockDim.x) {
        const int j = b0 + threadIdx.x;
        bool acc = false, keep = false;
        int i = 0;
        EdgeK x;
        x.hi = 0; x.lo = 0;
        if (j < m) {
            const int2 r = a.roots[j];
            if (r.x >= 0) {
                i = a.list[j];
                x = a.e[i];
                if (a.Rhi[r.y] == x.hi && a.Rlo[r.y] == x.lo) acc = atomicCAS(&uf[r.y], r.y, r.x) == r.y;
                else if (a.Rhi[r.x] == x.hi && a.Rlo[r.x] == x.lo) acc = atomicCAS(&uf[r.x], r.x, r.y) == r.x;
                keep = !acc;
            }
        }
        int slot = block_append(out_count, acc ? 1 : 0, sh);
        if (acc) {
            if (slot < out_cap) out[slot] = x;
            else atomicOr(bad, 2);
        }
        slot = block_append(a.next_cnt, keep ? 1 : 0, sh);
        if (keep) a.next[slot] = i;
    }
}

// The last steps of a batch, when few edges are pending: one CTA runs the steps to the end with
// block barriers between the phases instead of kernel boundaries (the phases are those of the
// kernels above; reservations use the step's set and are cleared after each step).  It does
// nothing when more than kTailMax edges are pending; the host then runs more grid-wide steps.
constexpr int kTailThreads = 1024, kTailMax = 16384;

__global__ void __launch_bounds__(kTailThreads) tail_kernel(StepArgs a, int *cnt_in, int *prev_cnt, int n, int *uf,
                                                            EdgeK *__restrict__ out, int *out_count, int out_cap,
                                                            int *bad)
{
    __shared__ int s_next;
    const int m0 = *cnt_in;
    if (m0 == 0 || m0 > kTailMax) return;
    const int lane = threadIdx.x & 31;
    clear_reservations(a.prev_roots, *prev_cnt, a.prev_hi, a.prev_lo);
    __syncthreads();
    if (threadIdx.x == 0) *prev_cnt = 0;
    int *lin = const_cast<int *>(a.list), *lout = a.next;
    int m = m0;
    for (int it = 0; it < m0 + 8 && m > 0; ++it) {
        if (threadIdx.x == 0) s_next = 0;
        for (int j = threadIdx.x; j < m; j += blockDim.x) {
            const EdgeK x = a.e[lin[j]];
            const int u = edge_u(x), v = edge_v(x);
            if (u < 0 || u >= v || v >= n) {
                atomicOr(bad, 1);
                a.roots[j] = make_int2(-1, -1);
                continue;
            }
            const int ru = uf_find_halving(uf, u), rv = uf_find_halving(uf, v);
            if (ru == rv) {
                a.roots[j] = make_int2(-1, -1);
            } else {
                a.roots[j] = make_int2(ru, rv);
                if (x.hi < *(volatile unsigned long long *)&a.Rhi[ru]) atomicMin(&a.Rhi[ru], x.hi);
                if (x.hi < *(volatile unsigned long long *)&a.Rhi[rv]) atomicMin(&a.Rhi[rv], x.hi);
            }
        }
        __syncthreads();
        for (int j = threadIdx.x; j < m; j += blockDim.x) {
            const int2 r = a.roots[j];
            if (r.x < 0) continue;
            const EdgeK x = a.e[lin[j]];
            if (a.Rhi[r.x] == x.hi && x.lo < *(volatile unsigned long long *)&a.Rlo[r.x]) atomicMin(&a.Rlo[r.x], x.lo);
            if (a.Rhi[r.y] == x.hi && x.lo < *(volatile unsigned long long *)&a.Rlo[r.y]) atomicMin(&a.Rlo[r.y], x.lo);
        }
        __syncthreads();
        const int limit = (m + 31) & ~31;
        for (int j = threadIdx.x; j - lane < limit; j += blockDim.x) {
            bool acc = false, keep = false;
            int i = 0;
            EdgeK x;
            x.hi = 0; x.lo = 0;
            if (j < m) {
                const int2 r = a.roots[j];
                if (r.x >= 0) {
                    i = lin[j];
                    x = a.e[i];
                    if (a.Rhi[r.y] == x.hi && a.Rlo[r.y] == x.lo) acc = atomicCAS(&uf[r.y], r.y, r.x) == r.y;
                    else if (a.Rhi[r.x] == x.hi && a.Rlo[r.x] == x.lo) acc = atomicCAS(&uf[r.x], r.x, r.y) == r.x;
                    keep = !acc;
                }
            }
            warp_append(x, acc, out, out_count, out_cap, bad);
            warp_append(i, keep, lout, &s_next, 0x7fffffff, bad);
        }
        __syncthreads();
        for (int j = threadIdx.x; j < m; j += blockDim.x) {
            const int2 r = a.roots[j];
            if (r.x >= 0) {
                a.Rhi[r.x] = ~0ull; a.Rhi[r.y] = ~0ull;
                a.Rlo[r.x] = ~0ull; a.Rlo[r.y] = ~0ull;
            }
        }
        m = s_next;
        int *t = lin; lin = lout; lout = t;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *cnt_in = m;
        if (m > 0) atomicOr(bad, 4);
    }
}

__global__ void clear_kernel(const int2 *__restrict__ roots, const int *__restrict__ cnt, unsigned long long *Rhi,
                             unsigned long long *Rlo)
{
    clear_reservations(roots, *cnt, Rhi, Rlo);
}

}  // namespace

// Kruskal over the batch e[0..m) (any order).  R holds 4 n 64-bit reservation words (two sets
// of two), all ~0 on entry (kept so).  Accepted edges are appended to out at out_base (in no
// particular order); *accepted receives their number.
int batch_kruskal(const EdgeK *e, int m, int n, int *uf, unsigned long long *R, EdgeK *out, int out_base, int *accepted,
                  Arena &ar, cudaStream_t st, int *pinned)
{
    *accepted = 0;
    if (m <= 0) return 0;
    size_t mark = ar.off;
    int *list[2] = {ar.get<int>(m), ar.get<int>(m)};
    int2 *roots[2] = {ar.get<int2>(m), ar.get<int2>(m)};
    // [0..3] pending counts (step s reads s % 4, appends into (s + 1) % 4, zeroes (s + 2) % 4),
    // [4] accepted, [5] bad
    int *cnt = ar.get<int>(8);
    if (ar.failed) return WM_ENOMEM;
    unsigned long long *Rhi[2] = {R, R + 2LL * n}, *Rlo[2] = {R + n, R + 3LL * n};
    launch(init_list_kernel, grid_for(m, 256), 256, 0, st, list[0], m);
    const int init[8] = {m, 0, 0, 0, 0, 0, 0, 0};   // pageable source: copied out before the call returns
    cudaMemcpyAsync(cnt, init, sizeof init, cudaMemcpyHostToDevice, st);
    int step = 0;
    const int grid = grid_for(m, 256);
    auto args = [&](int s) {
        const int c = s & 1, p = c ^ 1;
        StepArgs a;
        a.e = e;
        a.list = list[c];
        a.cnt = cnt + (s & 3);
        a.roots = roots[c];
        a.Rhi = Rhi[c];
        a.Rlo = Rlo[c];
        a.prev_roots = roots[p];
        a.prev_cnt = cnt + ((s + 3) & 3);   // 0 before the first step
        a.prev_hi = Rhi[p];
        a.prev_lo = Rlo[p];
        a.zero_cnt = cnt + ((s + 2) & 3);
        a.next = list[p];
        a.next_cnt = cnt + ((s + 1) & 3);
        return a;
    };
    int base_m = m, base_step = 0;   // pending edges at the last host sync, and that step
    while (true) {
        for (int b = 0; b < 4; ++b, ++step) {
            // the pending list shrinks by a factor of about 2 to 4 per step: a smaller grid (the
            // loops are grid-strided, so any size is correct) keeps the nearly empty steps short
            const int g = std::max(num_sms(), grid_for(std::max(1, base_m >> std::min(step - base_step, 30)), 256));
            const StepArgs a = args(step);
            launch(reserve_hi_kernel, g, 256, 0, st, a, n, uf, cnt + 5);
            launch(reserve_lo_kernel, g, 256, 0, st, a);
            launch(commit_kernel, g, 256, 0, st, a, uf, out + out_base, cnt + 4, n - 1 - out_base, cnt + 5);
        }
        launch(tail_kernel, 1, kTailThreads, 0, st, args(step), cnt + (step & 3), cnt + ((step + 3) & 3), n, uf,
               out + out_base, cnt + 4, n - 1 - out_base, cnt + 5);
        cudaMemcpyAsync(pinned, cnt, 6 * sizeof(int), cudaMemcpyDeviceToHost, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) return WM_ECUDA;
        if (pinned[5] & 1) {
            set_error_detail("a candidate edge handed to Kruskal has an endpoint outside [0, n) or u >= v");
            return WM_EINTERNAL;
        }
        if (pinned[5] & 2) {
            set_error_detail("Kruskal accepted more than n-1 edges in total");
            return WM_EINTERNAL;
        }
        if (pinned[5] & 4) {
            set_error_detail("batched Kruskal made no progress in its single-block steps");
            return WM_EINTERNAL;
        }
        if (pinned[step & 3] == 0) break;
        base_m = pinned[step & 3];
        base_step = step;
        if (step > 4 * (m + 8)) {
            char msg[160];
            snprintf(msg, sizeof msg, "batched Kruskal made no progress (reservations): %d of %d edges pending",
                     pinned[step & 3], m);
            set_error_detail(msg);
            return WM_EINTERNAL;
        }
    }
    // the last step's reservations are still set
    const int last = (step - 1) & 1;
    launch(clear_kernel, grid, 256, 0, st, roots[last], cnt + ((step - 1) & 3), Rhi[last], Rlo[last]);
    *accepted = pinned[4];
    ar.off = mark;
    return 0;
}

}  // namespace wm
