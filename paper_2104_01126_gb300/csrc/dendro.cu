// dendro.cu -- ordered dendrogram and reachability plot of a weighted spanning tree (Sec. 4).
//
// Input: the n-1 tree edges sorted by K (rank i = position).  Dendrogram node n+i is the merge
// of edge i; leaves are the points.  The construction follows the top-down heavy/light scheme
// of Sec. 4.2 with the heavy set of a subproblem taken as the edges in the upper half of its
// rank interval (interval halves are global bit positions of the rank, so there are
// ceil(log2(n-1)) levels).  At each level, per subproblem:
//   light components  = connected components of the light edges over the current supervertices
//                       (union-find over supervertex ids);
//   a light component's dendrogram root (its heaviest light edge) hangs below the lightest
//   heavy edge incident to the component (a WriteMin), which is the first merge touching it;
//   heavy edges are relabelled to the light components' roots and form the next subproblem.
// Every leaf hangs below its lightest incident edge.
//
// Order (Sec. 4.2, ordering theorem): with the tree rooted at s, the child of merge (u,v) that
// contains the endpoint nearer s is the left child.  The tree is rooted by an Euler tour and list
// ranking (Sec. 2.2); a cluster lies on the far side of edge (u,v) iff a representative vertex of
// it lies in the Euler interval of the deeper endpoint.  The reachability plot is the in-order
// sequence of leaves, obtained by list ranking an Euler tour of the ordered dendrogram; the bar
// of leaf i is the height of the in-order internal node before it.
#include <cmath>
#include <cstring>

#include "hdb.cuh"

namespace wm {

namespace {

// ---------------------------------------------------------------------------- list ranking
// Pointer jumping (Wyllie): S[a] = sum of w from a to the end of its list.
__global__ void lr_init_kernel(const int *__restrict__ succ, const int *__restrict__ w, int m, int *__restrict__ nxt,
                               int *__restrict__ S)
{
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < m; a += gridDim.x * blockDim.x) {
        nxt[a] = succ[a];
        S[a] = w[a];
    }
}

__global__ void lr_step_kernel(const int *__restrict__ nxt, const int *__restrict__ S, int m, int *__restrict__ nxt2,
                               int *__restrict__ S2)
{
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < m; a += gridDim.x * blockDim.x) {
        int b = nxt[a];
        if (b >= 0) {
            S2[a] = S[a] + S[b];
            nxt2[a] = nxt[b];
        } else {
            S2[a] = S[a];
            nxt2[a] = -1;
        }
    }
}

// Ruling-set list ranking: every head and about one element in 16 (picked by a multiplicative
// hash of its index, so that no index pattern of the list lengthens the sublists) is a splitter.
// A splitter walks its sublist up to the next splitter (prefix sums on the way), the splitters'
// list is ranked by pointer jumping, and every element adds its splitter's rank: O(m) work, walks
// of about 16 dependent steps, pointer jumping over about m/16 elements.
__global__ void lr_mark_kernel(const int *__restrict__ succ, int m, int *__restrict__ haspred)
{
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < m; a += gridDim.x * blockDim.x)
        if (succ[a] >= 0) haspred[succ[a]] = 1;
}

__global__ void lr_flag_kernel(const int *__restrict__ haspred, int m, int *__restrict__ flag)
{
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < m; a += gridDim.x * blockDim.x)
        flag[a] = !haspred[a] || ((unsigned)a * 0x9E3779B1u) >> 28 == 0;
}

__global__ void lr_walk_kernel(const int *__restrict__ succ, const int *__restrict__ w, const int *__restrict__ flag,
                               const int *__restrict__ sid, int m, int *__restrict__ owner, int *__restrict__ pre,
                               int *__restrict__ snext, int *__restrict__ ssum)
{
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < m; a += gridDim.x * blockDim.x) {
        if (!flag[a]) continue;
        const int s = sid[a];
        int x = a, p = 0, nx = -1;
        for (int it = 0; it < m; ++it) {
            owner[x] = s;
            p += w[x];
            pre[x] = p;
            const int y = succ[x];
            if (y < 0) break;
            if (flag[y]) { nx = sid[y]; break; }
            x = y;
        }
        snext[s] = nx;
        ssum[s] = p;
    }
}

__global__ void lr_finish_kernel(const int *__restrict__ owner, const int *__restrict__ pre, const int *__restrict__ w,
                                 const int *__restrict__ SS, int m, int *__restrict__ S)
{
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < m; a += gridDim.x * blockDim.x)
        S[a] = SS[owner[a]] - pre[a] + w[a];
}

// --------------------------------------------------------------------------- Euler tour (tree)
__global__ void degree_kernel(const EdgeK *__restrict__ E, int m, int *deg)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        atomicAdd(&deg[edge_u(E[i])], 1);
        atomicAdd(&deg[edge_v(E[i])], 1);
    }
}

__global__ void adjacency_kernel(const EdgeK *__restrict__ E, int m, const int *__restrict__ off, int *cur,
                                 int *__restrict__ adj, int *__restrict__ slot_of)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        int u = edge_u(E[i]), v = edge_v(E[i]);
        int s0 = off[u] + atomicAdd(&cur[u], 1);
        adj[s0] = 2 * i;          // arc u -> v
        slot_of[2 * i] = s0;
        int s1 = off[v] + atomicAdd(&cur[v], 1);
        adj[s1] = 2 * i + 1;      // arc v -> u
        slot_of[2 * i + 1] = s1;
    }
}

__device__ inline int arc_head(const EdgeK *__restrict__ E, int a) { return (a & 1) ? edge_u(E[a >> 1]) : edge_v(E[a >> 1]); }

__global__ void tour_succ_kernel(const EdgeK *__restrict__ E, int m, const int *__restrict__ off,
                                 const int *__restrict__ adj, const int *__restrict__ slot_of, int s,
                                 int *__restrict__ succ, int *__restrict__ w)
{
    const int start = adj[off[s]];
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < 2 * m; a += gridDim.x * blockDim.x) {
        int y = arc_head(E, a);
        int p = slot_of[a ^ 1] + 1;
        if (p == off[y + 1]) p = off[y];
        int nx = adj[p];
        succ[a] = nx == start ? -1 : nx;
        w[a] = 1;
    }
}

// child endpoint (deeper) of each edge and the Euler interval of every vertex
__global__ void rooting_kernel(const EdgeK *__restrict__ E, int m, const int *__restrict__ S, int L,
                               int *__restrict__ child, int *__restrict__ tin, int *__restrict__ tout)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        int p0 = L - S[2 * i], p1 = L - S[2 * i + 1];   // tour positions of the two arcs
        int down = p0 < p1 ? 2 * i : 2 * i + 1;
        int c = arc_head(E, down);
        child[i] = c;
        tin[c] = p0 < p1 ? p0 : p1;
        tout[c] = p0 < p1 ? p1 : p0;
    }
}

// ------------------------------------------------------------------ heavy/light recursion
__global__ void leaf_parent_kernel(const EdgeK *__restrict__ E, int m, int *pmin)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        atomicMin(&pmin[edge_u(E[i])], i);
        atomicMin(&pmin[edge_v(E[i])], i);
    }
}

__global__ void leaf_parent_set_kernel(const int *__restrict__ pmin, int n, int *__restrict__ par)
{
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x)
        par[x] = pmin[x] == 0x7fffffff ? -1 : n + pmin[x];
}

__global__ void endpoints_init_kernel(const EdgeK *__restrict__ E, int m, int *__restrict__ ex, int *__restrict__ ey)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        ex[i] = edge_u(E[i]);
        ey[i] = edge_v(E[i]);
    }
}

__device__ inline int uf_find(int *uf, int x)
{
    for (int it = 0; it < (1 << 30); ++it) {
        int p = uf[x];
        if (p == x) return x;
        int g = uf[p];
        if (g != p) uf[x] = g;
        x = p;
    }
    return x;
}

__global__ void level_init_kernel(const int *__restrict__ ex, const int *__restrict__ ey, int m, int *uf, int *rootrank,
                                  int *minheavy)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        int a = ex[i], b = ey[i];
        uf[a] = a; uf[b] = b;
        rootrank[a] = -1; rootrank[b] = -1;
        minheavy[a] = 0x7fffffff; minheavy[b] = 0x7fffffff;
    }
}

__global__ void level_union_kernel(const int *__restrict__ ex, const int *__restrict__ ey, int m, int bit, int *uf)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        if ((i >> bit) & 1) continue;   // heavy at this level
        int x = ex[i], y = ey[i];
        for (int it = 0; it < (1 << 24); ++it) {
            int a = uf_find(uf, x), b = uf_find(uf, y);
            if (a == b) break;
            if (a > b) { int t = a; a = b; b = t; }
            if (atomicCAS(&uf[b], b, a) == b) break;
        }
    }
}

// Component roots of every edge's endpoints (rx, ry; ry for heavy edges only), rootrank (largest
// light edge of a component) and minheavy (smallest heavy edge touching it).  The updates are
// aggregated per warp: edges of one warp often share a component (a large one at the top levels),
// so each group of equal roots issues one atomic.
__global__ void level_mark_kernel(const int *__restrict__ ex, const int *__restrict__ ey, int m, int bit, int *uf,
                                  int *rootrank, int *minheavy, int *__restrict__ rx, int *__restrict__ ry)
{
    const int lane = threadIdx.x & 31;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i - lane < m; i += gridDim.x * blockDim.x) {
        const bool ok = i < m;
        const bool light = ok && ((i >> bit) & 1) == 0, heavy = ok && !light;
        const int kx = ok ? uf_find(uf, ex[i]) : -1;
        const int ky = heavy ? uf_find(uf, ey[i]) : -1;
        if (ok) { rx[i] = kx; ry[i] = ky; }
        int key = light ? kx : -1;
        unsigned grp = __match_any_sync(0xffffffffu, key);
        int v = __reduce_max_sync(grp, light ? i : -1);
        if (key >= 0 && lane == __ffs(grp) - 1) atomicMax(&rootrank[key], v);
        key = heavy ? kx : -1;
        grp = __match_any_sync(0xffffffffu, key);
        v = __reduce_min_sync(grp, heavy ? i : 0x7fffffff);
        if (key >= 0 && lane == __ffs(grp) - 1) atomicMin(&minheavy[key], v);
        grp = __match_any_sync(0xffffffffu, ky);
        v = __reduce_min_sync(grp, heavy ? i : 0x7fffffff);
        if (ky >= 0 && lane == __ffs(grp) - 1) atomicMin(&minheavy[ky], v);
    }
}

// Parents of the light components' top merges; heavy endpoints relabelled to their component's
// top merge.  The next level's union-find entries and its (other) rootrank / minheavy set are
// initialised here for the endpoints each edge has from now on: this level reads neither.
__global__ void level_link_kernel(int *ex, int *ey, int m, int bit, int n, const int *__restrict__ rx,
                                  const int *__restrict__ ry, const int *__restrict__ rootrank,
                                  const int *__restrict__ minheavy, int *__restrict__ par, int *uf, int *rr_next,
                                  int *mh_next)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        int x = ex[i], y = ey[i];
        if (((i >> bit) & 1) == 0) {
            const int c = rx[i];
            if (rootrank[c] == i && minheavy[c] != 0x7fffffff) par[n + i] = n + minheavy[c];
        } else {
            const int cx = rx[i], cy = ry[i];
            x = rootrank[cx] >= 0 ? n + rootrank[cx] : cx;
            y = rootrank[cy] >= 0 ? n + rootrank[cy] : cy;
            ex[i] = x;
            ey[i] = y;
        }
        uf[x] = x; uf[y] = y;
        rr_next[x] = -1; rr_next[y] = -1;
        mh_next[x] = 0x7fffffff; mh_next[y] = 0x7fffffff;
    }
}

// The lowest kLeafLevels levels: the subproblems are aligned blocks of at most kLeafChunk edges
// that share no vertex (after the relabelling of the levels above, every vertex and merge node
// occurs in one subproblem of a level), so one CTA runs all of them for its block in shared
// memory.  Vertices get local ids on entry (the first occurrence claims map[v]); the merge node
// of local edge r is 2 * kLeafChunk + r.  The steps of a level are those of the global kernels.
constexpr int kLeafLevels = 11;
constexpr int kLeafChunk = 1 << kLeafLevels;
constexpr int kLeafThreads = 1024;
constexpr int kLeafSmem = (3 * 3 * kLeafChunk + 2 * kLeafChunk) * (int)sizeof(int);   // uf, rr, mh; lx, ly

__device__ inline int sm_find(int *uf, int x)
{
    for (int it = 0; it < 3 * kLeafChunk; ++it) {
        int p = uf[x];
        if (p == x) return x;
        int g = uf[p];
        if (g != p) uf[x] = g;
        x = p;
    }
    return x;
}

__global__ void __launch_bounds__(kLeafThreads) level_leaf_kernel(const int *__restrict__ ex, const int *__restrict__ ey,
                                                                  int m, int n, int top, int *map,
                                                                  int *__restrict__ par)
{
    extern __shared__ int leaf_smem[];
    int *uf = leaf_smem, *rr = uf + 3 * kLeafChunk, *mh = rr + 3 * kLeafChunk;
    int *lx = mh + 3 * kLeafChunk, *ly = lx + kLeafChunk;
    const int b = blockIdx.x * kLeafChunk;
    const int cnt = min(kLeafChunk, m - b);
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
        const int me = 2 * t;
        int prev = atomicCAS(&map[ex[b + t]], -1, me);
        lx[t] = prev < 0 ? me : prev;
        prev = atomicCAS(&map[ey[b + t]], -1, me + 1);
        ly[t] = prev < 0 ? me + 1 : prev;
    }
    for (int bit = top - 1; bit >= 0; --bit) {
        for (int v = threadIdx.x; v < 3 * kLeafChunk; v += blockDim.x) {
            uf[v] = v;
            rr[v] = -1;
            mh[v] = 0x7fffffff;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
            if ((t >> bit) & 1) continue;
            const int x = lx[t], y = ly[t];
            for (int it = 0; it < 3 * kLeafChunk; ++it) {
                int a = sm_find(uf, x), c = sm_find(uf, y);
                if (a == c) break;
                if (a > c) { int q = a; a = c; c = q; }
                if (atomicCAS(&uf[c], c, a) == c) break;
            }
        }
        __syncthreads();
        for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
            if (((t >> bit) & 1) == 0) {
                atomicMax(&rr[sm_find(uf, lx[t])], t);
            } else {
                atomicMin(&mh[sm_find(uf, lx[t])], t);
                atomicMin(&mh[sm_find(uf, ly[t])], t);
            }
        }
        __syncthreads();
        for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
            if (((t >> bit) & 1) == 0) {
                const int c = sm_find(uf, lx[t]);
                if (rr[c] == t && mh[c] != 0x7fffffff) par[n + b + t] = n + b + mh[c];
            } else {
                const int cx = sm_find(uf, lx[t]), cy = sm_find(uf, ly[t]);
                lx[t] = rr[cx] >= 0 ? 2 * kLeafChunk + rr[cx] : cx;
                ly[t] = rr[cy] >= 0 ? 2 * kLeafChunk + rr[cy] : cy;
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------------ children / order
__global__ void children_kernel(const int *__restrict__ par, int total, int n, int *nch, int *__restrict__ ch,
                                int *bad)
{
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < total; x += gridDim.x * blockDim.x) {
        int p = par[x];
        if (p < 0) {
            if (x != total - 1) atomicOr(bad, 1);   // only the last merge is the root
            continue;
        }
        int s = atomicAdd(&nch[p - n], 1);
        if (s < 2) ch[2 * (p - n) + s] = x;
        else atomicOr(bad, 2);
    }
}

__global__ void order_children_kernel(const EdgeK *__restrict__ E, int m, int n, const int *__restrict__ ch,
                                      const int *__restrict__ nch, const int *__restrict__ child,
                                      const int *__restrict__ tin, const int *__restrict__ tout,
                                      int *__restrict__ lc, int *__restrict__ rc, int *bad)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        if (nch[i] != 2) { atomicOr(bad, 4); continue; }
        int c = child[i];
        int a = ch[2 * i], b = ch[2 * i + 1];
        int ra = a < n ? a : edge_u(E[a - n]);
        int rb = b < n ? b : edge_u(E[b - n]);
        bool ina = tin[ra] >= tin[c] && tin[ra] <= tout[c];
        bool inb = tin[rb] >= tin[c] && tin[rb] <= tout[c];
        if (ina == inb) { atomicOr(bad, 8); continue; }
        lc[i] = ina ? b : a;
        rc[i] = ina ? a : b;
    }
}

// Euler tour of the ordered dendrogram: event 2x = enter x, 2x+1 = exit x.
__global__ void dtour_kernel(int total, int n, const int *__restrict__ par, const int *__restrict__ lc,
                             const int *__restrict__ rc, int *__restrict__ succ, int *__restrict__ w)
{
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < total; x += gridDim.x * blockDim.x) {
        bool leaf = x < n;
        succ[2 * x] = leaf ? 2 * x + 1 : 2 * lc[x - n];
        w[2 * x] = leaf ? 1 : 0;
        int p = par[x];
        int sx;
        if (p < 0) sx = -1;
        else if (lc[p - n] == x) sx = 2 * rc[p - n];
        else sx = 2 * p + 1;
        succ[2 * x + 1] = sx;
        w[2 * x + 1] = 0;
    }
}

__global__ void dendro_out_kernel(const EdgeK *__restrict__ E, int m, int n, const int *__restrict__ lc,
                                  const int *__restrict__ rc, const int *__restrict__ S, int key_squared,
                                  wm_dnode *__restrict__ out_d, double *__restrict__ reach)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        int x = n + i;
        double key = edge_w2(E[i]);
        double h = key_squared ? sqrt(key) : key;
        if (out_d) {
            wm_dnode o;
            o.left = lc[i];
            o.right = rc[i];
            o.height = h;
            o.size = S[2 * x] - S[2 * x + 1];
            o.reserved = 0;
            out_d[i] = o;
        }
        if (reach) reach[n - S[2 * rc[i]]] = h;
    }
}

__global__ void order_out_kernel(int n, const int *__restrict__ S, int *__restrict__ order, double *reach)
{
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
        int idx = n - S[2 * x];
        if (order) order[idx] = x;
        if (reach && idx == 0) reach[0] = INFINITY;
    }
}

__global__ void wm_to_edgek_kernel(const wm_edge *__restrict__ src, int m, int n, EdgeK *__restrict__ out, int *bad)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        wm_edge e = src[i];
        if (e.u < 0 || e.u >= n || e.v < 0 || e.v >= n || e.u == e.v || !(e.w >= 0.0) || isinf(e.w)) {
            atomicOr(bad, 1);
            e.u = 0; e.v = 0; e.w = 0.0;
        }
        out[i] = make_edge(e.w, e.u, e.v);
    }
}

}  // namespace

int edges_from_wm(const wm_edge *src, int n, EdgeK *out, int *bad, cudaStream_t st)
{
    cudaMemsetAsync(bad, 0, sizeof(int), st);
    if (n > 1) launch(wm_to_edgek_kernel, grid_for(n - 1, 256), 256, 0, st, src, n - 1, n, out, bad);
    return 0;
}

static bool dev_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) { cudaGetLastError(); return false; }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// pointer jumping over m elements (the splitter list)
static int wyllie(const int *succ, const int *w, int m, int *S, Arena &ar, cudaStream_t st)
{
    size_t mark = ar.off;
    int *n0 = ar.get<int>(m), *n1 = ar.get<int>(m), *S1 = ar.get<int>(m);
    if (ar.failed) return WM_ENOMEM;
    int g = grid_for(m, 256);
    launch(lr_init_kernel, g, 256, 0, st, succ, w, m, n0, S);
    int steps = 1;
    while ((1LL << steps) < (long long)m) ++steps;
    int *na = n0, *nb = n1, *Sa = S, *Sb = S1;
    for (int t = 0; t < steps + 1; ++t) {
        launch(lr_step_kernel, g, 256, 0, st, na, Sa, m, nb, Sb);
        int *x = na; na = nb; nb = x;
        x = Sa; Sa = Sb; Sb = x;
    }
    if (Sa != S) cudaMemcpyAsync(S, Sa, sizeof(int) * m, cudaMemcpyDeviceToDevice, st);
    ar.off = mark;
    return 0;
}

// S[a] = sum of w over the list from a to its end (inclusive), for every element of the lists
// given by succ (-1 ends a list).
static int list_rank(const int *succ, const int *w, int m, int *S, Arena &ar, cudaStream_t st, int *pin)
{
    if (m <= 0) return 0;
    size_t mark = ar.off;
    int *haspred = ar.get<int>(m), *flag = ar.get<int>(m + 1), *sid = ar.get<int>(m + 1);
    int *owner = ar.get<int>(m), *pre = ar.get<int>(m);
    int *snext = ar.get<int>(m), *ssum = ar.get<int>(m), *SS = ar.get<int>(m), *ns_d = ar.get<int>(1);
    if (ar.failed) return WM_ENOMEM;
    const int g = grid_for(m, 256);
    cudaMemsetAsync(haspred, 0, sizeof(int) * m, st);
    launch(lr_mark_kernel, g, 256, 0, st, succ, m, haspred);
    launch(lr_flag_kernel, g, 256, 0, st, haspred, m, flag);
    int rc = scan_exclusive_i32(flag, sid, m, ns_d, st, ar);
    if (rc) return rc;
    launch(lr_walk_kernel, g, 256, 0, st, succ, w, flag, sid, m, owner, pre, snext, ssum);
    cudaMemcpyAsync(pin, ns_d, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return WM_ECUDA;
    const int ns = pin[0];
    rc = wyllie(snext, ssum, ns, SS, ar, st);
    if (rc) return rc;
    launch(lr_finish_kernel, g, 256, 0, st, owner, pre, w, SS, m, S);
    ar.off = mark;
    return 0;
}

// E: n-1 edges sorted by K on the device; key_squared: keys are squared weights (heights = sqrt)
int dendrogram_impl(const EdgeK *E, int n, int start, int key_squared, wm_dnode *out_dendro, int *out_order,
                    double *out_reach, Arena &ar, cudaStream_t st, int *pin)
{
    if (!out_dendro && !out_order && !out_reach) return 0;
    size_t mark = ar.off;
    const bool dd = dev_ptr(out_dendro), dor = dev_ptr(out_order), dre = dev_ptr(out_reach);
    if (n == 1) {
        int z = 0;
        double inf = INFINITY;
        if (out_order) {
            if (dor) cudaMemcpyAsync(out_order, &z, sizeof(int), cudaMemcpyHostToDevice, st);
            else *out_order = 0;
        }
        if (out_reach) {
            if (dre) cudaMemcpyAsync(out_reach, &inf, sizeof(double), cudaMemcpyHostToDevice, st);
            else *out_reach = inf;
        }
        return cudaStreamSynchronize(st) == cudaSuccess ? 0 : WM_ECUDA;
    }
    const int m = n - 1, total = 2 * n - 1, L = 2 * m;
    int *deg = ar.get<int>(n + 1), *cur = ar.get<int>(n), *adj = ar.get<int>(L), *slot = ar.get<int>(L);
    int *succ = ar.get<int>(2 * total), *w = ar.get<int>(2 * total), *S = ar.get<int>(2 * total);
    int *child = ar.get<int>(m), *tin = ar.get<int>(n), *tout = ar.get<int>(n);
    int *par = ar.get<int>(total), *pmin = ar.get<int>(n), *ex = ar.get<int>(m), *ey = ar.get<int>(m);
    int *uf = ar.get<int>(total), *rootrank = ar.get<int>(total), *minheavy = ar.get<int>(total);
    int *rootrank2 = ar.get<int>(total), *minheavy2 = ar.get<int>(total), *rxa = ar.get<int>(m), *rya = ar.get<int>(m);
    int *nch = ar.get<int>(m), *ch = ar.get<int>(2 * m), *lc = ar.get<int>(m), *rc = ar.get<int>(m);
    int *bad = ar.get<int>(1);
    if (ar.failed) return WM_ENOMEM;
    const int g = grid_for(total, 256);
    cudaMemsetAsync(bad, 0, sizeof(int), st);
    // ---- root the tree at start: Euler tour + list ranking
    cudaMemsetAsync(deg, 0, sizeof(int) * (n + 1), st);
    cudaMemsetAsync(cur, 0, sizeof(int) * n, st);
    launch(degree_kernel, g, 256, 0, st, E, m, deg);
    int rc0 = scan_exclusive_i32(deg, deg, n + 1, nullptr, st, ar);
    if (rc0) return rc0;
    launch(adjacency_kernel, g, 256, 0, st, E, m, deg, cur, adj, slot);
    launch(tour_succ_kernel, g, 256, 0, st, E, m, deg, adj, slot, start, succ, w);
    rc0 = list_rank(succ, w, L, S, ar, st, pin);
    if (rc0) return rc0;
    fill_i32(tin, -1, n, st);
    {
        int hl = L;
        cudaMemcpyAsync(tout + start, &hl, sizeof(int), cudaMemcpyHostToDevice, st);
    }
    launch(rooting_kernel, g, 256, 0, st, E, m, S, L, child, tin, tout);
    {
        int neg = -1;
        cudaMemcpyAsync(tin + start, &neg, sizeof(int), cudaMemcpyHostToDevice, st);
    }
    // ---- merge parents (heavy/light levels)
    fill_i32(pmin, 0x7fffffff, n, st);
    fill_i32(par, -1, total, st);
    launch(leaf_parent_kernel, g, 256, 0, st, E, m, pmin);
    launch(leaf_parent_set_kernel, g, 256, 0, st, pmin, n, par);
    launch(endpoints_init_kernel, g, 256, 0, st, E, m, ex, ey);
    int levels = 0;
    while ((1LL << levels) < (long long)m) ++levels;
    if (levels > kLeafLevels) launch(level_init_kernel, g, 256, 0, st, ex, ey, m, uf, rootrank, minheavy);
    for (int k = levels, set = 0; k > kLeafLevels; --k, set ^= 1) {
        const int bit = k - 1;
        int *rr = set ? rootrank2 : rootrank, *mh = set ? minheavy2 : minheavy;
        int *rrn = set ? rootrank : rootrank2, *mhn = set ? minheavy : minheavy2;
        launch(level_union_kernel, g, 256, 0, st, ex, ey, m, bit, uf);
        launch(level_mark_kernel, g, 256, 0, st, ex, ey, m, bit, uf, rr, mh, rxa, rya);
        launch(level_link_kernel, g, 256, 0, st, ex, ey, m, bit, n, rxa, rya, rr, mh, par, uf, rrn, mhn);
    }
    fill_i32(uf, -1, total, st);
    cudaFuncSetAttribute(level_leaf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kLeafSmem);
    launch(level_leaf_kernel, (m + kLeafChunk - 1) / kLeafChunk, kLeafThreads, kLeafSmem, st, ex, ey, m, n,
           std::min(levels, kLeafLevels), uf, par);
    // ---- children, left/right, in-order
    cudaMemsetAsync(nch, 0, sizeof(int) * m, st);
    launch(children_kernel, g, 256, 0, st, par, total, n, nch, ch, bad);
    launch(order_children_kernel, g, 256, 0, st, E, m, n, ch, nch, child, tin, tout, lc, rc, bad);
    launch(dtour_kernel, g, 256, 0, st, total, n, par, lc, rc, succ, w);
    rc0 = list_rank(succ, w, 2 * total, S, ar, st, pin);
    if (rc0) return rc0;
    wm_dnode *od = out_dendro;
    int *oo = out_order;
    double *orr = out_reach;
    if (out_dendro && !dd) od = ar.get<wm_dnode>(m);
    if (out_order && !dor) oo = ar.get<int>(n);
    if (out_reach && !dre) orr = ar.get<double>(n);
    if (ar.failed) return WM_ENOMEM;
    launch(dendro_out_kernel, g, 256, 0, st, E, m, n, lc, rc, S, key_squared, od, orr);
    launch(order_out_kernel, g, 256, 0, st, n, S, oo, orr);
    if (out_dendro && !dd) cudaMemcpyAsync(out_dendro, od, sizeof(wm_dnode) * m, cudaMemcpyDeviceToHost, st);
    if (out_order && !dor) cudaMemcpyAsync(out_order, oo, sizeof(int) * n, cudaMemcpyDeviceToHost, st);
    if (out_reach && !dre) cudaMemcpyAsync(out_reach, orr, sizeof(double) * n, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(pin, bad, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return WM_ECUDA;
    ar.off = mark;
    return pin[0] ? WM_EINTERNAL : 0;
}

int dendrogram(const EdgeK *E, int n, int start, wm_dnode *out_dendro, int *out_order, double *out_reach, Arena &ar,
               cudaStream_t st, int *pin)
{
    return dendrogram_impl(E, n, start, 1, out_dendro, out_order, out_reach, ar, st, pin);
}

}  // namespace wm
