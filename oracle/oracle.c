/*
 * oracle.c -- plain, slow, obviously correct FP64 CPU reference for EMST and HDBSCAN*.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline
 * and reference legs load this code.  The CUDA library never links, calls or includes it, and it
 * shares no source, header, table or helper with the CUDA path.
 *
 * What it computes (Wang, Yu, Gu, Shun, "Fast Parallel Algorithms for Euclidean Minimum
 * Spanning Tree and Hierarchical Spatial Clustering", SIGMOD'21):
 *   - EMST: a minimum spanning tree of the complete Euclidean graph (Sec. 2.1, "EMST").
 *   - Core distance cd(p): distance from p to its minPts-th nearest neighbour, p itself counted
 *     (Sec. 2.1, "HDBSCAN*").
 *   - Mutual reachability d_m(p,q) = max{cd(p), cd(q), d(p,q)} and the MST of that complete
 *     graph G_MR (Sec. 2.1).
 *   - The dendrogram: removing MST edges in decreasing weight order splits clusters; equivalently
 *     merging in increasing order with union-find (Sec. 4, first paragraphs).
 *   - The ordered dendrogram of a start point s: for the node of tree edge (u,v) with u nearer s
 *     (unweighted hop distance), u's side is the left child (Sec. 4.2, proof of the ordering
 *     theorem); its in-order leaves are the reachability plot.
 *   - The reachability plot: points in the order Prim's algorithm visits them on the MST from s,
 *     each bar the weight of the edge that reached it (Sec. 2.1, "reachability plot").
 *
 * Conventions fixed here (the paper leaves them open):
 *   - Squared distance D(p,q) = sum_{k=0}^{d-1} (x_k(p) - x_k(q))^2 evaluated in IEEE FP64 in
 *     dimension order k = 0..d-1, one rounding per subtract, multiply and add, no fused
 *     multiply-add (this file is compiled with -ffp-contract=off).
 *   - Every edge comparison uses the strict total key K(u,v) = (w2, min(u,v), max(u,v)) compared
 *     lexicographically, w2 the squared weight.  The MST under K is unique.
 *   - Reported weights are sqrt(w2) (IEEE correctly rounded).
 *
 * Points are row-major: x[i*d + k] is coordinate k of point i.
 *
 * The definitions are evaluated by brute force (wmo_core_dist2, wmo_prim).  For sizes brute
 * force cannot reach, wmo_core_dist2_kdtree and wmo_boruvka compute the same values by exact
 * searches over a k-d tree (end of this file); tests/test_oracle.py pins them to the brute force.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ distances (Sec. 2.1) */

double wmo_sqdist(const double *x, int32_t d, int64_t i, int64_t j)
{
    const double *a = x + i * (int64_t)d, *b = x + j * (int64_t)d;
    double s = 0.0;
    for (int32_t k = 0; k < d; ++k) {
        double t = a[k] - b[k];
        double t2 = t * t;
        s = s + t2;
    }
    return s;
}

/* K comparison: returns 1 iff (w1,a1,b1) < (w2,a2,b2) lexicographically. */
static int key_less(double w1, int32_t a1, int32_t b1, double w2, int32_t a2, int32_t b2)
{
    if (w1 != w2) return w1 < w2;
    if (a1 != a2) return a1 < a2;
    return b1 < b2;
}

/* ------------------------------------------------------------- core distances (Sec. 2.1) */

/*
 * cd2[p] = the minpts-th smallest of { D(p,q) : q in P }, q = p included (value 0).
 * Brute force: keep the minpts smallest values seen so far in a sorted buffer.
 * Returns 0, or -1 on bad arguments (minpts < 1 or minpts > n).
 */
int wmo_core_dist2(const double *x, int64_t n, int32_t d, int32_t minpts, double *cd2)
{
    if (minpts < 1 || (int64_t)minpts > n) return -1;
    int err = 0;
#pragma omp parallel
    {
        double *best = (double *)malloc(sizeof(double) * (size_t)minpts);
        if (!best) {
#pragma omp atomic write
            err = -2;
        }
#pragma omp for schedule(dynamic, 64)
        for (int64_t p = 0; p < n; ++p) {
            if (!best) continue;
            int32_t cnt = 0;
            for (int64_t q = 0; q < n; ++q) {
                double v = (q == p) ? 0.0 : wmo_sqdist(x, d, p, q);
                if (cnt < minpts) {
                    int32_t j = cnt++;
                    while (j > 0 && best[j - 1] > v) { best[j] = best[j - 1]; --j; }
                    best[j] = v;
                } else if (v < best[minpts - 1]) {
                    int32_t j = minpts - 1;
                    while (j > 0 && best[j - 1] > v) { best[j] = best[j - 1]; --j; }
                    best[j] = v;
                }
            }
            cd2[p] = best[minpts - 1];
        }
        free(best);
    }
    return err;
}

/* The same definition for m selected query points q[0..m) only (brute force over all n). */
int wmo_core_dist2_subset(const double *x, int64_t n, int32_t d, int32_t minpts, const int64_t *q, int64_t m,
                          double *cd2)
{
    if (minpts < 1 || (int64_t)minpts > n) return -1;
    int err = 0;
#pragma omp parallel
    {
        double *best = (double *)malloc(sizeof(double) * (size_t)minpts);
        if (!best) {
#pragma omp atomic write
            err = -2;
        }
#pragma omp for schedule(dynamic, 1)
        for (int64_t t = 0; t < m; ++t) {
            if (!best) continue;
            int64_t p = q[t];
            int32_t cnt = 0;
            for (int64_t r = 0; r < n; ++r) {
                double v = (r == p) ? 0.0 : wmo_sqdist(x, d, p, r);
                if (cnt < minpts || v < best[minpts - 1]) {
                    int32_t j = cnt < minpts ? cnt++ : minpts - 1;
                    while (j > 0 && best[j - 1] > v) { best[j] = best[j - 1]; --j; }
                    best[j] = v;
                }
            }
            cd2[t] = best[minpts - 1];
        }
        free(best);
    }
    return err;
}

/* The K-minimum edge from point p to any other point (EMST weights), brute force. */
int wmo_nearest_edge(const double *x, int64_t n, int32_t d, int64_t p, int32_t *other, double *w2)
{
    double bw = INFINITY;
    int64_t bq = -1;
    for (int64_t r = 0; r < n; ++r) {
        if (r == p) continue;
        double v = wmo_sqdist(x, d, p, r);
        int32_t a = (int32_t)(p < r ? p : r), b = (int32_t)(p < r ? r : p);
        int32_t ca = (int32_t)(p < bq ? p : bq), cb = (int32_t)(p < bq ? bq : p);
        if (bq < 0 || key_less(v, a, b, bw, ca, cb)) { bw = v; bq = r; }
    }
    *other = (int32_t)bq;
    *w2 = bw;
    return bq < 0 ? -1 : 0;
}

/* --------------------------------------------------- MST of the complete graph (Sec. 2.1) */

/*
 * Prim's algorithm from vertex 0 over the complete graph on n points, edge key
 * K = (w2, min id, max id) with w2 = D(u,v) (EMST) or, when cd2 != NULL,
 * w2 = max(cd2[u], cd2[v], D(u,v)) (the mutual reachability graph G_MR).
 *
 * Output: the n-1 tree edges in the order Prim adds them, eu[i] < ev[i], ew2[i] = w2.
 * *tie_flag is set to 1 if any two keys compared anywhere had equal w2 (the K tie-break decided),
 * else 0: a "tie certificate" for the input.
 * Returns 0 on success, -1 on bad arguments, -2 on allocation failure.
 */
int wmo_prim(const double *x, int64_t n, int32_t d, const double *cd2,
             int32_t *eu, int32_t *ev, double *ew2, int32_t *tie_flag)
{
    if (n < 1 || d < 1) return -1;
    *tie_flag = 0;
    if (n == 1) return 0;
    double *kw = (double *)malloc(sizeof(double) * (size_t)n);      /* best key to tree: w2 */
    int32_t *kfrom = (int32_t *)malloc(sizeof(int32_t) * (size_t)n); /* its tree endpoint    */
    int32_t *rem = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);   /* vertices not in tree */
    int nthr = 1;
#ifdef _OPENMP
    nthr = omp_get_max_threads();
#endif
    int64_t *tbest = (int64_t *)malloc(sizeof(int64_t) * (size_t)nthr);
    int32_t *ttie = (int32_t *)calloc((size_t)nthr, sizeof(int32_t));
    if (!kw || !kfrom || !rem || !tbest || !ttie) {
        free(kw); free(kfrom); free(rem); free(tbest); free(ttie);
        return -2;
    }
    int64_t nrem = n - 1;
    for (int64_t i = 0; i < nrem; ++i) {
        rem[i] = (int32_t)(i + 1);
        kw[i + 1] = INFINITY;
        kfrom[i + 1] = -1;
    }
    int32_t last = 0; /* most recently added tree vertex */
    int64_t step = 0;
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        while (nrem > 0) {
            /* 1. relax keys of remaining vertices against the newly added vertex `last`,
             *    2. each thread finds its K-minimum remaining vertex. */
            int64_t mybest = -1;
#pragma omp for schedule(static)
            for (int64_t i = 0; i < nrem; ++i) {
                int32_t v = rem[i];
                double w = wmo_sqdist(x, d, last, v);
                if (cd2) {
                    if (cd2[last] > w) w = cd2[last];
                    if (cd2[v] > w) w = cd2[v];
                }
                int32_t a = last < v ? last : v, b = last < v ? v : last;
                if (kfrom[v] < 0) {
                    kw[v] = w; kfrom[v] = last;
                } else {
                    int32_t ca = kfrom[v] < v ? kfrom[v] : v, cb = kfrom[v] < v ? v : kfrom[v];
                    if (w == kw[v]) ttie[tid] = 1;
                    if (key_less(w, a, b, kw[v], ca, cb)) { kw[v] = w; kfrom[v] = last; }
                }
                if (mybest < 0) {
                    mybest = i;
                } else {
                    int32_t u = rem[mybest];
                    int32_t ua = kfrom[u] < u ? kfrom[u] : u, ub = kfrom[u] < u ? u : kfrom[u];
                    int32_t va = kfrom[v] < v ? kfrom[v] : v, vb = kfrom[v] < v ? v : kfrom[v];
                    if (kw[v] == kw[u]) ttie[tid] = 1;
                    if (key_less(kw[v], va, vb, kw[u], ua, ub)) mybest = i;
                }
            }
            tbest[tid] = mybest;
#pragma omp barrier
#pragma omp single
            {
                int64_t bi = -1;
                for (int t = 0; t < nthr; ++t) {
                    int64_t i = tbest[t];
                    if (i < 0) continue;
                    if (bi < 0) { bi = i; continue; }
                    int32_t u = rem[bi], v = rem[i];
                    int32_t ua = kfrom[u] < u ? kfrom[u] : u, ub = kfrom[u] < u ? u : kfrom[u];
                    int32_t va = kfrom[v] < v ? kfrom[v] : v, vb = kfrom[v] < v ? v : kfrom[v];
                    if (kw[v] == kw[u]) ttie[0] = 1;
                    if (key_less(kw[v], va, vb, kw[u], ua, ub)) bi = i;
                }
                int32_t v = rem[bi];
                int32_t f = kfrom[v];
                eu[step] = f < v ? f : v;
                ev[step] = f < v ? v : f;
                ew2[step] = kw[v];
                ++step;
                rem[bi] = rem[nrem - 1];
                --nrem;
                last = v;
            }
            /* implicit barrier after single */
        }
    }
    for (int t = 0; t < nthr; ++t) *tie_flag |= ttie[t];
    free(kw); free(kfrom); free(rem); free(tbest); free(ttie);
    return 0;
}

/* Sort m edges by K (stable order is irrelevant: K is a strict total order on distinct edges). */
typedef struct { double w; int32_t u, v; } kedge;

static int kedge_cmp(const void *pa, const void *pb)
{
    const kedge *a = (const kedge *)pa, *b = (const kedge *)pb;
    if (key_less(a->w, a->u, a->v, b->w, b->u, b->v)) return -1;
    if (key_less(b->w, b->u, b->v, a->w, a->u, a->v)) return 1;
    return 0;
}

int wmo_sort_edges(int64_t m, int32_t *eu, int32_t *ev, double *ew2)
{
    kedge *e = (kedge *)malloc(sizeof(kedge) * (size_t)(m > 0 ? m : 1));
    if (!e) return -2;
    for (int64_t i = 0; i < m; ++i) {
        int32_t a = eu[i] < ev[i] ? eu[i] : ev[i], b = eu[i] < ev[i] ? ev[i] : eu[i];
        e[i].w = ew2[i]; e[i].u = a; e[i].v = b;
    }
    qsort(e, (size_t)m, sizeof(kedge), kedge_cmp);
    for (int64_t i = 0; i < m; ++i) { eu[i] = e[i].u; ev[i] = e[i].v; ew2[i] = e[i].w; }
    free(e);
    return 0;
}

/* Neumaier-compensated sum of sqrt(w2) over the edges in the given order. */
double wmo_total_weight(int64_t m, const double *ew2)
{
    double s = 0.0, c = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        double v = sqrt(ew2[i]);
        double t = s + v;
        if (fabs(s) >= fabs(v)) c += (s - t) + v; else c += (v - t) + s;
        s = t;
    }
    return s + c;
}

/* ------------------------------------------------------------ tree helpers (adjacency) */

typedef struct { int32_t *off, *nbr, *eid; } adj_t;

static int build_adj(int64_t n, int64_t m, const int32_t *eu, const int32_t *ev, adj_t *g)
{
    g->off = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    g->nbr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * m + 1));
    g->eid = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * m + 1));
    int32_t *fill = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    if (!g->off || !g->nbr || !g->eid || !fill) { free(fill); return -2; }
    for (int64_t i = 0; i < m; ++i) { g->off[eu[i] + 1]++; g->off[ev[i] + 1]++; }
    for (int64_t i = 0; i < n; ++i) g->off[i + 1] += g->off[i];
    for (int64_t i = 0; i < m; ++i) {
        int32_t a = eu[i], b = ev[i];
        g->nbr[g->off[a] + fill[a]] = b; g->eid[g->off[a] + fill[a]] = (int32_t)i; fill[a]++;
        g->nbr[g->off[b] + fill[b]] = a; g->eid[g->off[b] + fill[b]] = (int32_t)i; fill[b]++;
    }
    free(fill);
    return 0;
}

static void free_adj(adj_t *g) { free(g->off); free(g->nbr); free(g->eid); }

/* Unweighted hop distance from s over the tree edges (breadth-first search). */
int wmo_hop_distance(int64_t n, const int32_t *eu, const int32_t *ev, int32_t s, int32_t *hop)
{
    if (n < 1 || s < 0 || s >= n) return -1;
    adj_t g;
    if (build_adj(n, n - 1, eu, ev, &g)) { free_adj(&g); return -2; }
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!queue) { free_adj(&g); return -2; }
    for (int64_t i = 0; i < n; ++i) hop[i] = -1;
    int64_t qh = 0, qt = 0;
    queue[qt++] = s; hop[s] = 0;
    while (qh < qt) {
        int32_t u = queue[qh++];
        for (int32_t k = g.off[u]; k < g.off[u + 1]; ++k) {
            int32_t v = g.nbr[k];
            if (hop[v] < 0) { hop[v] = hop[u] + 1; queue[qt++] = v; }
        }
    }
    free(queue); free_adj(&g);
    return qt == n ? 0 : -3; /* -3: the edges do not span a tree */
}

/* ---------------------------------------------------------- dendrogram (Sec. 4, 4.1-4.2) */

static int32_t uf_find(int32_t *par, int32_t x)
{
    while (par[x] != x) { par[x] = par[par[x]]; x = par[x]; }
    return x;
}

/*
 * Ordered dendrogram from the n-1 tree edges given in K order (eu, ev, ew2).
 * Merge i (edge i) creates node n+i; leaves are 0..n-1.  Children are the current clusters of
 * the two endpoints; the cluster holding the endpoint with the smaller hop distance from s is
 * the left child.  height = sqrt(w2), size = number of leaves below.
 * Returns 0, -1 bad args, -2 alloc, -3 edges are not a spanning tree / not in K order.
 */
int wmo_dendrogram(int64_t n, const int32_t *eu, const int32_t *ev, const double *ew2, int32_t s,
                   int32_t *left, int32_t *right, double *height, int32_t *size)
{
    if (n < 1 || s < 0 || s >= n) return -1;
    if (n == 1) return 0;
    for (int64_t i = 1; i < n - 1; ++i)
        if (key_less(ew2[i], eu[i], ev[i], ew2[i - 1], eu[i - 1], ev[i - 1])) return -3;
    int32_t *hop = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *par = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *node = (int32_t *)malloc(sizeof(int32_t) * (size_t)n); /* root -> dendrogram node */
    int32_t *sz = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * n));
    if (!hop || !par || !node || !sz) { free(hop); free(par); free(node); free(sz); return -2; }
    int rc = wmo_hop_distance(n, eu, ev, s, hop);
    if (rc) { free(hop); free(par); free(node); free(sz); return rc; }
    for (int64_t i = 0; i < n; ++i) { par[i] = (int32_t)i; node[i] = (int32_t)i; sz[i] = 1; }
    for (int64_t i = 0; i < n - 1; ++i) {
        int32_t u = eu[i], v = ev[i];
        if (hop[u] > hop[v]) { int32_t t = u; u = v; v = t; } /* u nearer s */
        int32_t ru = uf_find(par, u), rv = uf_find(par, v);
        if (ru == rv) { free(hop); free(par); free(node); free(sz); return -3; }
        int32_t id = (int32_t)(n + i);
        left[i] = node[ru];
        right[i] = node[rv];
        height[i] = sqrt(ew2[i]);
        sz[id] = sz[node[ru]] + sz[node[rv]];
        size[i] = sz[id];
        par[rv] = ru;
        node[ru] = id;
    }
    free(hop); free(par); free(node); free(sz);
    return 0;
}

/* In-order sequence of the leaves of a dendrogram (left subtree, then right subtree). */
int wmo_inorder_leaves(int64_t n, const int32_t *left, const int32_t *right, int32_t *out)
{
    if (n < 1) return -1;
    if (n == 1) { out[0] = 0; return 0; }
    int32_t *stack = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * n));
    if (!stack) return -2;
    int64_t sp = 0, k = 0;
    stack[sp++] = (int32_t)(2 * n - 2); /* root = last merge */
    while (sp > 0) {
        int32_t x = stack[--sp];
        if (x < n) { out[k++] = x; continue; }
        stack[sp++] = right[x - n]; /* pushed first, visited second */
        stack[sp++] = left[x - n];
    }
    free(stack);
    return k == n ? 0 : -3;
}

/* ------------------------------------------------------- reachability plot (Sec. 2.1) */

/* binary min-heap of (w2, a, b, vertex) keyed by K(w2, a, b) */
typedef struct { double w; int32_t a, b, v; } hent;

static int hless(const hent *x, const hent *y) { return key_less(x->w, x->a, x->b, y->w, y->a, y->b); }

static void hpush(hent *h, int64_t *hn, hent e)
{
    int64_t i = (*hn)++;
    h[i] = e;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (!hless(&h[i], &h[p])) break;
        hent t = h[i]; h[i] = h[p]; h[p] = t; i = p;
    }
}

static hent hpop(hent *h, int64_t *hn)
{
    hent top = h[0];
    h[0] = h[--(*hn)];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, m = i;
        if (l < *hn && hless(&h[l], &h[m])) m = l;
        if (r < *hn && hless(&h[r], &h[m])) m = r;
        if (m == i) break;
        hent t = h[i]; h[i] = h[m]; h[m] = t; i = m;
    }
    return top;
}

/*
 * Prim's algorithm on the tree edges from s, each step taking the K-minimum edge leaving the
 * visited set.  order[i] = the i-th visited vertex; reach[i] = sqrt(w2) of the edge that reached
 * it, reach[0] = +infinity.
 */
int wmo_reachability(int64_t n, const int32_t *eu, const int32_t *ev, const double *ew2, int32_t s,
                     int32_t *order, double *reach)
{
    if (n < 1 || s < 0 || s >= n) return -1;
    adj_t g;
    if (build_adj(n, n - 1, eu, ev, &g)) { free_adj(&g); return -2; }
    char *vis = (char *)calloc((size_t)n, 1);
    hent *h = (hent *)malloc(sizeof(hent) * (size_t)(2 * n));
    if (!vis || !h) { free(vis); free(h); free_adj(&g); return -2; }
    int64_t hn = 0, k = 0;
    order[k] = s; reach[k] = INFINITY; ++k; vis[s] = 1;
    int32_t cur = s;
    for (;;) {
        for (int32_t j = g.off[cur]; j < g.off[cur + 1]; ++j) {
            int32_t v = g.nbr[j], e = g.eid[j];
            if (vis[v]) continue;
            hent x; x.w = ew2[e]; x.a = eu[e] < ev[e] ? eu[e] : ev[e]; x.b = eu[e] < ev[e] ? ev[e] : eu[e]; x.v = v;
            hpush(h, &hn, x);
        }
        int found = 0;
        while (hn > 0) {
            hent t = hpop(h, &hn);
            if (vis[t.v]) continue;
            vis[t.v] = 1; order[k] = t.v; reach[k] = sqrt(t.w); ++k; cur = t.v; found = 1;
            break;
        }
        if (!found) break;
    }
    free(vis); free(h); free_adj(&g);
    return k == n ? 0 : -3;
}

/* ==================================================================================
 * Exact solvers for sizes where the O(n^2) definitions above are too slow.  They compute the
 * same things (the K-minimum spanning tree of the complete graph, the core distances) by other
 * algorithms over a k-d tree in FP64, pruning only with bounds that can never exceed the value
 * they bound, and are pinned against the brute-force functions above in tests/test_oracle.py.
 * ================================================================================== */

typedef struct {
    int32_t lo, hi;       /* points perm[lo..hi) */
    int32_t left, right;  /* children, -1 for a leaf (leaves hold at most 8 points) */
} kdnode_t;

typedef struct {
    int64_t n;
    int32_t d, nn;
    const double *x;
    int32_t *perm;
    kdnode_t *node;
    double *blo, *bhi;    /* bounding box of node t: blo[t*d + k], bhi[t*d + k] */
} kdtree_t;

/* the points of perm[lo..hi) with coordinate k of rank < mid first (quickselect) */
static void kd_select(const double *x, int32_t d, int32_t *perm, int32_t lo, int32_t hi, int32_t mid, int32_t k)
{
    while (hi - lo > 1) {
        double piv = x[(int64_t)perm[lo + (hi - lo) / 2] * d + k];
        int32_t i = lo, j = hi - 1;
        while (i <= j) {
            while (x[(int64_t)perm[i] * d + k] < piv) ++i;
            while (x[(int64_t)perm[j] * d + k] > piv) --j;
            if (i <= j) {
                int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
                ++i; --j;
            }
        }
        if (mid <= j) hi = j + 1;
        else if (mid >= i) lo = i;
        else return;
    }
}

static int32_t kd_build_rec(kdtree_t *t, int32_t lo, int32_t hi)
{
    const int32_t d = t->d, me = t->nn++;
    double *blo = t->blo + (int64_t)me * d, *bhi = t->bhi + (int64_t)me * d;
    for (int32_t k = 0; k < d; ++k) { blo[k] = INFINITY; bhi[k] = -INFINITY; }
    for (int32_t i = lo; i < hi; ++i) {
        const double *p = t->x + (int64_t)t->perm[i] * d;
        for (int32_t k = 0; k < d; ++k) {
            if (p[k] < blo[k]) blo[k] = p[k];
            if (p[k] > bhi[k]) bhi[k] = p[k];
        }
    }
    t->node[me].lo = lo; t->node[me].hi = hi; t->node[me].left = -1; t->node[me].right = -1;
    if (hi - lo <= 8) return me;
    int32_t kw = 0;
    for (int32_t k = 1; k < d; ++k)
        if (bhi[k] - blo[k] > bhi[kw] - blo[kw]) kw = k;
    const int32_t mid = lo + (hi - lo) / 2;
    kd_select(t->x, d, t->perm, lo, hi, mid, kw);
    const int32_t l = kd_build_rec(t, lo, mid);
    const int32_t r = kd_build_rec(t, mid, hi);
    t->node[me].left = l; t->node[me].right = r;
    return me;
}

static int kd_build(kdtree_t *t, const double *x, int64_t n, int32_t d)
{
    t->n = n; t->d = d; t->x = x; t->nn = 0;
    const int64_t cap = 2 * (n / 4 + 2) + 8;   /* leaves hold >= 4 points except small inputs */
    t->perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    t->node = (kdnode_t *)malloc(sizeof(kdnode_t) * (size_t)(cap + 2 * n / 4 + 8));
    t->blo = (double *)malloc(sizeof(double) * (size_t)d * (size_t)(cap + 2 * n / 4 + 8));
    t->bhi = (double *)malloc(sizeof(double) * (size_t)d * (size_t)(cap + 2 * n / 4 + 8));
    if (!t->perm || !t->node || !t->blo || !t->bhi) return -2;
    for (int64_t i = 0; i < n; ++i) t->perm[i] = (int32_t)i;
    if (n > 0) kd_build_rec(t, 0, (int32_t)n);
    return 0;
}

static void kd_free(kdtree_t *t) { free(t->perm); free(t->node); free(t->blo); free(t->bhi); }

/* Capacity (node ids) of the per-thread search stacks of the two k-d tree solvers below.  A
 * median-split tree of n < 2^31 points is at most 32 levels deep and a search holds at most two
 * entries per level, so 256 is never reached; a search that would exceed it fails with -3 instead
 * of dropping nodes.  wmo_set_kd_stack_cap lowers it so that tests can reach that path. */
static int32_t g_kd_stack_cap = 256;

int wmo_set_kd_stack_cap(int32_t cap)
{
    if (cap < 2 || cap > 256) return -1;
    g_kd_stack_cap = cap;
    return 0;
}

/* Lower bound of D(p, q) over every q in the box of node t.  Each gap is rounded from an exact
 * difference at least as large as the box's (rounding is monotone), squared and summed in the
 * order of wmo_sqdist, so the bound never exceeds the FP64 distance of any point inside. */
static double kd_box_lb(const kdtree_t *t, int32_t nd, const double *p)
{
    const double *lo = t->blo + (int64_t)nd * t->d, *hi = t->bhi + (int64_t)nd * t->d;
    double s = 0.0;
    for (int32_t k = 0; k < t->d; ++k) {
        double g = 0.0;
        if (p[k] < lo[k]) g = lo[k] - p[k];
        else if (p[k] > hi[k]) g = p[k] - hi[k];
        double g2 = g * g;
        s = s + g2;
    }
    return s;
}

/*
 * cd2[p] = the minpts-th smallest D(p,q), q = p included: the value wmo_core_dist2 computes, found
 * by a nearest-first search that skips a box only when its lower bound is not below the current
 * minpts-th smallest value.  Returns 0, -1 on bad arguments, -2 on allocation failure, -3 when a
 * search stack would overflow (the values are then not valid).
 */
int wmo_core_dist2_kdtree(const double *x, int64_t n, int32_t d, int32_t minpts, double *cd2)
{
    if (minpts < 1 || (int64_t)minpts > n || n > 0x7fffffff) return -1;
    kdtree_t t;
    if (kd_build(&t, x, n, d)) { kd_free(&t); return -2; }
    int err = 0;
#pragma omp parallel
    {
        double *heap = (double *)malloc(sizeof(double) * (size_t)minpts);   /* max-heap of the best */
        int32_t *stk = (int32_t *)malloc(sizeof(int32_t) * 256);
        if (!heap || !stk) {
#pragma omp atomic write
            err = -2;
        }
#pragma omp for schedule(dynamic, 256)
        for (int64_t p = 0; p < n; ++p) {
            if (!heap || !stk) continue;
            const double *xp = x + p * d;
            int32_t hn = 0, sp = 0;
            stk[sp++] = 0;
            while (sp > 0) {
                const int32_t nd = stk[--sp];
                if (hn == minpts && kd_box_lb(&t, nd, xp) >= heap[0]) continue;
                const kdnode_t *N = &t.node[nd];
                if (N->left < 0) {
                    for (int32_t i = N->lo; i < N->hi; ++i) {
                        const double w = wmo_sqdist(x, d, p, t.perm[i]);
                        if (hn < minpts) {              /* sift up */
                            int32_t c = hn++;
                            while (c > 0 && heap[(c - 1) / 2] < w) { heap[c] = heap[(c - 1) / 2]; c = (c - 1) / 2; }
                            heap[c] = w;
                        } else if (w < heap[0]) {       /* replace the maximum, sift down */
                            int32_t c = 0;
                            for (;;) {
                                int32_t l = 2 * c + 1, r = l + 1, m = c;
                                double vm = w;
                                if (l < hn && heap[l] > vm) { m = l; vm = heap[l]; }
                                if (r < hn && heap[r] > vm) { m = r; vm = heap[r]; }
                                if (m == c) break;
                                heap[c] = heap[m];
                                c = m;
                            }
                            heap[c] = w;
                        }
                    }
                } else if (sp + 2 <= g_kd_stack_cap) {
                    const double l0 = kd_box_lb(&t, N->left, xp), l1 = kd_box_lb(&t, N->right, xp);
                    stk[sp++] = l0 <= l1 ? N->right : N->left;   /* nearer child on top */
                    stk[sp++] = l0 <= l1 ? N->left : N->right;
                } else {
#pragma omp atomic write
                    err = -3;   /* the search would drop a subtree: fail instead */
                    break;
                }
            }
            cd2[p] = heap[0];
        }
        free(heap);
        free(stk);
    }
    kd_free(&t);
    return err;
}

/*
 * The K-minimum spanning tree of the complete graph (EMST, or G_MR when cd2 != NULL) by Boruvka's
 * algorithm: every round, each point finds its K-minimum edge to a point of another component
 * (a search over the tree that skips boxes whose points all lie in its component and boxes whose
 * lower bound exceeds the best w2 so far), each component keeps the K-minimum of its points', and
 * those edges are added (K is a strict total order, so they form a forest; each is the K-minimum
 * edge across its component's cut, so it is in the tree).  Output in K order, eu < ev.
 * Returns 0, -1 on bad arguments, -2 on allocation failure, -3 when a search stack would overflow,
 * -4 when a round adds no edge.
 */
static int32_t bv_find(int32_t *par, int32_t x)
{
    while (par[x] != x) { par[x] = par[par[x]]; x = par[x]; }
    return x;
}

int wmo_boruvka(const double *x, int64_t n, int32_t d, const double *cd2, int32_t *eu, int32_t *ev, double *ew2)
{
    if (n < 1 || n > 0x7fffffff) return -1;
    if (n == 1) return 0;
    kdtree_t t;
    if (kd_build(&t, x, n, d)) { kd_free(&t); return -2; }
    int32_t *par = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *comp = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *ncomp = (int32_t *)malloc(sizeof(int32_t) * (size_t)t.nn);
    double *ncd = (double *)malloc(sizeof(double) * (size_t)t.nn);
    double *bw = (double *)malloc(sizeof(double) * (size_t)n);     /* per point: best edge */
    int32_t *bq = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    double *cw = (double *)malloc(sizeof(double) * (size_t)n);     /* per component root */
    int32_t *ca = (int32_t *)malloc(sizeof(int32_t) * (size_t)n), *cb = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!par || !comp || !ncomp || !ncd || !bw || !bq || !cw || !ca || !cb) {
        free(par); free(comp); free(ncomp); free(ncd); free(bw); free(bq); free(cw); free(ca); free(cb);
        kd_free(&t);
        return -2;
    }
    for (int64_t i = 0; i < n; ++i) par[i] = (int32_t)i;
    /* node minimum core distance (children have larger ids than their parent) */
    for (int32_t nd = t.nn - 1; nd >= 0; --nd) {
        const kdnode_t *N = &t.node[nd];
        if (!cd2) { ncd[nd] = 0.0; continue; }
        if (N->left < 0) {
            double m = INFINITY;
            for (int32_t i = N->lo; i < N->hi; ++i) if (cd2[t.perm[i]] < m) m = cd2[t.perm[i]];
            ncd[nd] = m;
        } else {
            ncd[nd] = ncd[N->left] < ncd[N->right] ? ncd[N->left] : ncd[N->right];
        }
    }
    int64_t m = 0;
    int err = 0;
    while (m < n - 1 && !err) {
        for (int64_t i = 0; i < n; ++i) comp[i] = bv_find(par, (int32_t)i);
        for (int32_t nd = t.nn - 1; nd >= 0; --nd) {
            const kdnode_t *N = &t.node[nd];
            if (N->left < 0) {
                int32_t c = comp[t.perm[N->lo]];
                for (int32_t i = N->lo + 1; i < N->hi && c >= 0; ++i) if (comp[t.perm[i]] != c) c = -1;
                ncomp[nd] = c;
            } else {
                ncomp[nd] = (ncomp[N->left] >= 0 && ncomp[N->left] == ncomp[N->right]) ? ncomp[N->left] : -1;
            }
        }
#pragma omp parallel
        {
            int32_t *stk = (int32_t *)malloc(sizeof(int32_t) * 256);
            if (!stk) {
#pragma omp atomic write
                err = -2;
            }
#pragma omp for schedule(dynamic, 256)
            for (int64_t p = 0; p < n; ++p) {
                double best = INFINITY;
                int32_t bestq = -1;
                if (!stk) { bw[p] = best; bq[p] = bestq; continue; }
                const double *xp = x + p * d;
                const int32_t cp = comp[p];
                const double cdp = cd2 ? cd2[p] : 0.0;
                int32_t sp = 0;
                stk[sp++] = 0;
                while (sp > 0) {
                    const int32_t nd = stk[--sp];
                    if (ncomp[nd] == cp) continue;
                    double lb = kd_box_lb(&t, nd, xp);
                    if (cd2) {
                        if (cdp > lb) lb = cdp;
                        if (ncd[nd] > lb) lb = ncd[nd];
                    }
                    if (lb > best) continue;
                    const kdnode_t *N = &t.node[nd];
                    if (N->left < 0) {
                        for (int32_t i = N->lo; i < N->hi; ++i) {
                            const int32_t q = t.perm[i];
                            if (comp[q] == cp) continue;
                            double w = wmo_sqdist(x, d, p, q);
                            if (cd2) {
                                if (cdp > w) w = cdp;
                                if (cd2[q] > w) w = cd2[q];
                            }
                            const int32_t a = (int32_t)p < q ? (int32_t)p : q, b = (int32_t)p < q ? q : (int32_t)p;
                            if (bestq < 0 ||
                                key_less(w, a, b, best, (int32_t)p < bestq ? (int32_t)p : bestq,
                                         (int32_t)p < bestq ? bestq : (int32_t)p)) {
                                best = w;
                                bestq = q;
                            }
                        }
                    } else if (sp + 2 <= g_kd_stack_cap) {
                        const double l0 = kd_box_lb(&t, N->left, xp), l1 = kd_box_lb(&t, N->right, xp);
                        stk[sp++] = l0 <= l1 ? N->right : N->left;
                        stk[sp++] = l0 <= l1 ? N->left : N->right;
                    } else {
#pragma omp atomic write
                        err = -3;   /* deeper than a balanced tree can be */
                        break;
                    }
                }
                bw[p] = best;
                bq[p] = bestq;
            }
            free(stk);
        }
        if (err) break;
        for (int64_t i = 0; i < n; ++i) { cw[i] = INFINITY; ca[i] = -1; cb[i] = -1; }
        for (int64_t p = 0; p < n; ++p) {
            if (bq[p] < 0) continue;
            const int32_t c = comp[p];
            const int32_t a = (int32_t)p < bq[p] ? (int32_t)p : bq[p], b = (int32_t)p < bq[p] ? bq[p] : (int32_t)p;
            if (ca[c] < 0 || key_less(bw[p], a, b, cw[c], ca[c], cb[c])) { cw[c] = bw[p]; ca[c] = a; cb[c] = b; }
        }
        int64_t added = 0;
        for (int64_t c = 0; c < n; ++c) {
            if (ca[c] < 0) continue;
            const int32_t ra = bv_find(par, ca[c]), rb = bv_find(par, cb[c]);
            if (ra == rb) continue;   /* the other component chose the same edge */
            par[ra] = rb;
            eu[m] = ca[c]; ev[m] = cb[c]; ew2[m] = cw[c];
            ++m;
            ++added;
        }
        if (added == 0) { err = -4; break; }
    }
    free(par); free(comp); free(ncomp); free(ncd); free(bw); free(bq); free(cw); free(ca); free(cb);
    kd_free(&t);
    if (err) return err;
    return wmo_sort_edges(m, eu, ev, ew2);
}
