/*
 * wspdmst.h -- C ABI of the GB300 EMST / HDBSCAN* library (libwspdmst.so).
 *
 * The library computes, on one CUDA GPU (sm_103a), the problems stated in Sec. 2.1 of
 * Wang, Yu, Gu, Shun, "Fast Parallel Algorithms for Euclidean Minimum Spanning Tree and
 * Hierarchical Spatial Clustering" (SIGMOD'21):
 *   - EMST: a minimum spanning tree of the complete Euclidean graph of n points in d dimensions;
 *   - HDBSCAN*: the MST of the mutual reachability graph G_MR (core distance = distance to the
 *     minPts-th nearest neighbour counting the point itself, d_m(p,q) = max{cd(p), cd(q), d(p,q)}),
 *     its ordered dendrogram for a start point s and the reachability plot from s (Sec. 4).
 * Both follow the method of Sec. 3: a spatial-median k-d tree, the well-separated pair
 * decomposition traversed lazily by MemoGFK rounds (Algorithm 3) with batched BCCP / BCCP*
 * computations, and batched Kruskal over a union-find shared across rounds; the dendrogram and
 * plot come from a top-down heavy/light construction after Sec. 4.2 (the heavy set of a
 * subproblem is the upper half of its rank interval, light components come from a union-find,
 * and the output equals the sequential definition exactly).
 *
 * Canonical result.  Every edge comparison uses the strict total key
 *     K(u,v) = (w2, min(u,v), max(u,v))   (lexicographic),
 * where w2 is the squared weight evaluated in IEEE FP64 as sum_{k=0}^{d-1} (x_k(u)-x_k(v))^2 in
 * dimension order with one rounding per subtract, multiply and add (no fused multiply-add); for
 * HDBSCAN* w2 = max(cd2(u), cd2(v), that value).  The returned tree is the unique MST under K,
 * listed in increasing K order (Kruskal order), each edge with u < v and w = sqrt(w2).
 * (HDBSCAN*: this holds for inputs in general position, i.e. all pairwise FP64 squared
 * distances distinct; otherwise the tree returned is still an MST of G_MR.)
 *
 * Ids.  Point ids are input row indices 0..n-1.  Dendrogram node n+i is the i-th merge in K
 * order; leaves are the ids 0..n-1 (scipy-linkage-like numbering).
 *
 * Pointers.  Every input and output pointer may be host memory or device memory of the
 * current CUDA device; the library detects which with cudaPointerGetAttributes.  Outputs are
 * caller-owned and must be sized as stated.  Device work is issued on opts->stream; every call
 * returns only after its outputs are complete (it synchronises that stream).
 *
 * Errors.  Every call returns WM_OK (0) or a negative code; wm_strerror() gives the text and
 * wm_last_error_detail() a message for the last failure on the calling thread.  On error the
 * output buffers hold unspecified values.  No call aborts the process.
 *
 * Thread safety.  Calls on distinct wm_opts.workspace arenas (or distinct threads using the
 * library-managed workspace of different devices) may run concurrently; calls sharing the
 * library-managed workspace of one device are serialised by an internal mutex.
 */
#ifndef WSPDMST_H
#define WSPDMST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ codes and enums */
#define WM_OK 0
#define WM_EINVAL (-1)    /* bad argument: n < 1, d not in [1,16], minPts < 1 or > n,
                              non-finite coordinate or |coordinate| > 2^60, bad enum value */
#define WM_ENOMEM (-2)    /* device memory (or the caller's workspace) exhausted */
#define WM_ETIMEOUT (-3)  /* reserved for a bounded device-side wait that gives up; no call
                              returns it in this version (the kernels never wait on one another) */
#define WM_ECUDA (-4)     /* a CUDA runtime call failed */
#define WM_EINTERNAL (-5) /* an internal consistency check failed (a bug) */

#define WM_F32 0 /* coordinates stored as float  */
#define WM_F64 1 /* coordinates stored as double */
#define WM_AOS 0 /* pts[i*d + k]: row per point              */
#define WM_SOA 1 /* pts[k*n + i]: one contiguous array per dim */

#define WM_PREC_FP32_SCREEN 0 /* FP32 distance screen, FP64 recheck of every candidate inside a
                                  rigorous error band (default) */
#define WM_PREC_FP64 1        /* the plain form: every point distance evaluated in FP64 */

/* Methods (wm_opts.method): an algorithm, optionally OR'ed with WM_SEPARATION_GEOMETRIC; all
 * compute the same tree. */
#define WM_METHOD_MEMOGFK 0   /* MemoGFK rounds (Sec. 3.2.3, Algorithm 3), the default */
#define WM_METHOD_GFK 1       /* GFK (Sec. 3.2.2, Algorithm 2): the full WSPD is materialised and each
                                 pair's BCCP computed once and kept until its round */
#define WM_METHOD_NAIVE 2     /* EMST-Naive (Sec. 5): the BCCP of every pair of the full WSPD, then
                                 one Kruskal over all of them */
#define WM_SEPARATION_GEOMETRIC 0x100   /* HDBSCAN*: pairs are well-separated by geometry alone,
                                 without the mutual-unreachability disjunction of Sec. 3.1.2 */
#define WM_METHOD_GANTAO (WM_METHOD_MEMOGFK | WM_SEPARATION_GEOMETRIC)
                              /* HDBSCAN*: the baseline of Sec. 3.1.1 (standard WSPD, BCCP*, MemoGFK
                                 rounds); for EMST the same as WM_METHOD_MEMOGFK */

/* ------------------------------------------------------------------------- records */

/* One tree edge: endpoints (u < v) and weight w (Euclidean or mutual-reachability distance,
 * not squared).  16 bytes. */
typedef struct {
    int32_t u, v;
    double w;
} wm_edge;

/* One dendrogram merge (internal node n+i).  left/right are node ids (leaf = point id);
 * height = weight of the merging edge; size = number of points below.  24 bytes. */
typedef struct {
    int32_t left, right;
    double height;
    int32_t size;
    int32_t reserved;
} wm_dnode;

/* Per-call statistics (optional output). */
typedef struct {
    double ms_total;      /* wall time of the call, host clock                      */
    double ms_ingest;     /* device phase times (CUDA events on the call's stream)  */
    double ms_build_tree;
    double ms_core_dist;
    double ms_wspd;       /* GetRho + GetPairs traversals (including inline BCCP)   */
    double ms_bccp;       /* BCCP flushes (all size classes and their readbacks)    */
    double ms_kruskal;    /* batched Kruskal of every round + final sort of the tree */
    double ms_dendrogram;
    int64_t rounds;       /* MemoGFK rounds                                         */
    int64_t pairs_retrieved;   /* well-separated pairs whose BCCP was evaluated     */
    int64_t bccp_evals;        /* point-pair distance evaluations in BCCP / BCCP*   */
    int64_t bccp_tile_evals;   /* of which in the tile kernel                        */
    int64_t knn_evals;         /* point-pair distance evaluations in the k-NN pass   */
    int64_t fp64_rechecks;     /* FP64 re-evaluations of screened candidates         */
    int64_t candidate_edges;   /* edges handed to Kruskal over all rounds            */
    int64_t tree_nodes;
    int64_t tree_depth;
    size_t workspace_bytes_used;   /* peak workspace use of this call               */
    double max_rel_screen_err;     /* largest |fp32 - fp64| / fp64 between a screened FP32
                                      value and its exact FP64 value, over every BCCP
                                      candidate re-evaluated in FP64 (every winner among
                                      them) and every core distance; 0 in the FP64 form.
                                      A priori bound: 2^-19 for FP32-exact coordinates  */
    int32_t tie_overflow;          /* HDBSCAN*: 1 when the pairs within some point's core
                                      distance (the tie-repair edges) exceeded their
                                      buffer, which takes inputs far from general position
                                      (many exact duplicates).  The call still returns
                                      WM_OK with an MST of G_MR, but that tree may differ
                                      from the K-minimum one; 0 otherwise             */
    int32_t edge_batch_grown;      /* 1 when a round's candidate edges outgrew the first
                                      part of the batch and the call, its work so far
                                      mostly traversal, grew the batch to the tuned
                                      capacity (wm_tuning.edges_per_point) instead of
                                      lowering rho_hi                                  */
    double ms_knn_kernel;          /* CUDA-event time of the k-NN kernel (one launch)   */
    double ms_tile_kernel;         /* CUDA-event time of the tile BCCP kernel (medium and
                                      big pairs), summed over the flushes               */
    int64_t tile_launches;         /* BCCP flushes that launched the big-pair kernels   */
    double ms_getpairs;            /* CUDA-event time summed over GetPairs step launches  */
    int64_t getpairs_launches;     /* number of GetPairs step launches                  */
    int64_t getpairs_visits;       /* node pairs examined by the GetPairs traversals     */
    int64_t getrho_visits;         /* node pairs examined by the GetRho traversals       */
    int64_t bccp_dual_evals;       /* distance evaluations in the pruned dual-tree BCCP */
    int64_t rho_shrinks;           /* times a round lowered rho_hi to fit its edge batch  */
    int64_t max_pending_pairs;     /* peak node pairs pending in a WSPD traversal         */
    int64_t bccp_pairs_below;      /* retrieved pairs whose BCCP lay below the round's
                                      range (found in an earlier round)                   */
    int64_t bccp_pairs_above;      /* retrieved pairs whose BCCP lay at or above the
                                      round's range (found again in a later round)        */
    int64_t bccp_evals_outside;    /* distance evaluations spent on those pairs (group
                                      and tile kernels)                                   */
    int64_t bccp_tile_evals_skipped; /* point pairs of the tile kernel whose evaluation a
                                        chunk's bounding box ruled out                   */
    double ms_getrho;              /* CUDA-event time of the GetRho traversals           */
    double ms_bccp_group;          /* ... of the group BCCP kernels (tiny, small pairs)  */
    double ms_bccp_dual;           /* ... of the dual-tree BCCP kernel (huge pairs)      */
    int64_t wspd_pairs;            /* GFK / EMST-Naive: pairs of the materialised WSPD     */
} wm_stats;

/* Options.  A zero-initialised struct (or NULL) gives the defaults. */
typedef struct {
    void *stream;           /* cudaStream_t to issue work on; NULL = legacy default stream */
    int32_t precision;      /* WM_PREC_FP32_SCREEN (0, default) or WM_PREC_FP64            */
    int32_t method;         /* WM_METHOD_* (0, default: MemoGFK)                           */
    void *workspace;        /* optional caller-owned device scratch arena; NULL = the
                               library manages a grow-only per-device cache               */
    size_t workspace_bytes; /* size of `workspace` in bytes                                */
    wm_stats *stats;        /* optional: filled on return                                  */
} wm_opts;

/* ---------------------------------------------------------------------- entry points */

/*
 * wm_emst -- Euclidean minimum spanning tree (Sec. 2.1 "EMST"; method: Sec. 3.2, Algorithm 3).
 *   pts        n points, dtype WM_F32/WM_F64, layout WM_AOS/WM_SOA (host or device)
 *   n >= 1, 1 <= d <= 16
 *   out_edges  n-1 wm_edge, K order (host or device; may be NULL when n == 1)
 *   out_total_weight  sum of the n-1 weights (host pointer; may be NULL)
 *   opts       may be NULL
 * Returns WM_OK or WM_EINVAL / WM_ENOMEM / WM_ECUDA / WM_EINTERNAL.
 */
int wm_emst(const void *pts, int64_t n, int32_t d, int32_t dtype, int32_t layout,
            wm_edge *out_edges, double *out_total_weight, const wm_opts *opts);

/*
 * wm_hdbscan -- HDBSCAN* (Sec. 2.1 "HDBSCAN*"; method: Sec. 3.1.2 with the disjunctive
 * well-separation, Algorithm 3 with BCCP*, and Sec. 4 for the ordered dendrogram).
 *   min_pts          1 <= min_pts <= n
 *   out_mst          n-1 wm_edge of the MST of G_MR, K order           (may be NULL)
 *   out_core_dist    n doubles, cd(p) (not squared); a point is noise at a cut eps when
 *                    cd(p) > eps (its self-edge, Sec. 2.1)               (may be NULL)
 *   out_dendro       n-1 wm_dnode, the ordered dendrogram of `start`     (may be NULL)
 *   out_order        n int32, the reachability-plot order (Prim order from `start`)
 *   out_reach        n doubles, bar heights; out_reach[0] = +infinity    (may be NULL)
 *   start            the start point s, 0 <= start < n
 */
int wm_hdbscan(const void *pts, int64_t n, int32_t d, int32_t dtype, int32_t layout,
               int32_t min_pts, wm_edge *out_mst, double *out_core_dist, wm_dnode *out_dendro,
               int32_t *out_order, double *out_reach, int32_t start, const wm_opts *opts);

/*
 * wm_batch -- many independent EMST / HDBSCAN* instances in one call (the problems of Sec. 2.1,
 * solved as above).  Instances with the same minPts run as one problem (in the dimension of the
 * largest, missing coordinates being 0, which adds exactly 0 to every distance): their
 * points share one k-d forest, one WSPD traversal per round, one set of BCCP kernels and one
 * Kruskal, with no pair or edge ever joining two instances; each instance's edges, core
 * distances, dendrogram, order and bars are exactly those of its own wm_emst / wm_hdbscan call
 * (bit for bit; the total weight is summed in another order).
 *   inst    count instances; every pointer in them may be host or device
 *   count   >= 1
 *   dtype, layout  as for wm_emst, for every instance
 * Per instance (wm_instance):
 *   pts, n, d         n >= 1, 1 <= d <= 15 (one coordinate is taken to separate instances)
 *   min_pts           0 or 1: EMST (out_edges, out_total_weight); 2..min(n, 256): HDBSCAN*
 *                     (out_edges = MST of G_MR, out_core_dist, out_dendro, out_order, out_reach
 *                     as for wm_hdbscan); NULL outputs are skipped
 *   start             HDBSCAN*: the start point of the dendrogram and plot, 0 <= start < n
 * Returns WM_OK, or the first error of any group (WM_EINVAL names the instance in
 * wm_last_error_detail()).  opts as for wm_emst; opts->stats sums the groups.
 */
typedef struct {
    const void *pts;
    int64_t n;
    int32_t d;
    int32_t min_pts;
    int32_t start;
    int32_t reserved;
    wm_edge *out_edges;
    double *out_total_weight;
    double *out_core_dist;
    wm_dnode *out_dendro;
    int32_t *out_order;
    double *out_reach;
} wm_instance;

int wm_batch(const wm_instance *inst, int32_t count, int32_t dtype, int32_t layout, const wm_opts *opts);

/*
 * wm_single_linkage -- ordered dendrogram and reachability plot of any weighted spanning tree
 * (Sec. 4: with the EMST as input this is single-linkage clustering).
 *   tree       n-1 wm_edge forming a spanning tree of 0..n-1 (any order; the library orders
 *              them by K using w2 = w*w as the primary key)
 *   out_dendro n-1 wm_dnode; out_order n int32; out_reach n doubles (each may be NULL)
 * Returns WM_EINVAL when the edges do not form a spanning tree.
 */
int wm_single_linkage(const wm_edge *tree, int64_t n, int32_t start, wm_dnode *out_dendro,
                      int32_t *out_order, double *out_reach, const wm_opts *opts);

/*
 * wm_emst_noalloc -- wm_emst for callers that cannot allocate.  The paper has no counterpart:
 * this entry point exists for integrating the library, not for the method.
 *
 * Some callers must not allocate device memory at the moment they need an EMST: a host
 * program (a database or inference server, say) that reserved nearly all device memory up
 * front for its own pool, where a library cudaMalloc would fail or fragment that pool; a
 * latency-critical loop that cannot afford cudaMalloc's implicit device synchronisation and
 * unbounded latency; a plugin whose host hands it buffers and forbids it to allocate.  This
 * variant computes exactly what wm_emst computes (same K-minimum tree, same order, same
 * rounding) with all of its device scratch taken from one array of WM_NOALLOC_SCRATCH_BYTES
 * bytes that the library declares statically in device memory.  It calls no cudaMalloc,
 * cudaFree, cudaMallocHost or other allocating routine and creates no CUDA events.  The caller
 * still owns the input and the outputs, which may be host or device memory as for wm_emst.
 *
 *   Limits   1 <= n <= WM_NOALLOC_MAX_POINTS, 1 <= d <= 16; a larger n returns WM_EINVAL.  When
 *            a traversal or edge-batch capacity overflows, the call doubles it and restarts, as
 *            wm_emst does; an input whose buffers then no longer fit in the array returns
 *            WM_ENOMEM with a message (wm_emst, which allocates, still handles it).
 *   Memory   the array is part of the library's device code: it is reserved on a GPU when that
 *            code is loaded there, which under CUDA's lazy module loading is the first call into
 *            the library on that GPU that launches a kernel or looks the array up (any entry
 *            point), and at library load otherwise.  It stays reserved until the process exits.
 *            A caller that reserves the rest of the device for a pool of its own should make one
 *            call first (a one-point input will do), so that the array is already in place.
 *   Set-up   the first call of this entry point on a device, with that device current, looks up
 *            the array's device address once (cudaGetSymbolAddress); make that first call before
 *            any stream capture.
 *   Sharing  all calls on a device use the same array, which keeps the last call's contents (the
 *            call initialises everything it reads).  Calls whose GPU work overlapped would race
 *            on it; within one process this entry point prevents that by holding a per-device
 *            lock for the whole call and returning only after its GPU work has completed, on
 *            every path including the error returns.
 */
#define WM_NOALLOC_MAX_POINTS 32768
#define WM_NOALLOC_SCRATCH_BYTES (64u << 20)
int wm_emst_noalloc(const void *pts, int64_t n, int32_t d, int32_t dtype, int32_t layout,
                    wm_edge *out_edges, double *out_total_weight, const wm_opts *opts);

/* ------------------------------------------------------------------------- serving */
/*
 * A server runs EMST / HDBSCAN* jobs as they arrive, several at a time on one device
 * (continuous batching; the paper's method is one job at a time).  Each of `workers` host
 * threads owns a CUDA stream; a job is admitted when its workspace estimate
 * (wm_query_footprint) fits in what is left of `hbm_budget_bytes`, its workspace comes from a
 * stream-ordered pool and returns to it when the job ends, so jobs that arrive while others run
 * start as soon as a worker and memory are free, and their kernels overlap on the device.
 * A job whose estimate exceeds the whole budget is rejected at submission (WM_ENOMEM).
 * Results are identical to running the same job alone with wm_emst / wm_hdbscan.
 */
typedef struct wm_server wm_server;

#define WM_JOB_EMST 0
#define WM_JOB_HDBSCAN 1

typedef struct {
    int32_t kind;            /* WM_JOB_EMST or WM_JOB_HDBSCAN */
    int32_t dtype, layout;   /* as wm_emst */
    int32_t d;
    int64_t n;
    const void *pts;         /* caller-owned until the job completes (host or device) */
    int32_t min_pts, start;  /* HDBSCAN* only */
    int32_t precision;       /* WM_PREC_* */
    int32_t reserved;
    /* caller-owned outputs, sized as for wm_emst / wm_hdbscan; NULL to skip */
    wm_edge *out_edges;
    double *out_total_weight;   /* EMST */
    double *out_core_dist;
    wm_dnode *out_dendro;
    int32_t *out_order;
    double *out_reach;
} wm_job;

/* status codes of a ticket */
#define WM_JOB_QUEUED 1
#define WM_JOB_RUNNING 2
#define WM_JOB_DONE 0        /* success */

int wm_server_create(int32_t device, size_t hbm_budget_bytes, int32_t workers, wm_server **out);
/* Waits for every submitted job, then stops the workers and frees the server. */
int wm_server_destroy(wm_server *s);
/* Queues a job; *ticket identifies it.  Never blocks on the device. */
int wm_submit(wm_server *s, const wm_job *job, int64_t *ticket);
/* Non-blocking: *status = WM_JOB_QUEUED / WM_JOB_RUNNING / WM_JOB_DONE or the job's negative
 * error code; *latency_ms (may be NULL) = submit-to-completion time once finished. */
int wm_poll(wm_server *s, int64_t ticket, int32_t *status, double *latency_ms);
/* Blocks until the job has finished; returns its result code. */
int wm_wait(wm_server *s, int64_t ticket, double *latency_ms);
/* Counters: jobs finished, peak admitted bytes, peak number of jobs running together. */
int wm_server_counters(wm_server *s, int64_t *finished, size_t *peak_bytes, int32_t *peak_running);

/*
 * Tuning.  Parameters that change how fast a call runs, never what it returns (every setting
 * yields the same K-minimum tree, dendrogram and plot).  A call takes them from a built-in table
 * chosen by (problem, d, n) and written by the project's autotuner (paper_2104_01126_gb300/
 * autotune.py), unless wm_set_tuning has set an override for the whole process.
 */
typedef struct {
    int32_t tight_diameters; /* 1: a node's diameter bound is the smallest of its box diagonal,
                                its largest pairwise distance (<= 32 points) and twice its
                                bounding-sphere radius; 0: the box diagonal alone           */
    int32_t chunk_log2;      /* WSPD traversal: node pairs popped per step = 2^chunk_log2;
                                0 = from n (min(2^21, max(2^12, 4n)))                        */
    int32_t dfs_budget;      /* WSPD traversal: depth-first rounds a warp runs on its own
                                stack per step (1..64)                                       */
    int32_t route_big;       /* BCCP: a flush's big pairs go to the pruned dual-tree kernel
                                when there are at most this many                              */
    int32_t medium_max;      /* BCCP: pairs with |A||B| up to this (65..4096) take one warp   */
    int32_t big_max;         /* BCCP: pairs up to this (>= medium_max) take the tile kernel;
                                larger ones the dual-tree kernel                              */
    int32_t combined;        /* 1: a round's GetRho minimum is found during its GetPairs
                                traversal (one pass); 0: a GetRho traversal first (Algorithm 3);
                                2: two passes until, after two rounds or more, the GetRho
                                traversals have visited at least half as many node pairs as
                                the GetPairs traversals; one pass afterwards                   */
    int32_t getrho_sample;   /* GetRho starts from every getrho_sample-th frontier pair (0 or 1:
                                all of them, Algorithm 3); its minimum is then an upper bound of
                                the exact one, a larger rho_hi with fewer GetRho visits         */
    int32_t edges_per_point; /* capacity of a round's candidate-edge batch: this many edges per
                                point (+ 2^20); 0 = 4.  A round whose edges would overflow it
                                lowers its rho_hi, and the dropped edges are found again in a
                                later round; a larger batch costs 48 bytes of workspace per
                                edge (0..64)                                                  */
    int32_t range_ratio;     /* MemoGFK: a round's rho_hi is at most range_ratio x its rho_lo
                                (once rho_lo > 0); 0 = no limit (GetRho's bound, Algorithm 3).
                                A smaller range means fewer retrieved pairs whose BCCP lies
                                above what the round's edge batch can hold, and more rounds
                                (0 or 2..2^20)                                                */
    int32_t range_gate;      /* with range_ratio: 0 = the limit applies in every round; else
                                only in rounds where the call's node-pair visits so far are
                                below range_gate x its BCCP distance evaluations (0..2^20)   */
    int32_t reserved[5];
} wm_tuning;

/* The parameters a call with these sizes uses (min_pts = 0 for EMST); n = 0 gives the built-in
 * defaults (the values before any table row or override). */
int wm_get_tuning(int64_t n, int32_t d, int32_t min_pts, wm_tuning *out);
/* Overrides the table for every later call of the process (NULL restores it).  WM_EINVAL for
 * out-of-range values.  Not for use while other threads are inside library calls. */
int wm_set_tuning(const wm_tuning *t);

/*
 * wm_query_footprint -- an upper estimate of the device workspace, in bytes, that a call with
 * these sizes needs (min_pts = 0 for EMST).  Data-dependent buffers (WSPD traversal frontiers,
 * candidate edges) are estimated; a call whose data needs more returns WM_ENOMEM when a
 * caller arena is used, and grows its cache otherwise.
 */
int wm_query_footprint(int64_t n, int32_t d, int32_t min_pts, size_t *bytes);

/* Frees the library-managed workspace cache of the current device. */
int wm_release_cache(void);

/* Text for an error code. */
const char *wm_strerror(int code);

/* Message describing the last failure on the calling thread ("" if none). */
const char *wm_last_error_detail(void);

/* Number of CUDA kernels this library has launched in this process (all devices, all
 * threads) -- a diagnostic counter for benchmarks.  Touches no device. */
int64_t wm_kernel_launch_count(void);

/* Measured FP32 throughput of the current device, in TFLOP/s (a diagnostic for benchmarks, the
 * denominator of the BCCP and k-NN roofline): a kernel of independent fused multiply-add chains
 * filling every SM, timed with CUDA events, best of five runs after a warm-up; *ms (may be NULL)
 * is that run's time.  Allocates and frees a few bytes of device memory. */
int wm_fp32_fma_peak(double *tflops, double *ms);

/* Library version string. */
const char *wm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* WSPDMST_H */
