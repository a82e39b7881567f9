// wspd.cuh -- arguments of the WSPD traversal and BCCP kernels (see wspd.cu).
#pragma once

#include "wm_internal.cuh"

namespace wm {

struct TravArgs {
    int N = 0, n = 0, d = 0;
    const float *lo = nullptr, *hi = nullptr, *diam2 = nullptr;
    const int *begin = nullptr, *end = nullptr, *left = nullptr, *right = nullptr;
    const int *comp = nullptr;
    const float *cdmin = nullptr, *cdmax = nullptr;   // HDBSCAN* node bounds (null for EMST)
    const float *x32 = nullptr;
    const float4 *x4 = nullptr;        // the FP32 copy point-major: dp / 4 float4s per point, padded
                                       // coordinates 0 (the group BCCP kernel reads whole points)
    const double *x64 = nullptr;
    const int *pid = nullptr;
    const float *cd32 = nullptr;                       // HDBSCAN* cd2 per tree position
    const double *cd64 = nullptr;
    double eta = 0.0;          // absolute distance error of the FP32 copy (FP64 input), else 0
    float delta32 = 0.f;       // largest |x64 - x32| of a coordinate (0 for FP32 input)
    int exact32 = 1;           // eta == 0: the FP32 copy is exact
    int fp64 = 0;              // plain FP64 form
    int beta = 2;
    int collect_all = 0;       // GetPairs sends every retrieved pair to list 0 (the full WSPD)
    int rho_sample = 1;        // GetRho starts from every rho_sample-th frontier pair (tuning)
    int disjunctive = 1;       // HDBSCAN*: the separation of Sec. 3.1.2 (0: geometric only)
    int dfs_budget = 8;        // depth-first rounds per warp and traversal step (tuning)
    int medium_max = 1024;     // pair-size classes (tuning): |A||B| <= medium_max: one warp,
    long long big_max = 65536; //   <= big_max: tile kernel, larger: dual-tree kernel
    double rho_lo = 0.0, rho_hi = 0.0;
    float rho_lo_f = 0.f, rho_hi_f = 0.f;   // the smallest floats >= rho_lo, rho_hi
    float above_f = 0.f;                    // a screened value >= this proves a weight >= rho_hi
    unsigned *rho_bits = nullptr;           // GetRho result: bits of a non-negative float (WriteMin)
    int frontier_cap = 0;
    // packed node records used by the traversals (see wspd.cu)
    const NodeRec *rec = nullptr;
    const float *box = nullptr;         // [N][2 dp], groups of four dimensions (box_lo, box_hi)
    int dp = 4;                         // box stride: d rounded up to 4, 8 or 16
    // retrieved well-separated pairs by size class: 0 tiny, 1 small, 2 medium, 3 big (tiles),
    // 4 huge (pruned dual-tree BCCP)
    int2 *list[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    float *list_lb[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};   // each pair's lower bound
    int *list_count = nullptr;          // [5]
    int list_cap[5] = {0, 0, 0, 0, 0};
    int2 *big = nullptr;                // = list[3]
    EdgeK *huge_best = nullptr;         // per huge pair: K-minimum
    unsigned *huge_sbest = nullptr;     // per huge pair: screened minimum (FP32 bits), WriteMin
    int *stack = nullptr;               // per-warp traversal stacks of the dual-tree kernel
    int stack_cap = 0;
    int *big_count = nullptr;           // = list_count + 3
    EdgeK *edges = nullptr;
    int *edge_count = nullptr;
    int edge_cap = 0;
    unsigned *overflow = nullptr;      // bit 0 frontier, bit 1 edges, bit 2 big pairs,
                                       // bit 3 a traversal stack overflowed (internal error)
    // internal nodes not known to be connected, kept from round to round (connectivity only
    // grows): the GetRho frontier reads node_in (all nodes when null) and writes the survivors
    // to node_out, which the GetPairs frontier of the same round reads
    const int *node_in = nullptr, *node_in_n = nullptr;
    int *node_out = nullptr, *node_out_n = nullptr;
    unsigned long long *stat = nullptr; // [0] pairs retrieved, [1] evals, [2] fp64 rechecks,
                                        // [3] tile evals, [4] GetPairs visits, [5] GetRho visits,
                                        // [6] dual-tree evals, [7] peak pending pairs,
                                        // [8] / [9] retrieved pairs whose BCCP fell below / above
                                        // the round's range, [10] evaluations of those pairs
                                        // (group and tile kernels), [11] tile-kernel evaluations
                                        // skipped by the chunk box bound, [12] bits of the largest
                                        // relative FP32 screen error among the rechecks
};

// Traversal step (see findpair_dfs_kernel): warps per block and the capacity of a warp's own
// stack in shared memory (the depth-first rounds per step are TravArgs::dfs_budget).
constexpr int kDfsWarpsPerBlock = 8;
constexpr int kDfsWarpCap = 320;
// traversal counters: [0] stack size, [1] / [2] counts of the two step output buffers,
// [3] input dispenser, [4] finished blocks
constexpr int kTravCounters = 8;

struct DfsArgs {
    int2 *S = nullptr;            // the stack
    int *top = nullptr;           // its size
    const int2 *xin = nullptr;    // previous step's output (top of the logical stack)
    int *xin_count = nullptr;
    int2 *xout = nullptr;         // this step's output
    int *xout_count = nullptr;
    int *next = nullptr;
    unsigned *done = nullptr;
    int chunk = 0, xcap = 0, budget = 0;
};

int dfs_warps(int chunk, int budget);
long long dfs_out_cap(int chunk, int budget);       // pairs one step can write to its output buffer
long long dfs_step_visits(int chunk, int budget);   // pairs one step can visit

// component label of every node (-1 when its points span several components), into T.comp and
// rec[x].l.w; scratch holds 2 n + 1 ints
int launch_comp_labels(const Tree &T, const Points &P, int *uf, NodeRec *rec, int *scratch,
                       Arena &ar, cudaStream_t st);
int run_traversal(TravArgs &a, int2 *stack, int2 *const xbuf[2], int *cnt, int chunk, cudaStream_t st, int *pinned,
                  unsigned *overflow_out, int *steps_out);
void traversal_init(int mode, TravArgs &a, int2 *stack, int *cnt, cudaStream_t st);
void traversal_step(int mode, TravArgs &a, int2 *stack, int2 *const xbuf[2], int *cnt, int step, int chunk,
                    cudaStream_t st);
// histogram of the w2 of e[0, m) over [lo, largest w2] in kSplitBins equal bins (maxbits: the
// largest w2's bits); order-independent, so a split chosen from it is deterministic
constexpr int kSplitBins = 4096;
void w2_histogram(const EdgeK *e, int m, double lo, unsigned long long *maxbits, int *hist, cudaStream_t st);
void keep_below(const EdgeK *in, int m, double bound, EdgeK *out, int *count, cudaStream_t st);
void run_bccp_tiles(TravArgs &a, const int *counts_host, int *next, cudaStream_t st, bool hdb, bool fp64);
void run_bccp_groups(TravArgs &a, const int *counts_host, cudaStream_t st);
int run_bccp_huge(TravArgs &a, const int2 *pairs, const float *lbs, int m, long long *items, long long *total,
                  cudaStream_t st, Arena &ar, bool hdb, bool fp64, int stack_warps);
void pack_nodes(const Tree &T, int d, int dp, NodeRec *rec, float *box, cudaStream_t st);
// the point-major copy x4 of x32 (dp / 4 float4s per point)
void point_major(const float *x32, int n, int d, int dp, float4 *x4, cudaStream_t st);

// gfk.cu: the list steps of the GFK and EMST-Naive forms
void gfk_split(const TravArgs &a, const int2 *S, const float *lb, int m, long long beta, int2 *keep, float *keep_lb,
               int *keep_count, cudaStream_t st);
void gfk_min_lb(const float *lb, int m, unsigned *rho_bits, cudaStream_t st);
void gfk_partition(const EdgeK *pool, int m, double hi, EdgeK *batch, int *batch_count, int batch_cap, EdgeK *rest,
                   int *rest_count, unsigned *overflow, cudaStream_t st);
void gfk_filter_pairs(const int2 *S, const float *lb, int m, const NodeRec *rec, int2 *out, float *out_lb, int *count,
                      cudaStream_t st);
void gfk_filter_edges(const EdgeK *pool, int m, const int *uf, EdgeK *out, int *count, cudaStream_t st);

}  // namespace wm
