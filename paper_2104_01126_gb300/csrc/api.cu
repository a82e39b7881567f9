// api.cu -- the C ABI (include/wspdmst.h) and the host orchestration of the MemoGFK rounds
// (Algorithm 3).  Every step of the computation runs in the kernels of this library; the host
// only sequences launches and reads back the few scalars that steer the rounds (rho_hi, counts).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <string>
#include <vector>

#include "wm_internal.cuh"
#include "wspd.cuh"
#include "batch.cuh"
#include "hdb.cuh"

namespace wm {

std::atomic<long long> g_launch_count{0};

int ingest_points(const void *dev_src, int n, int d, int dtype, int layout, Points &P, Arena &ar, cudaStream_t st,
                  unsigned *pinned);
int build_tree(Points &P, Tree &T, Arena &ar, cudaStream_t st, int *pinned, bool tight_diameters);
int batch_kruskal(const EdgeK *e, int m, int n, int *uf, unsigned long long *R, EdgeK *out, int out_base, int *accepted,
                  Arena &ar, cudaStream_t st, int *pinned);

// ----------------------------------------------------------------------------- error state
static thread_local std::string g_detail;
static void set_detail(const char *fmt, const char *a = "", long long b = 0)
{
    char buf[512];
    snprintf(buf, sizeof buf, fmt, a, b);
    g_detail = buf;
}
static void set_detail(const char *fmt, long long b, const char *a)
{
    char buf[512];
    snprintf(buf, sizeof buf, fmt, b, a);
    g_detail = buf;
}

void set_error_detail(const char *msg) { g_detail = msg; }

// pinned host scratch for scalar readbacks (one per thread)
// 64 KiB of pinned host memory per thread, freed when the thread ends
struct PinnedScratch {
    int *p = nullptr;
    ~PinnedScratch()
    {
        if (p) cudaFreeHost(p);
    }
};

static int *pinned_scratch()
{
    static thread_local PinnedScratch s;
    if (!s.p) {
        if (cudaMallocHost((void **)&s.p, 1 << 16) != cudaSuccess) s.p = nullptr;
    }
    return s.p;
}

// Timing events are reused: creating and destroying CUDA events around every launch of the
// host-steered rounds would leave the device idle while the host does it.  One pool per thread and
// device (an event belongs to the device that was current when it was created).
struct EventPool {
    std::vector<cudaEvent_t> free_[64];
    ~EventPool()
    {
        for (auto &v : free_)
            for (cudaEvent_t e : v) cudaEventDestroy(e);
    }
};
static thread_local EventPool g_event_pool;

static cudaEvent_t pooled_event(int dev)
{
    std::vector<cudaEvent_t> &v = g_event_pool.free_[dev & 63];
    if (!v.empty()) {
        cudaEvent_t e = v.back();
        v.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

static void return_events(int dev, std::vector<cudaEvent_t> &evs)
{
    std::vector<cudaEvent_t> &v = g_event_pool.free_[dev & 63];
    for (cudaEvent_t e : evs)
        if (e) v.push_back(e);
    evs.clear();
}

// ------------------------------------------------------------------ library-managed cache
struct DevCache {
    std::mutex mu;
    char *ptr = nullptr;
    size_t cap = 0;
};
static DevCache g_cache[64];

// Stream-ordered pool of the workspaces of concurrent batch groups, one per device; it keeps what
// it has allocated between calls (wm_release_cache returns it to the system).
struct BatchPool {
    std::mutex mu;
    cudaMemPool_t pool = nullptr;
};
static BatchPool g_batch_pool[64];

static cudaMemPool_t batch_pool(int dev)
{
    BatchPool &bp = g_batch_pool[dev & 63];
    std::lock_guard<std::mutex> lk(bp.mu);
    if (!bp.pool) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        if (cudaMemPoolCreate(&bp.pool, &props) != cudaSuccess) {
            cudaGetLastError();
            bp.pool = nullptr;
            return nullptr;
        }
        unsigned long long keep = ~0ull;
        cudaMemPoolSetAttribute(bp.pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    return bp.pool;
}

struct Caps {
    long long chunk = 0;        // pairs popped per traversal step (= capacity of each pair list)
    long long edges = 0;        // candidate edges per round (the allocated batch)
    long long edges_soft = 0;   // MemoGFK: the batch a round fills before it may grow to `edges`
                                // (0: all of it; see the overflow policy in memogfk)
    int frontier_scale = 1;     // multiplier of the stack bound (grown after an overflow)
    long long extra_bytes = 0;  // additional arena bytes (grown after the arena ran out)
    long long wspd_pairs = 0;   // GFK / EMST-Naive: capacity of the materialised WSPD (0 otherwise)
};

// Well-separated pairs per point of the full WSPD by dimension (measured on uniform and
// clustered inputs; it grows with the dimension and slowly with n): the first capacity of the
// materialised WSPD, grown after an overflow.
static long long wspd_pairs_guess(long long n, int d)
{
    const long long per = d <= 1 ? 4 : d == 2 ? 16 : d == 3 ? 64 : d == 4 ? 200 : d == 5 ? 800 : 4000;
    return std::max<long long>(1 << 16, per * n);
}

static size_t estimate_bytes(long long n, int d, int min_pts, const Caps &c)
{
    const long long N = 2 * n;
    long long lg = 1;
    while ((1LL << lg) < n) ++lg;
    const long long depth = 2 * lg + 16;   // typical; memogfk sizes the stack from the real depth
    const int dp = d <= 4 ? 4 : d <= 8 ? 8 : 16;
    size_t b = 0;
    b += (size_t)n * d * 8;                 // device copy of the input
    b += (size_t)n * d * 28;                // points in input order, in tree order, build scratch
    b += (size_t)n * 60;                    // ids (3), pos, uf, R (4 x 8 B), component-label scratch
    b += (size_t)N * (8 * d + 48);          // tree arrays (+ build scratch counters)
    b += (size_t)n * 8;                     // small lists
    b += (size_t)N * (32 + 8 * dp);         // packed node records
    b += (size_t)n * 4 * dp;                // point-major FP32 copy
    b += (size_t)((N / 2 + 2 + (2 * depth + 4) * 2 * c.chunk) * c.frontier_scale + 8 * c.chunk) * 8;   // stack, step outputs
    b += (size_t)8 * (c.chunk + 1) * (5 * 12 + 16 + 4 + 8);  // pair lists with bounds (8 chunks each), huge-pair slots
    b += (size_t)num_sms() * 64 * (depth + 4) * 4;                                                           // dual stacks
    b += (size_t)c.edges * 16 * 3 + (size_t)c.edges * 24;   // batch, filtered, sort tmp, kruskal
    b += (size_t)n * 16 * 2;                // output tree + conversion
    if (c.wspd_pairs > 0)                   // GFK / EMST-Naive: pairs and bounds (x2), pool (x2), batch, sort
        b += (size_t)c.wspd_pairs * (12 * 2 + 16 * 2 + 16 + 16) + (size_t)n * 16;
    if (min_pts > 0) {
        long long kk = min_pts + 16;
        b += (size_t)n * 12 + (size_t)n * 8;            // cd64, cd32, node bounds
        b += (size_t)n * kk * 16 * 2;                   // repair edges + sort tmp
        b += (size_t)n * 192;                           // dendrogram / Euler tour scratch
    }
    return b + (8u << 20) + (size_t)n * 64 + (size_t)c.extra_bytes;
}

// Edge counters and capacities are 32-bit ints on the device; the batch stays below 2^31 with
// room for the appends in flight past its end (a round that needs more lowers its rho_hi).
constexpr long long kMaxEdgeCap = (1LL << 31) - (1LL << 24);

static Caps default_caps(long long n, int min_pts)
{
    Caps c;
    c.chunk = std::min<long long>(1 << 21, std::max<long long>(1 << 12, 4 * n));
    c.edges = std::min(kMaxEdgeCap, 4 * n + (1 << 20) + (min_pts > 0 ? (long long)n * (min_pts + 16) : 0));
    c.edges_soft = 0;
    c.frontier_scale = 1;
    c.extra_bytes = 0;
    c.wspd_pairs = 0;
    return c;
}

// ------------------------------------------------------------------------------- tuning
// The built-in table (written by the autotuner): builtin_tuning(n, d, min_pts, &t).
#include "tuning_table.inc"

static std::mutex g_tune_mu;
static bool g_tune_set = false;
static wm_tuning g_tune_override{};

static bool tuning_valid(const wm_tuning &t)
{
    return (t.tight_diameters == 0 || t.tight_diameters == 1) &&
           (t.chunk_log2 == 0 || (t.chunk_log2 >= 12 && t.chunk_log2 <= 24)) && t.dfs_budget >= 1 &&
           t.dfs_budget <= 64 && t.route_big >= 0 && t.medium_max >= 65 && t.medium_max <= 4096 &&
           t.big_max >= t.medium_max && t.combined >= 0 && t.combined <= 2 && t.getrho_sample >= 0 &&
           t.getrho_sample <= 1024 && t.edges_per_point >= 0 && t.edges_per_point <= 64 &&
           (t.range_ratio == 0 || (t.range_ratio >= 2 && t.range_ratio <= 1 << 20)) && t.range_gate >= 0 &&
           t.range_gate <= 1 << 20;
}

static wm_tuning tuning_for(long long n, int d, int min_pts)
{
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        if (g_tune_set) return g_tune_override;
    }
    wm_tuning t{};
    builtin_tuning(n, d, min_pts, &t);
    return t;
}

// Capacities of a call: the defaults, with the traversal chunk of the tuning (never above the
// default's max(2^12, 4n): a larger chunk only enlarges the stack of a small problem) and its
// edge batch.  Every estimate of a call's workspace (wm_query_footprint, the batch and serving
// workspaces) uses it.
static Caps caps_for(long long n, int d, int min_pts)
{
    Caps c = default_caps(n, min_pts);
    const wm_tuning t = tuning_for(n, d, min_pts);
    if (t.chunk_log2) c.chunk = std::min<long long>(1LL << t.chunk_log2, std::max<long long>(1 << 12, 4 * n));
    if (t.edges_per_point > 4) {
        c.edges_soft = c.edges;
        c.edges = std::min(kMaxEdgeCap, c.edges + (long long)(t.edges_per_point - 4) * n);
        if (c.edges_soft >= c.edges) c.edges_soft = 0;
    }
    return c;
}

// ------------------------------------------------------------------------------- kernels
namespace {

__global__ void init_uf_kernel(int *uf, unsigned long long *R, int n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        uf[i] = i;
        R[i] = ~0ull;   // four reservation words per vertex (two sets of two)
        R[n + i] = ~0ull;
        R[2LL * n + i] = ~0ull;
        R[3LL * n + i] = ~0ull;
    }
}

// wm_edge output: u, v, w = sqrt(w2)
__global__ void to_wm_edge_kernel(const EdgeK *__restrict__ e, int m, wm_edge *__restrict__ out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        EdgeK x = e[i];
        wm_edge o;
        o.u = edge_u(x);
        o.v = edge_v(x);
        o.w = sqrt(edge_w2(x));
        out[i] = o;
    }
}

// pairwise FP64 sum of sqrt(w2) (block partials, then one block)
__global__ void sum_sqrt_kernel(const EdgeK *__restrict__ e, int m, double *partial)
{
    __shared__ double sm[256];
    double s = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) s += sqrt(edge_w2(e[i]));
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o; o >>= 1) {
        if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sm[0];
}

__global__ void sum_partials_kernel(const double *partial, int m, double *out)
{
    __shared__ double sm[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) s += partial[i];
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o; o >>= 1) {
        if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sm[0];
}

// appends the edges of src whose w2 lies in [lo, hi) to dst (non-negative doubles and +inf order
// like their bit patterns)
__global__ void take_range_kernel(const EdgeK *__restrict__ src, int m, double lo, double hi, EdgeK *__restrict__ dst,
                                  int *count, int cap, unsigned *overflow)
{
    __shared__ int sh[32];
    const unsigned long long blo = (unsigned long long)__double_as_longlong(lo);
    const unsigned long long bhi = (unsigned long long)__double_as_longlong(hi);
    for (int b0 = blockIdx.x * blockDim.x; b0 < m; b0 += gridDim.x * blockDim.x) {
        const int t = b0 + threadIdx.x;
        EdgeK e;
        bool take = false;
        if (t < m) {
            e = src[t];
            take = e.hi >= blo && e.hi < bhi;
        }
        const int slot = block_append(count, take ? 1 : 0, sh);
        if (take) {
            if (slot < cap) dst[slot] = e;
            else atomicOr(overflow, 2u);
        }
    }
}

// FP32 throughput probe: every thread runs eight independent chains of fused multiply-adds
// (enough in flight per warp to hide the FMA latency); the result is stored only on a condition
// that never holds, which keeps the arithmetic from being removed.
__global__ void __launch_bounds__(256) ffma_probe_kernel(float *out, int iters, float x, float y)
{
    float c0 = threadIdx.x * 1e-7f, c1 = c0 + 1e-3f, c2 = c0 + 2e-3f, c3 = c0 + 3e-3f;
    float c4 = c0 + 4e-3f, c5 = c0 + 5e-3f, c6 = c0 + 6e-3f, c7 = c0 + 7e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            c0 = fmaf(c0, x, y); c1 = fmaf(c1, x, y); c2 = fmaf(c2, x, y); c3 = fmaf(c3, x, y);
            c4 = fmaf(c4, x, y); c5 = fmaf(c5, x, y); c6 = fmaf(c6, x, y); c7 = fmaf(c7, x, y);
        }
    }
    const float t = ((c0 + c1) + (c2 + c3)) + ((c4 + c5) + (c6 + c7));
    if (t == -1.0f) out[blockIdx.x] = t;
}

}  // namespace

// ------------------------------------------------------------------------------ call state
struct Call {
    cudaStream_t st = nullptr;
    Arena ar;
    int *pin = nullptr;
    wm_stats stats{};
    wm_tuning tune{};
    int method = WM_METHOD_MEMOGFK;   // wm_opts.method
    int disjunctive = 1;              // HDBSCAN*: the separation of Sec. 3.1.2 (0: GanTao's)
    int precision = WM_PREC_FP32_SCREEN;
    bool timing = true;   // per-kernel CUDA-event timing into stats
    double event_ms(cudaEvent_t a, cudaEvent_t b)
    {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        return ms;
    }
};

static bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

#define WM_TRY(x)                                   \
    do {                                            \
        int rc_ = (x);                              \
        if (rc_) return rc_;                        \
    } while (0)
#define WM_CK(x)                                                                     \
    do {                                                                             \
        cudaError_t e_ = (x);                                                        \
        if (e_ != cudaSuccess) {                                                     \
            set_detail("CUDA error %s (line %lld)", cudaGetErrorString(e_), __LINE__); \
            return WM_ECUDA;                                                         \
        }                                                                            \
    } while (0)

struct Timer {
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
    double ms() const { return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count(); }
};

// the smallest float >= r (r >= 0 or +inf)
static float float_ru(double r)
{
    float f = (float)r;
    if ((double)f < r) f = std::nextafter(f, INFINITY);
    return f;
}

// The smallest float s whose rigorous lower bound on the exact FP64 weight of a pair screened at s
// reaches hi.  The FP32 screen errs by at most 2^-19 relative plus subnormal rounding when the FP32
// copy is exact, so the weight is at least s (1 - 2^-18) - 2e-42; otherwise the copy's distance
// error eta (absolute) comes on top: (sqrt(s (1 - 2^-18) - 2e-42) - eta)^2 (1 - 2^-40).  For
// HDBSCAN* a screened value may be a core distance, which bounds its FP64 value from below within
// 2^-22, so s must also reach hi / (1 - 2^-22).  Inverted with outward margins.
static float above_threshold(double hi, const TravArgs &a)
{
    if (!(hi < INFINITY)) return INFINITY;
    double t = a.exact32 ? hi : std::pow(std::sqrt(hi / (1.0 - 1.0 / 1099511627776.0)) + a.eta, 2.0);
    t = (t * (1.0 + 1e-15) + 2e-42) / (1.0 - 1.0 / 262144.0);
    if (a.cd64) t = std::max(t, hi / (1.0 - 1.0 / 4194304.0));
    return float_ru(t * (1.0 + 1e-12));
}

static void set_rho(TravArgs &a, double lo, double hi)
{
    a.rho_lo = lo;
    a.rho_hi = hi;
    a.rho_lo_f = float_ru(lo);
    a.rho_hi_f = float_ru(hi);
    a.above_f = above_threshold(hi, a);
}

// MemoGFK rounds (Algorithm 3).  On return E_out holds the tree edges in K order: n-1 of them, or
// `target` when the points form several instances that must not be joined (a batch): then every
// edge weight is below rho_cap, rho_hi never exceeds it, and no pair at or above it is retrieved.
// hdb: optional HDBSCAN* state (node cd bounds, per-position cd2, repair edges).
static int memogfk(Call &C, Points &P, Tree &T, const HdbState *hdb, const Caps &caps, EdgeK *E_out, int *uf,
                   unsigned long long *R, unsigned *overflow_bits, long long target = -1, double rho_cap = INFINITY)
{
    const int n = P.n;
    if (target < 0) target = (long long)n - 1;
    cudaStream_t st = C.st;
    Arena &ar = C.ar;
    *overflow_bits = 0;
    if (n <= 1) return 0;
    size_t mark = ar.off;
    const int chunk = (int)caps.chunk;
    const long long fcap = ((long long)T.N / 2 + 2 + (2LL * T.depth + 4) * 2 * chunk) * caps.frontier_scale;
    if (fcap > 0x7fffffffLL) { set_detail("WSPD stack capacity exceeds 2^31 pairs%s", ""); return WM_ENOMEM; }
    int2 *stack = ar.get<int2>(fcap);
    int2 *const xbuf[2] = {ar.get<int2>(4LL * chunk), ar.get<int2>(4LL * chunk)};   // step outputs
    // pair lists hold kListChunks chunks' worth of retrieved pairs; they are flushed (BCCP) when
    // one of them could overflow within the next poll interval, and when the traversal ends
    const int kPoll = 3, kListChunks = 8;
    const long long lcap = (long long)kListChunks * chunk;
    int2 *lists[5];
    float *list_lbs[5];
    for (int c = 0; c < 5; ++c) {
        lists[c] = ar.get<int2>(lcap);
        list_lbs[c] = ar.get<float>(lcap);
    }
    EdgeK *huge_best = ar.get<EdgeK>(lcap + 1);
    unsigned *huge_sbest = ar.get<unsigned>(lcap + 1);
    long long *huge_items = ar.get<long long>(lcap + 1);
    const int stack_warps = num_sms() * 8 * 8;   // warps of the dual-tree kernel (grid-stride)
    int *dual_stack = ar.get<int>((size_t)stack_warps * (T.depth + 4));
    const int dp = P.d <= 4 ? 4 : P.d <= 8 ? 8 : 16;
    NodeRec *rec = ar.get<NodeRec>(T.N);
    float *box = ar.get<float>((size_t)T.N * 2 * dp);
    float4 *x4 = ar.get<float4>((size_t)n * (dp / 4));
    EdgeK *batch = ar.get<EdgeK>(caps.edges), *filt = ar.get<EdgeK>(caps.edges), *tmp = ar.get<EdgeK>(caps.edges);
    int *cnts = ar.get<int>(64);
    unsigned *rho = ar.get<unsigned>(2);
    int *split_hist = ar.get<int>(kSplitBins);
    unsigned long long *split_max = ar.get<unsigned long long>(1);
    unsigned *ovf = ar.get<unsigned>(2);
    unsigned long long *stat = ar.get<unsigned long long>(16);
    int *comp_scratch = ar.get<int>(2LL * n + 1);
    if (ar.failed) return WM_ENOMEM;
    // counters: [2..6] pair-list counts, [7] edge count, [10..11] counts of the two node lists,
    // [12..13] 64-bit huge-pair item total, [16..17] tile-kernel pair dispensers,
    // [32..32+kTravCounters) traversal state
    int *lcount = cnts + 2, *ecount = cnts + 7, *tcnt = cnts + 32;
    {
        Tree T2 = T;
        if (hdb) { T2.cdmin = hdb->cdmin; T2.cdmax = hdb->cdmax; }
        pack_nodes(T2, P.d, dp, rec, box, st);
        point_major(P.x32, n, P.d, dp, x4, st);
    }
    WM_CK(cudaMemsetAsync(stat, 0, 16 * sizeof(unsigned long long), st));
    WM_CK(cudaMemsetAsync(ovf, 0, 2 * sizeof(unsigned), st));
    WM_CK(cudaMemsetAsync(cnts, 0, 64 * sizeof(int), st));

    TravArgs a;
    a.N = T.N; a.n = n; a.d = P.d;
    a.lo = T.lo; a.hi = T.hi; a.diam2 = T.diam2;
    a.begin = T.begin; a.end = T.end; a.left = T.left; a.right = T.right; a.comp = T.comp;
    a.x32 = P.x32; a.x4 = x4; a.x64 = P.x64; a.pid = P.pid;
    a.fp64 = C.precision == WM_PREC_FP64;
    a.eta = a.fp64 ? 0.0 : 2.0 * (double)P.delta * std::sqrt((double)P.d) * (1.0 + 1e-6);
    a.exact32 = a.eta == 0.0;
    a.delta32 = P.delta;
    a.dfs_budget = C.tune.dfs_budget;
    a.medium_max = C.tune.medium_max;
    a.big_max = C.tune.big_max;
    a.disjunctive = C.disjunctive;
    a.rho_sample = C.tune.getrho_sample > 0 ? C.tune.getrho_sample : 1;
    if (hdb) {
        a.cdmin = hdb->cdmin; a.cdmax = hdb->cdmax; a.cd32 = hdb->cd32; a.cd64 = hdb->cd64;
    }
    a.frontier_cap = (int)fcap;
    a.rec = rec; a.box = box; a.dp = dp;
    for (int c = 0; c < 5; ++c) { a.list[c] = lists[c]; a.list_lb[c] = list_lbs[c]; a.list_cap[c] = (int)lcap; }
    a.list_count = lcount;
    a.big = lists[3]; a.big_count = lcount + 3;
    a.huge_best = huge_best; a.huge_sbest = huge_sbest;
    a.stack = dual_stack; a.stack_cap = T.depth + 4;
    a.edges = batch; a.edge_count = ecount;
    a.edge_cap = (int)(caps.edges_soft > 0 && caps.edges_soft < caps.edges ? caps.edges_soft : caps.edges);
    a.overflow = ovf;
    a.stat = stat;
    a.rho_bits = rho;
    EdgeK *spare = filt;   // second edge buffer for compaction when rho_hi shrinks
    int *nodes[2] = {ar.get<int>(T.N / 2 + 1), ar.get<int>(T.N / 2 + 1)};
    if (ar.failed) return WM_ENOMEM;
    a.node_in = nullptr;
    a.node_in_n = nullptr;
    a.node_out = nodes[0];
    a.node_out_n = cnts + 10;

    // CUDA-event intervals of the round's kernels (when C.timing), summed into the stats per kind
    enum { kSpanGetPairs, kSpanGetRho, kSpanFlush, kSpanGroup, kSpanTile, kSpanDual };
    std::vector<cudaEvent_t> evs;
    std::vector<int3> spans;   // (start event, end event, kind)
    int dev = 0;
    cudaGetDevice(&dev);
    auto mark_event = [&]() -> int {
        if (!C.timing) return -1;
        cudaEvent_t e = pooled_event(dev);
        if (!e) return -1;
        cudaEventRecord(e, st);
        evs.push_back(e);
        return (int)evs.size() - 1;
    };
    auto add_span = [&](int i, int j, int kind) {
        if (i >= 0 && j >= 0) spans.push_back(make_int3(i, j, kind));
    };
    struct EventsGuard {   // events left by an early return go back to the pool too
        std::vector<cudaEvent_t> &v;
        int dev;
        ~EventsGuard() { return_events(dev, v); }
    } events_guard{evs, dev};
    auto collect_spans = [&]() -> int {
        if (evs.empty()) return 0;
        WM_CK(cudaEventSynchronize(evs.back()));
        for (const int3 &sp : spans) {
            const double ms = C.event_ms(evs[sp.x], evs[sp.y]);
            switch (sp.z) {
            case kSpanGetPairs: C.stats.ms_getpairs += ms; break;
            case kSpanGetRho: C.stats.ms_getrho += ms; break;
            case kSpanFlush: C.stats.ms_bccp += ms; break;
            case kSpanGroup: C.stats.ms_bccp_group += ms; break;
            case kSpanTile: C.stats.ms_tile_kernel += ms; break;
            default: C.stats.ms_bccp_dual += ms; break;
            }
        }
        return_events(dev, evs);
        spans.clear();
        return 0;
    };
    int nE = 0;
    double rho_lo = 0.0;
    long long beta = 2;
    // tuning combined = 2: rounds start as two passes; once, after two rounds or more, the GetRho
    // traversals have visited at least kOnePassRatio times as many node pairs as the GetPairs
    // traversals, the remaining rounds find the GetRho minimum during GetPairs instead (the
    // first round's ratio says little: it is high on every input)
    constexpr double kOnePassRatio = 0.5;
    bool adaptive_one_pass = false;
    const double inf = INFINITY;
    int rounds = 0;
    while (nE < target) {
        if (++rounds > 4096) { set_detail("MemoGFK made no progress%s (%lld rounds)", "", rounds); return WM_EINTERNAL; }
        Timer tw;
        WM_TRY(launch_comp_labels(T, P, uf, rec, comp_scratch, ar, st));
        a.beta = (int)std::min<long long>(beta, 0x7fffffff);
        double rho_hi;
        // Combined pass (tuning): GetRho's minimum R is kept on the device while GetPairs runs;
        // each flush takes the R read at that moment as rho_hi and the round ends with the final
        // R, i.e. GetRho's value, whose edges at or above it are dropped before Kruskal.
        const bool combined = C.tune.combined == 1 || (C.tune.combined == 2 && adaptive_one_pass);
        // Tuning range_ratio: the round's range [rho_lo, rho_hi) ends at most at range_ratio x
        // rho_lo.  Any rho_hi up to GetRho's bound is correct (GetPairs takes pairs of any size
        // whose lower bound is below it); a smaller one retrieves fewer pairs whose BCCP lies
        // beyond what the edge batch can hold, at the price of more rounds.
        // With range_gate > 0 the limit applies only while the call's BCCP work is not small
        // beside its traversal work so far (node-pair visits < range_gate x BCCP evaluations):
        // a traversal-bound call loses more to the extra rounds than it saves in BCCPs.
        double round_cap = rho_cap;
        if (C.tune.range_ratio > 0 && rho_lo > 0.0) {
            bool apply = true;
            if (C.tune.range_gate > 0) {
                WM_CK(cudaMemcpyAsync(C.pin + 64, stat, 6 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
                WM_CK(cudaStreamSynchronize(st));
                unsigned long long hs6[6];
                memcpy(hs6, C.pin + 64, sizeof hs6);
                apply = (double)(hs6[4] + hs6[5]) < (double)C.tune.range_gate * (double)hs6[1];
            }
            if (apply) round_cap = std::min<double>(rho_cap, rho_lo * C.tune.range_ratio);
        }
        const int tmode = combined ? 2 : 1;
        double rho_used = 0.0;   // largest rho_hi a flush of this round has used
        if (!combined) {
            // ---- GetRho
            fill_i32((int *)rho, 0x7f800000, 1, st);   // +inf
            set_rho(a, rho_lo, inf);
            unsigned ob = 0;
            const int r0 = mark_event();
            WM_TRY(run_traversal(a, stack, xbuf, tcnt, chunk, st, C.pin, &ob, nullptr));
            add_span(r0, mark_event(), kSpanGetRho);
            if (ob) { *overflow_bits = ob; return 0; }
            WM_CK(cudaMemcpyAsync(C.pin, rho, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
            WM_CK(cudaStreamSynchronize(st));
            float rho_f;
            memcpy(&rho_f, C.pin, sizeof rho_f);
            rho_hi = std::min<double>(rho_f, round_cap);
            if (rho_hi < rho_lo) rho_hi = rho_lo;
        } else {
            float cap_f = float_ru(round_cap);
            unsigned cap_bits;
            memcpy(&cap_bits, &cap_f, sizeof cap_bits);
            fill_i32((int *)rho, (int)cap_bits, 1, st);
            rho_hi = std::max<double>(std::min<double>(cap_f, round_cap), rho_lo);
        }
        double rho_shrunk = inf;   // bound set by an edge-batch overflow in this round
        // ---- GetPairs in chunks; the retrieved pairs of every chunk get their BCCP right away
        set_rho(a, rho_lo, rho_hi);
        a.edges = batch;
        spare = filt;
        WM_CK(cudaMemsetAsync(cnts + 2, 0, 6 * sizeof(int), st));
        traversal_init(tmode, a, stack, tcnt, st);
        int steps = 0;
        int last_e = 0;                  // edge count and overflow bits read after the last flush
        unsigned last_ovf = 0;
        int span0 = mark_event();
        while (true) {
            for (int b = 0; b < kPoll; ++b, ++steps) traversal_step(tmode, a, stack, xbuf, tcnt, steps, chunk, st);
            WM_CK(cudaMemcpyAsync(C.pin, cnts, 8 * sizeof(int), cudaMemcpyDeviceToHost, st));
            WM_CK(cudaMemcpyAsync(C.pin + 8, ovf, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
            WM_CK(cudaMemcpyAsync(C.pin + 16, tcnt, kTravCounters * sizeof(int), cudaMemcpyDeviceToHost, st));
            if (combined) WM_CK(cudaMemcpyAsync(C.pin + 24, rho, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
            WM_CK(cudaStreamSynchronize(st));
            if (C.pin[8]) { *overflow_bits = (unsigned)C.pin[8]; return 0; }
            if (combined) {
                float rf;
                memcpy(&rf, C.pin + 24, sizeof rf);
                rho_hi = std::max<double>(std::min<double>(std::min<double>(rf, round_cap), rho_shrunk), rho_lo);
            }
            const bool empty = C.pin[16] == 0 && C.pin[17] == 0 && C.pin[18] == 0;
            int lc[5] = {C.pin[2], C.pin[3], C.pin[4], C.pin[5], C.pin[6]};
            int e = C.pin[7];
            bool flush = empty;
            for (int c = 0; c < 5; ++c) flush = flush || lc[c] > lcap - (long long)kPoll * dfs_step_visits(chunk, a.dfs_budget);
            if (!flush) continue;
            add_span(span0, mark_event(), kSpanGetPairs);
            const int flush0 = mark_event();
            if (combined && rho_hi != a.rho_hi) set_rho(a, rho_lo, rho_hi);
            rho_used = std::max(rho_used, a.rho_hi);
            // BCCP of the retrieved pairs.  Emission is capacity-checked; if this flush overflows the
            // edge batch, its partial output is dropped, rho_hi is lowered to a quantile of the valid
            // edges (pairs seen so far were retrieved under the larger bound, so they stay complete
            // for the smaller range) and the flush is redone from the intact lists.
            const int e_before = e;
            for (int attempt = 0;; ++attempt) {
                const int g0 = mark_event();
                run_bccp_groups(a, lc, st);
                const int g1 = mark_event();
                add_span(g0, g1, kSpanGroup);
                // a short list of big pairs would occupy a few warps for long: the pruned
                // dual-tree kernel spreads each pair over warps of 32 query points instead
                const bool route_big = lc[3] > 0 && lc[3] <= C.tune.route_big;
                int lt[5] = {lc[0], lc[1], lc[2], route_big ? 0 : lc[3], lc[4]};
                run_bccp_tiles(a, lt, cnts + 16, st, hdb != nullptr, a.fp64 != 0);
                const int g2 = mark_event();
                add_span(g1, g2, kSpanTile);
                if (route_big)
                    WM_TRY(run_bccp_huge(a, a.list[3], a.list_lb[3], lc[3], huge_items, (long long *)(cnts + 12), st,
                                         ar, hdb != nullptr, a.fp64 != 0, stack_warps));
                WM_TRY(run_bccp_huge(a, a.list[4], a.list_lb[4], lc[4], huge_items, (long long *)(cnts + 12), st, ar,
                                     hdb != nullptr, a.fp64 != 0, stack_warps));
                add_span(g2, mark_event(), kSpanDual);
                WM_CK(cudaMemcpyAsync(C.pin, ecount, sizeof(int), cudaMemcpyDeviceToHost, st));
                WM_CK(cudaMemcpyAsync(C.pin + 1, ovf, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
                WM_CK(cudaStreamSynchronize(st));
                last_e = C.pin[0];
                last_ovf = (unsigned)C.pin[1];
                if (!(C.pin[1] & 2u)) break;
                if (attempt >= 8) { *overflow_bits = 2; return 0; }
                // Overflow policy.  Lowering rho_hi defers the rest of the round's range to later
                // rounds, where more points are connected and more pairs are filtered out before
                // their BCCP; but every later round traverses the WSPD again.  So a call whose work
                // so far is mostly traversal (node-pair visits >= kGrowRatio x BCCP evaluations)
                // first grows its batch to the allocated capacity and redoes the flush with the
                // same range; otherwise (or once grown) it lowers rho_hi.  On GB300 the ratio at
                // the first overflow was 64-114 for uniform 7-D points (10^6, 10^7), where growing
                // halved the call's time, and at most 13 for variable-density blobs in 5-D and 7-D,
                // where lowering rho_hi was faster.
                if (a.edge_cap < caps.edges) {
                    constexpr double kGrowRatio = 20.0;
                    WM_CK(cudaMemcpyAsync(C.pin + 64, stat, 6 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
                    WM_CK(cudaStreamSynchronize(st));
                    unsigned long long hs6[6];
                    memcpy(hs6, C.pin + 64, sizeof hs6);
                    if ((double)(hs6[4] + hs6[5]) >= kGrowRatio * (double)hs6[1]) {
                        a.edge_cap = (int)caps.edges;
                        fill_i32(ecount, e_before, 1, st);
                        WM_CK(cudaMemsetAsync(ovf, 0, sizeof(unsigned), st));
                        C.stats.edge_batch_grown = 1;
                        continue;
                    }
                }
                const int valid = std::min<long long>(C.pin[0], a.edge_cap) > 0 ? (int)std::min<long long>(C.pin[0], a.edge_cap) : 0;
                if (valid < 1) { *overflow_bits = 2; return 0; }
                // the new bound: the 40% point of the valid edges' weights, from a histogram (the
                // same choice whatever order the edges were appended in)
                w2_histogram(a.edges, valid, rho_lo, split_max, split_hist, st);
                WM_CK(cudaMemcpyAsync(C.pin + 8192, split_hist, sizeof(int) * kSplitBins, cudaMemcpyDeviceToHost, st));
                WM_CK(cudaMemcpyAsync(C.pin + 64, split_max, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
                WM_CK(cudaStreamSynchronize(st));
                double wmax;
                memcpy(&wmax, C.pin + 64, sizeof wmax);
                long long acc = 0;
                int bin = 0;
                while (bin < kSplitBins - 1 && acc + C.pin[8192 + bin] < (long long)(0.4 * valid)) acc += C.pin[8192 + bin++];
                double nh = rho_lo + (wmax - rho_lo) * ((double)(bin + 1) / kSplitBins);
                if (!(nh > rho_lo)) nh = std::nextafter(rho_lo, inf);
                if (!(nh < a.rho_hi)) { *overflow_bits = 2; return 0; }   // cannot shrink: grow and restart
                keep_below(a.edges, e_before, nh, spare, ecount, st);
                std::swap(a.edges, spare);
                rho_hi = nh;
                rho_shrunk = nh;
                set_rho(a, rho_lo, rho_hi);
                if (combined) {   // the traversal's running bound may not exceed it either
                    float nf = float_ru(nh);
                    unsigned nb;
                    memcpy(&nb, &nf, sizeof nb);
                    fill_i32((int *)rho, (int)nb, 1, st);
                }
                WM_CK(cudaMemsetAsync(ovf, 0, sizeof(unsigned), st));
                C.stats.rho_shrinks += 1;
            }
            WM_CK(cudaMemsetAsync(lcount, 0, 5 * sizeof(int), st));
            if (lc[3] > 0 || lc[4] > 0) C.stats.tile_launches += 1;
            span0 = mark_event();
            add_span(flush0, span0, kSpanFlush);
            if (empty) break;
            if (steps > 10000000) { set_detail("WSPD GetPairs traversal did not terminate%s", ""); return WM_EINTERNAL; }
        }
        // the traversal ends with a flush whose sync read the edge count and the overflow bits;
        // nothing has run since
        if (last_ovf) { *overflow_bits = last_ovf; return 0; }
        int m = last_e;
        if (combined && rho_used > rho_hi) {
            // earlier flushes ran with a larger running bound than the final one: keep only the
            // edges of this round's range
            keep_below(a.edges, m, rho_hi, spare, ecount, st);
            std::swap(a.edges, spare);
            WM_CK(cudaMemcpyAsync(C.pin, ecount, sizeof(int), cudaMemcpyDeviceToHost, st));
            WM_CK(cudaStreamSynchronize(st));
            m = C.pin[0];
        }
        C.stats.getpairs_launches += steps;
        C.stats.ms_wspd += tw.ms();
        // ---- HDBSCAN*: repair edges of this weight range join the batch
        if (hdb && hdb->nrep > 0 && rho_hi > rho_lo) {
            launch(take_range_kernel, grid_for(hdb->nrep, 256), 256, 0, st, hdb->rep, hdb->nrep, rho_lo, rho_hi,
                   a.edges, ecount, (int)caps.edges, ovf);
            WM_CK(cudaMemcpyAsync(C.pin, ecount, sizeof(int), cudaMemcpyDeviceToHost, st));
            WM_CK(cudaMemcpyAsync(C.pin + 1, ovf, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
            WM_CK(cudaStreamSynchronize(st));
            if (C.pin[1]) { *overflow_bits = (unsigned)C.pin[1]; return 0; }
            m = C.pin[0];
        }
        // ---- Kruskal (its first step rejects the edges whose endpoints are already connected)
        Timer tk;
        int accepted = 0;
        if (m > 0) {
            C.stats.candidate_edges += m;
            WM_TRY(batch_kruskal(a.edges, m, n, uf, R, E_out, nE, &accepted, ar, st, C.pin));
        }
        C.stats.ms_kruskal += tk.ms();
        // the timed intervals of this round are complete once the stream has synced (Kruskal)
        WM_TRY(collect_spans());
        nE += accepted;
        if (C.tune.combined == 2 && !combined) {
            WM_CK(cudaMemcpyAsync(C.pin, stat + 4, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
            WM_CK(cudaStreamSynchronize(st));
            unsigned long long v[2];
            memcpy(v, C.pin, sizeof v);
            if (rounds >= 2 && v[1] >= kOnePassRatio * v[0] && v[0] > 0) adaptive_one_pass = true;
        }
        if (rho_hi >= rho_cap && nE < target) {
            set_detail("MemoGFK round with rho_hi = its cap left the forest incomplete%s (%lld edges)", "", nE);
            return WM_EINTERNAL;
        }
        rho_lo = rho_hi;
        beta *= 2;
        // this round's surviving nodes are the next round's input
        a.node_in = a.node_out;
        a.node_in_n = a.node_out_n;
        a.node_out = a.node_out == nodes[0] ? nodes[1] : nodes[0];
        a.node_out_n = a.node_out_n == cnts + 10 ? cnts + 11 : cnts + 10;
    }
    {
        // every round appended its tree edges unordered: put the tree in K order
        Timer ts;
        EdgeK *sorted = E_out;
        WM_TRY(radix_sort_edges(E_out, tmp, (int)target, st, ar, &sorted, C.pin + 4096));
        if (sorted != E_out) WM_CK(cudaMemcpyAsync(E_out, sorted, sizeof(EdgeK) * target, cudaMemcpyDeviceToDevice, st));
        WM_CK(cudaStreamSynchronize(st));
        C.stats.ms_kruskal += ts.ms();
    }
    WM_CK(cudaMemcpyAsync(C.pin, stat, 16 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    WM_CK(cudaStreamSynchronize(st));
    unsigned long long hs[16];
    memcpy(hs, C.pin, sizeof hs);
    C.stats.getpairs_visits = (int64_t)hs[4];
    C.stats.getrho_visits = (int64_t)hs[5];
    C.stats.bccp_dual_evals = (int64_t)hs[6];
    C.stats.max_pending_pairs = (int64_t)hs[7];
    C.stats.rounds = rounds;
    C.stats.pairs_retrieved = (int64_t)hs[0];
    C.stats.bccp_evals = (int64_t)hs[1];
    C.stats.fp64_rechecks += (int64_t)hs[2];
    C.stats.bccp_tile_evals = (int64_t)hs[3];
    C.stats.bccp_pairs_below = (int64_t)hs[8];
    C.stats.bccp_pairs_above = (int64_t)hs[9];
    C.stats.bccp_evals_outside = (int64_t)hs[10];
    C.stats.bccp_tile_evals_skipped = (int64_t)hs[11];
    {
        float e;
        const unsigned eb = (unsigned)hs[12];
        memcpy(&e, &eb, sizeof e);
        C.stats.max_rel_screen_err = std::max(C.stats.max_rel_screen_err, (double)e);
    }
    ar.off = mark;
    return 0;
}

// The GFK form (Sec. 3.2.2, Algorithm 2) and, with naive = true, EMST-Naive (the BCCP of every
// pair, then one Kruskal): the full WSPD is materialised by one traversal over [0, +inf) without
// connectivity pruning.  A round then computes the BCCP of the pairs of at most beta points (its
// edge joins the pool, which caches it), sets rho_hi to the smallest lower bound d(A,B) of the
// pairs left, hands the pool's edges lighter than rho_hi (and, for HDBSCAN*, the repair edges of
// [rho_lo, rho_hi)) to Kruskal, drops the pairs whose points are all connected and the pool edges
// whose endpoints are, and doubles beta.  Overflow bits as memogfk (bit 2 for the pair list).
static int gfk_rounds(Call &C, Points &P, Tree &T, const HdbState *hdb, const Caps &caps, EdgeK *E_out, int *uf,
                      unsigned long long *R, unsigned *overflow_bits, bool naive)
{
    const int n = P.n;
    const long long target = (long long)n - 1;
    cudaStream_t st = C.st;
    Arena &ar = C.ar;
    *overflow_bits = 0;
    if (n <= 1) return 0;
    size_t mark = ar.off;
    const int chunk = (int)caps.chunk;
    const long long fcap = ((long long)T.N / 2 + 2 + (2LL * T.depth + 4) * 2 * chunk) * caps.frontier_scale;
    const long long scap = caps.wspd_pairs;
    if (fcap > 0x7fffffffLL || scap > 0x7fffffffLL) { set_detail("GFK capacities exceed 2^31%s", ""); return WM_ENOMEM; }
    int2 *stack = ar.get<int2>(fcap);
    int2 *const xbuf[2] = {ar.get<int2>(4LL * chunk), ar.get<int2>(4LL * chunk)};
    const long long lcap = 8LL * chunk;   // BCCP size-class lists: the pairs are split in segments of lcap
    int2 *lists[5];
    float *list_lbs[5];
    for (int c = 0; c < 5; ++c) {
        lists[c] = ar.get<int2>(lcap);
        list_lbs[c] = ar.get<float>(lcap);
    }
    EdgeK *huge_best = ar.get<EdgeK>(lcap + 1);
    unsigned *huge_sbest = ar.get<unsigned>(lcap + 1);
    long long *huge_items = ar.get<long long>(lcap + 1);
    const int stack_warps = num_sms() * 8 * 8;
    int *dual_stack = ar.get<int>((size_t)stack_warps * (T.depth + 4));
    const int dp = P.d <= 4 ? 4 : P.d <= 8 ? 8 : 16;
    NodeRec *rec = ar.get<NodeRec>(T.N);
    float *box = ar.get<float>((size_t)T.N * 2 * dp);
    float4 *x4 = ar.get<float4>((size_t)n * (dp / 4));
    int2 *S[2] = {ar.get<int2>(scap), ar.get<int2>(scap)};
    float *Slb[2] = {ar.get<float>(scap), ar.get<float>(scap)};
    EdgeK *pool[2] = {ar.get<EdgeK>(scap), ar.get<EdgeK>(scap)};
    EdgeK *batch = ar.get<EdgeK>(scap + 1), *tmp = ar.get<EdgeK>(std::max<long long>(scap, n) + 1);
    int *cnts = ar.get<int>(64);
    unsigned *rho = ar.get<unsigned>(2);
    unsigned *ovf = ar.get<unsigned>(2);
    unsigned long long *stat = ar.get<unsigned long long>(16);
    int *comp_scratch = ar.get<int>(2LL * n + 1);
    if (ar.failed) return WM_ENOMEM;
    // counters: [2..6] class-list counts, [7] pool count, [8] kept pairs, [9] batch count,
    // [10..11] node lists, [12..13] huge items, [16..17] tile dispensers, [32..] traversal state
    int *lcount = cnts + 2, *pcount = cnts + 7, *kcount = cnts + 8, *bcount = cnts + 9, *tcnt = cnts + 32;
    {
        Tree T2 = T;
        if (hdb) { T2.cdmin = hdb->cdmin; T2.cdmax = hdb->cdmax; }
        pack_nodes(T2, P.d, dp, rec, box, st);
        point_major(P.x32, n, P.d, dp, x4, st);
    }
    WM_CK(cudaMemsetAsync(stat, 0, 16 * sizeof(unsigned long long), st));
    WM_CK(cudaMemsetAsync(ovf, 0, 2 * sizeof(unsigned), st));
    WM_CK(cudaMemsetAsync(cnts, 0, 64 * sizeof(int), st));
    TravArgs a;
    a.N = T.N; a.n = n; a.d = P.d;
    a.lo = T.lo; a.hi = T.hi; a.diam2 = T.diam2;
    a.begin = T.begin; a.end = T.end; a.left = T.left; a.right = T.right; a.comp = T.comp;
    a.x32 = P.x32; a.x4 = x4; a.x64 = P.x64; a.pid = P.pid;
    a.fp64 = C.precision == WM_PREC_FP64;
    a.eta = a.fp64 ? 0.0 : 2.0 * (double)P.delta * std::sqrt((double)P.d) * (1.0 + 1e-6);
    a.exact32 = a.eta == 0.0;
    a.delta32 = P.delta;
    a.dfs_budget = C.tune.dfs_budget;
    a.medium_max = C.tune.medium_max;
    a.big_max = C.tune.big_max;
    a.disjunctive = C.disjunctive;
    a.rho_sample = C.tune.getrho_sample > 0 ? C.tune.getrho_sample : 1;
    if (hdb) { a.cdmin = hdb->cdmin; a.cdmax = hdb->cdmax; a.cd32 = hdb->cd32; a.cd64 = hdb->cd64; }
    a.frontier_cap = (int)fcap;
    a.rec = rec; a.box = box; a.dp = dp;
    a.list_count = lcount;
    a.big = lists[3]; a.big_count = lcount + 3;
    a.huge_best = huge_best; a.huge_sbest = huge_sbest;
    a.stack = dual_stack; a.stack_cap = T.depth + 4;
    a.overflow = ovf;
    a.stat = stat;
    a.rho_bits = rho;
    // no node lists: the collecting traversal starts from every internal node
    a.node_in = nullptr; a.node_in_n = nullptr;
    a.node_out = nullptr; a.node_out_n = nullptr;
    Timer tw;
    // ---- the full WSPD: every well-separated pair into S[0]
    WM_TRY(launch_comp_labels(T, P, uf, rec, comp_scratch, ar, st));
    set_rho(a, 0.0, INFINITY);
    a.collect_all = 1;
    a.list[0] = S[0]; a.list_lb[0] = Slb[0]; a.list_cap[0] = (int)scap;
    for (int c = 1; c < 5; ++c) { a.list[c] = lists[c]; a.list_lb[c] = list_lbs[c]; a.list_cap[c] = (int)lcap; }
    traversal_init(1, a, stack, tcnt, st);
    for (int steps = 0;; steps += 3) {
        for (int b = 0; b < 3; ++b) traversal_step(1, a, stack, xbuf, tcnt, steps + b, chunk, st);
        WM_CK(cudaMemcpyAsync(C.pin, cnts, 8 * sizeof(int), cudaMemcpyDeviceToHost, st));
        WM_CK(cudaMemcpyAsync(C.pin + 8, ovf, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
        WM_CK(cudaMemcpyAsync(C.pin + 16, tcnt, kTravCounters * sizeof(int), cudaMemcpyDeviceToHost, st));
        WM_CK(cudaStreamSynchronize(st));
        if (C.pin[8]) { *overflow_bits = (unsigned)C.pin[8]; return 0; }
        if (C.pin[16] == 0 && C.pin[17] == 0 && C.pin[18] == 0) break;
        if (steps > 10000000) { set_detail("WSPD traversal did not terminate%s", ""); return WM_EINTERNAL; }
        C.stats.getpairs_launches += 3;
    }
    int mS = C.pin[2];
    C.stats.wspd_pairs = mS;
    a.collect_all = 0;
    for (int c = 0; c < 5; ++c) { a.list[c] = lists[c]; a.list_lb[c] = list_lbs[c]; a.list_cap[c] = (int)lcap; }
    WM_CK(cudaMemsetAsync(cnts + 2, 0, 8 * sizeof(int), st));
    C.stats.ms_wspd += tw.ms();
    int cur = 0, pcur = 0, mP = 0, nE = 0, rounds = 0;
    long long bccp_pairs = 0;   // pairs whose BCCP was computed (each once)
    long long beta = naive ? (1LL << 62) : 2;
    double rho_lo = 0.0;
    while (nE < target) {
        if (++rounds > 4096) { set_detail("GFK made no progress%s (%lld rounds)", "", rounds); return WM_EINTERNAL; }
        Timer tb;
        // ---- BCCP of the pairs of at most beta points, in segments of the class lists' capacity;
        // every edge is emitted (range [0, +inf)) into the pool
        set_rho(a, 0.0, INFINITY);
        a.edges = pool[pcur]; a.edge_count = pcount; a.edge_cap = (int)scap;
        WM_CK(cudaMemsetAsync(kcount, 0, sizeof(int), st));
        for (long long off = 0; off < mS; off += lcap) {
            const int seg = (int)std::min<long long>(lcap, mS - off);
            WM_CK(cudaMemsetAsync(lcount, 0, 5 * sizeof(int), st));
            gfk_split(a, S[cur] + off, Slb[cur] + off, seg, beta, S[cur ^ 1], Slb[cur ^ 1], kcount, st);
            WM_CK(cudaMemcpyAsync(C.pin, lcount, 5 * sizeof(int), cudaMemcpyDeviceToHost, st));
            WM_CK(cudaStreamSynchronize(st));
            int lc[5] = {C.pin[0], C.pin[1], C.pin[2], C.pin[3], C.pin[4]};
            for (int c = 0; c < 5; ++c) bccp_pairs += lc[c];
            run_bccp_groups(a, lc, st);
            run_bccp_tiles(a, lc, cnts + 16, st, hdb != nullptr, a.fp64 != 0);
            WM_TRY(run_bccp_huge(a, a.list[4], a.list_lb[4], lc[4], huge_items, (long long *)(cnts + 12), st, ar,
                                 hdb != nullptr, a.fp64 != 0, stack_warps));
        }
        WM_CK(cudaMemcpyAsync(C.pin, cnts, 10 * sizeof(int), cudaMemcpyDeviceToHost, st));
        WM_CK(cudaMemcpyAsync(C.pin + 16, ovf, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
        WM_CK(cudaStreamSynchronize(st));
        if (C.pin[16]) { *overflow_bits = (unsigned)C.pin[16]; return 0; }
        mP = C.pin[7];
        mS = C.pin[8];
        cur ^= 1;
        C.stats.ms_bccp += tb.ms();
        // ---- rho_hi: the smallest lower bound of the pairs left (+inf when none is left)
        gfk_min_lb(Slb[cur], mS, rho, st);
        WM_CK(cudaMemcpyAsync(C.pin, rho, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
        WM_CK(cudaStreamSynchronize(st));
        float rf;
        memcpy(&rf, C.pin, sizeof rf);
        const double rho_hi = std::max<double>(rf, rho_lo);
        // ---- the pool's edges below rho_hi form the round's batch
        WM_CK(cudaMemsetAsync(bcount, 0, sizeof(int), st));
        WM_CK(cudaMemsetAsync(pcount, 0, sizeof(int), st));
        gfk_partition(pool[pcur], mP, rho_hi, batch, bcount, (int)scap, pool[pcur ^ 1], pcount, ovf, st);
        pcur ^= 1;
        if (hdb && hdb->nrep > 0 && rho_hi > rho_lo)
            launch(take_range_kernel, grid_for(hdb->nrep, 256), 256, 0, st, hdb->rep, hdb->nrep, rho_lo, rho_hi, batch,
                   bcount, (int)scap, ovf);
        WM_CK(cudaMemcpyAsync(C.pin, cnts, 10 * sizeof(int), cudaMemcpyDeviceToHost, st));
        WM_CK(cudaMemcpyAsync(C.pin + 16, ovf, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
        WM_CK(cudaStreamSynchronize(st));
        if (C.pin[16]) { *overflow_bits = (unsigned)C.pin[16]; return 0; }
        const int m = C.pin[9];
        mP = C.pin[7];
        Timer tk;
        int accepted = 0;
        if (m > 0) {
            C.stats.candidate_edges += m;
            WM_TRY(batch_kruskal(batch, m, n, uf, R, E_out, nE, &accepted, ar, st, C.pin));
        }
        C.stats.ms_kruskal += tk.ms();
        nE += accepted;
        if (nE >= target) break;
        if (!(rho_hi < INFINITY) && mS == 0 && mP == 0) {
            set_detail("GFK ran out of pairs before the tree was complete%s (%lld edges)", "", nE);
            return WM_EINTERNAL;
        }
        // ---- filter: pairs whose points are all connected, pool edges whose endpoints are
        WM_TRY(launch_comp_labels(T, P, uf, rec, comp_scratch, ar, st));
        WM_CK(cudaMemsetAsync(kcount, 0, sizeof(int), st));
        gfk_filter_pairs(S[cur], Slb[cur], mS, rec, S[cur ^ 1], Slb[cur ^ 1], kcount, st);
        WM_CK(cudaMemsetAsync(pcount, 0, sizeof(int), st));
        gfk_filter_edges(pool[pcur], mP, uf, pool[pcur ^ 1], pcount, st);
        WM_CK(cudaMemcpyAsync(C.pin, cnts, 10 * sizeof(int), cudaMemcpyDeviceToHost, st));
        WM_CK(cudaStreamSynchronize(st));
        mS = C.pin[8];
        mP = C.pin[7];
        cur ^= 1;
        pcur ^= 1;
        rho_lo = rho_hi;
        beta *= 2;
    }
    {
        Timer ts;
        EdgeK *sorted = E_out;
        WM_TRY(radix_sort_edges(E_out, tmp, (int)target, st, ar, &sorted, C.pin + 4096));
        if (sorted != E_out) WM_CK(cudaMemcpyAsync(E_out, sorted, sizeof(EdgeK) * target, cudaMemcpyDeviceToDevice, st));
        WM_CK(cudaStreamSynchronize(st));
        C.stats.ms_kruskal += ts.ms();
    }
    WM_CK(cudaMemcpyAsync(C.pin, stat, 16 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    WM_CK(cudaStreamSynchronize(st));
    unsigned long long hs[16];
    memcpy(hs, C.pin, sizeof hs);
    C.stats.rounds = rounds;
    C.stats.getpairs_visits = (int64_t)hs[4];
    C.stats.pairs_retrieved = bccp_pairs;
    C.stats.bccp_evals = (int64_t)hs[1];
    C.stats.fp64_rechecks += (int64_t)hs[2];
    C.stats.bccp_tile_evals = (int64_t)hs[3];
    C.stats.bccp_dual_evals = (int64_t)hs[6];
    ar.off = mark;
    return 0;
}

// ---------------------------------------------------------------------- shared front half
struct Prepared {
    Points P;
    Tree T;
};

static int prepare(Call &C, const void *pts, int64_t n, int32_t d, int32_t dtype, int32_t layout, Prepared &S)
{
    cudaStream_t st = C.st;
    const void *dsrc = pts;
    size_t bytes = (size_t)n * d * (dtype == WM_F32 ? 4 : 8);
    if (!is_device_ptr(pts)) {
        void *buf = C.ar.take(bytes);
        if (!buf) return WM_ENOMEM;
        WM_CK(cudaMemcpyAsync(buf, pts, bytes, cudaMemcpyHostToDevice, st));
        dsrc = buf;
    }
    Timer ti;
    int rc = ingest_points(dsrc, (int)n, d, dtype, layout, S.P, C.ar, st, (unsigned *)C.pin);
    if (rc == WM_EINVAL) { set_detail("non-finite coordinate or |coordinate| > 2^60%s", ""); return rc; }
    if (rc) return rc;
    C.stats.ms_ingest = ti.ms();
    Timer tt;
    WM_TRY(build_tree(S.P, S.T, C.ar, st, C.pin, C.tune.tight_diameters != 0));
    C.stats.ms_build_tree = tt.ms();
    C.stats.tree_nodes = S.T.N;
    C.stats.tree_depth = S.T.depth;
    return 0;
}

static int write_edges(Call &C, const EdgeK *E, int m, wm_edge *out, double *total)
{
    cudaStream_t st = C.st;
    if (m > 0 && out) {
        bool dev = is_device_ptr(out);
        wm_edge *dst = out;
        if (!dev) {
            dst = C.ar.get<wm_edge>(m);
            if (!dst) return WM_ENOMEM;
        }
        launch(to_wm_edge_kernel, grid_for(m, 256), 256, 0, st, E, m, dst);
        if (!dev) WM_CK(cudaMemcpyAsync(out, dst, sizeof(wm_edge) * m, cudaMemcpyDeviceToHost, st));
    }
    if (total) {
        double *part = C.ar.get<double>(256 + 1);
        if (!part) return WM_ENOMEM;
        if (m > 0) {
            int g = grid_for(m, 256, 256);
            launch(sum_sqrt_kernel, g, 256, 0, st, E, m, part);
            launch(sum_partials_kernel, 1, 256, 0, st, part, g, part + 256);
            WM_CK(cudaMemcpyAsync(C.pin, part + 256, sizeof(double), cudaMemcpyDeviceToHost, st));
        } else {
            double z = 0.0;
            memcpy(C.pin, &z, sizeof z);
        }
    }
    WM_CK(cudaStreamSynchronize(st));
    if (total) memcpy(total, C.pin, sizeof(double));
    return 0;
}

// ------------------------------------------------------------------------ the call driver
typedef int (*Body)(Call &C, void *ctx, const Caps &caps, unsigned *overflow);

static int run_call(const wm_opts *opts, long long n, int d, int min_pts, Body body, void *ctx,
                    long long extra_bytes = 0)
{
    g_detail.clear();
    Timer total;
    int dev = 0;
    WM_CK(cudaGetDevice(&dev));
    Call C;
    C.st = opts ? (cudaStream_t)opts->stream : nullptr;
    C.precision = opts ? opts->precision : WM_PREC_FP32_SCREEN;
    if (C.precision != WM_PREC_FP32_SCREEN && C.precision != WM_PREC_FP64) {
        set_detail("bad precision%s %lld", "", C.precision);
        return WM_EINVAL;
    }
    {
        const int m = opts ? opts->method : WM_METHOD_MEMOGFK;
        C.method = m & 0xff;
        C.disjunctive = (m & WM_SEPARATION_GEOMETRIC) ? 0 : 1;
        if (C.method > WM_METHOD_NAIVE || (m & ~(0xff | WM_SEPARATION_GEOMETRIC))) {
            set_detail("bad method%s %lld", "", m);
            return WM_EINVAL;
        }
    }
    C.pin = pinned_scratch();
    if (!C.pin) { set_detail("cudaMallocHost failed%s", ""); return WM_ENOMEM; }
    Caps caps = caps_for(n, d, min_pts);
    caps.extra_bytes = extra_bytes;
    if (C.method == WM_METHOD_GFK || C.method == WM_METHOD_NAIVE) caps.wspd_pairs = wspd_pairs_guess(n, d);
    C.tune = tuning_for(n, d, min_pts);
    const bool user_ws = opts && opts->workspace;
    int rc = 0;
    unsigned ovf_seen = 0;   // capacities that overflowed in earlier attempts
    for (int attempt = 0; attempt < 8; ++attempt) {
        size_t need = estimate_bytes(n, d, min_pts, caps);
        std::unique_lock<std::mutex> lk;
        if (user_ws) {
            C.ar.base = (char *)opts->workspace;
            C.ar.cap = opts->workspace_bytes;
        } else {
            DevCache &dc = g_cache[dev & 63];
            lk = std::unique_lock<std::mutex>(dc.mu);
            if (dc.cap < need) {
                if (dc.ptr) { cudaStreamSynchronize(C.st); cudaFree(dc.ptr); dc.ptr = nullptr; dc.cap = 0; }
                if (cudaMalloc((void **)&dc.ptr, need) != cudaSuccess) {
                    cudaGetLastError();
                    char what[96];
                    snprintf(what, sizeof what, "%s%s%s", (ovf_seen & 1u) ? " frontier" : "",
                             (ovf_seen & 2u) ? " edge-batch" : "", (ovf_seen & 4u) ? " pair-list" : "");
                    set_detail("cudaMalloc of %lld bytes failed (capacities grown after overflow of:%s)",
                               (long long)need, ovf_seen ? what : " none");
                    return WM_ENOMEM;
                }
                dc.cap = need;
            }
            C.ar.base = dc.ptr;
            C.ar.cap = dc.cap;
        }
        C.ar.off = 0;
        C.ar.peak = 0;
        C.ar.failed = false;
        C.stats = wm_stats{};
        unsigned ovf = 0;
        rc = body(C, ctx, caps, &ovf);
        if (rc == 0 && C.ar.failed) rc = WM_ENOMEM;
        if (rc == WM_ENOMEM && !user_ws && !C.ar.failed) break;
        if (rc == WM_ENOMEM && !user_ws && C.ar.failed) {
            // the arena estimate was short (deep tree, many repair edges): grow it and retry
            caps.extra_bytes += std::max<long long>(256LL << 20, (long long)(need / 2));
            continue;
        }
        if (rc == 0 && (ovf & 8u)) {
            set_detail("a BCCP traversal stack overflowed (internal error)%s", "");
            rc = WM_EINTERNAL;
            break;
        }
        if (rc == 0 && ovf == 0) break;
        if (rc == WM_ENOMEM && user_ws) {
            set_detail("caller workspace too small%s (%lld bytes given)", "", (long long)C.ar.cap);
            break;
        }
        if (rc && rc != WM_ENOMEM) break;
        ovf_seen |= ovf;
        // grow whichever capacity overflowed and start over
        if (ovf & 1u) caps.frontier_scale *= 2;
        if (ovf & 2u) caps.edges = std::min(kMaxEdgeCap, caps.edges * 2);
        if ((ovf & 6u) && caps.wspd_pairs) caps.wspd_pairs *= 2;   // the materialised WSPD or its pool
        if (user_ws && ovf && estimate_bytes(n, d, min_pts, caps) > opts->workspace_bytes) {
            rc = WM_ENOMEM;
            set_detail("caller workspace too small: this input needs about %lld bytes%s",
                       (long long)estimate_bytes(n, d, min_pts, caps), "");
            break;
        }
        rc = WM_ENOMEM;
    }
    cudaError_t le = cudaGetLastError();
    if (rc == 0 && le != cudaSuccess) {
        set_detail("CUDA error %s%lld", cudaGetErrorString(le), 0);
        rc = WM_ECUDA;
    }
    C.stats.workspace_bytes_used = C.ar.peak;
    C.stats.ms_total = total.ms();
    if (opts && opts->stats) *opts->stats = C.stats;
    return rc;
}

// ------------------------------------------------------------------------------ bodies
struct EmstCtx {
    const void *pts;
    long long n;
    int d, dtype, layout;
    wm_edge *out;
    double *total;
};

static int emst_body(Call &C, void *vctx, const Caps &caps, unsigned *ovf)
{
    EmstCtx &x = *(EmstCtx *)vctx;
    Prepared S;
    WM_TRY(prepare(C, x.pts, x.n, x.d, x.dtype, x.layout, S));
    const int n = (int)x.n;
    int *uf = C.ar.get<int>(n);
    unsigned long long *R = C.ar.get<unsigned long long>(4LL * n);
    EdgeK *E = C.ar.get<EdgeK>(n);
    if (C.ar.failed) return WM_ENOMEM;
    launch(init_uf_kernel, grid_for(n, 256), 256, 0, C.st, uf, R, n);
    if (C.method == WM_METHOD_GFK || C.method == WM_METHOD_NAIVE)
        WM_TRY(gfk_rounds(C, S.P, S.T, nullptr, caps, E, uf, R, ovf, C.method == WM_METHOD_NAIVE));
    else
        WM_TRY(memogfk(C, S.P, S.T, nullptr, caps, E, uf, R, ovf));
    if (*ovf) return 0;
    return write_edges(C, E, n - 1, x.out, x.total);
}

struct HdbCtx {
    const void *pts;
    long long n;
    int d, dtype, layout, min_pts, start;
    wm_edge *mst;
    double *cd;
    wm_dnode *dendro;
    int *order;
    double *reach;
};

static int hdbscan_body(Call &C, void *vctx, const Caps &caps, unsigned *ovf)
{
    HdbCtx &x = *(HdbCtx *)vctx;
    Prepared S;
    WM_TRY(prepare(C, x.pts, x.n, x.d, x.dtype, x.layout, S));
    const int n = (int)x.n;
    HdbState H;
    Timer tc;
    WM_TRY(core_distances(S.P, S.T, x.min_pts, C.precision == WM_PREC_FP64, H, C.ar, C.st, C.pin, &C.stats));
    C.stats.ms_core_dist = tc.ms();
    int *uf = C.ar.get<int>(n);
    unsigned long long *R = C.ar.get<unsigned long long>(4LL * n);
    EdgeK *E = C.ar.get<EdgeK>(n);
    if (C.ar.failed) return WM_ENOMEM;
    launch(init_uf_kernel, grid_for(n, 256), 256, 0, C.st, uf, R, n);
    if (C.method == WM_METHOD_GFK || C.method == WM_METHOD_NAIVE)
        WM_TRY(gfk_rounds(C, S.P, S.T, &H, caps, E, uf, R, ovf, C.method == WM_METHOD_NAIVE));
    else
        WM_TRY(memogfk(C, S.P, S.T, &H, caps, E, uf, R, ovf));
    if (*ovf) return 0;
    WM_TRY(write_core_distances(S.P, H, x.cd, C.ar, C.st));
    WM_TRY(write_edges(C, E, n - 1, x.mst, nullptr));
    Timer td;
    WM_TRY(dendrogram(E, n, x.start, x.dendro, x.order, x.reach, C.ar, C.st, C.pin));
    C.stats.ms_dendrogram = td.ms();
    return 0;
}

struct SlCtx {
    const wm_edge *tree;
    long long n;
    int start;
    wm_dnode *dendro;
    int *order;
    double *reach;
};

static int sl_body(Call &C, void *vctx, const Caps &, unsigned *ovf)
{
    SlCtx &x = *(SlCtx *)vctx;
    *ovf = 0;
    const int n = (int)x.n;
    EdgeK *E = C.ar.get<EdgeK>(n), *tmp = C.ar.get<EdgeK>(n);
    if (C.ar.failed) return WM_ENOMEM;
    if (n > 1) {
        const wm_edge *src = x.tree;
        if (!is_device_ptr(src)) {
            wm_edge *b = C.ar.get<wm_edge>(n - 1);
            if (!b) return WM_ENOMEM;
            WM_CK(cudaMemcpyAsync(b, src, sizeof(wm_edge) * (n - 1), cudaMemcpyHostToDevice, C.st));
            src = b;
        }
        int *bad = C.ar.get<int>(1);
        if (!bad) return WM_ENOMEM;
        WM_TRY(edges_from_wm(src, n, E, bad, C.st));
        EdgeK *sorted = E;
        WM_TRY(radix_sort_edges(E, tmp, n - 1, C.st, C.ar, &sorted, C.pin + 4096));
        WM_CK(cudaMemcpyAsync(C.pin, bad, sizeof(int), cudaMemcpyDeviceToHost, C.st));
        WM_CK(cudaStreamSynchronize(C.st));
        if (C.pin[0]) { set_detail("tree edge with an endpoint outside [0, n) or a bad weight%s", ""); return WM_EINVAL; }
        Timer td;
        WM_TRY(dendrogram_impl(sorted, n, x.start, 0, x.dendro, x.order, x.reach, C.ar, C.st, C.pin));
        C.stats.ms_dendrogram = td.ms();
    } else {
        WM_TRY(dendrogram_impl(E, n, x.start, 0, x.dendro, x.order, x.reach, C.ar, C.st, C.pin));
    }
    return 0;
}

// ------------------------------------------------------------------------------ batches
// Instances of one group (same d, same minPts) solved as one point set; see batch.cu.
struct BatchCtx {
    const wm_instance *inst;
    const std::vector<int> *idx;
    int d, min_pts, dtype, layout;
};

// copy stage[off[j], off[j+1]) to every instance's output dst[j]: device outputs by one kernel,
// host outputs through one device-to-host copy of the whole stage
template <typename T>
static int scatter_outputs(Call &C, const T *stage, const std::vector<long long> &off, const long long *off_d,
                           const std::vector<T *> &dst)
{
    const int k = (int)dst.size();
    const long long cnt = off[k];
    std::vector<T *> dev(k, nullptr);
    bool any_host = false, any_dev = false;
    for (int j = 0; j < k; ++j) {
        if (!dst[j] || off[j + 1] == off[j]) continue;
        if (is_device_ptr(dst[j])) { dev[j] = dst[j]; any_dev = true; }
        else any_host = true;
    }
    if (any_dev) {
        T **dt = (T **)C.ar.take(sizeof(T *) * k);
        if (!dt) return WM_ENOMEM;
        WM_CK(cudaMemcpyAsync(dt, dev.data(), sizeof(T *) * k, cudaMemcpyHostToDevice, C.st));
        batch_scatter<T>(stage, cnt, off_d, k, dt, C.st);
    }
    if (any_host && cnt > 0) {
        std::vector<T> h((size_t)cnt);
        WM_CK(cudaMemcpyAsync(h.data(), stage, sizeof(T) * cnt, cudaMemcpyDeviceToHost, C.st));
        WM_CK(cudaStreamSynchronize(C.st));
        for (int j = 0; j < k; ++j)
            if (dst[j] && !dev[j] && off[j + 1] > off[j])
                memcpy(dst[j], h.data() + off[j], sizeof(T) * (off[j + 1] - off[j]));
    }
    return 0;
}

static int batch_body(Call &C, void *vctx, const Caps &caps, unsigned *ovf)
{
    BatchCtx &x = *(BatchCtx *)vctx;
    cudaStream_t st = C.st;
    Arena &ar = C.ar;
    *ovf = 0;
    const std::vector<int> &idx = *x.idx;
    const int k = (int)idx.size();
    const int d = x.d, D = d + 1;
    const bool hdb = x.min_pts >= 2;
    auto I = [&](int j) -> const wm_instance & { return x.inst[idx[j]]; };
    std::vector<long long> base(k + 1, 0), eoff(k + 1, 0);
    for (int j = 0; j < k; ++j) base[j + 1] = base[j] + I(j).n;
    for (int j = 0; j <= k; ++j) eoff[j] = base[j] - j;   // tree edges of the instances before j
    const long long total = base[k];
    const int n = (int)total;
    const long long m = total - k;
    // ---- inputs: device pointers as given, host ones packed into one device buffer
    const size_t esz = x.dtype == WM_F32 ? 4 : 8;
    std::vector<const void *> src(k);
    std::vector<char> on_dev(k);
    size_t host_bytes = 0;
    std::vector<int> dims(k);
    for (int j = 0; j < k; ++j) {
        dims[j] = I(j).d;
        on_dev[j] = is_device_ptr(I(j).pts);
        if (!on_dev[j]) host_bytes += (size_t)I(j).n * I(j).d * esz;
        else src[j] = I(j).pts;
    }
    if (host_bytes) {
        char *hb = (char *)ar.take(host_bytes);
        if (!hb) return WM_ENOMEM;
        std::vector<char> pack(host_bytes);
        size_t off = 0;
        for (int j = 0; j < k; ++j) {
            if (on_dev[j]) continue;
            const size_t b = (size_t)I(j).n * I(j).d * esz;
            memcpy(pack.data() + off, I(j).pts, b);
            src[j] = hb + off;
            off += b;
        }
        WM_CK(cudaMemcpyAsync(hb, pack.data(), host_bytes, cudaMemcpyHostToDevice, st));
        WM_CK(cudaStreamSynchronize(st));
    }
    long long *base_d = ar.get<long long>(k + 1), *eoff_d = ar.get<long long>(k + 1);
    int *dims_d = ar.get<int>(k);
    const void **src_d = (const void **)ar.take(sizeof(void *) * k);
    unsigned *maxabs = ar.get<unsigned>(1);
    int *bad = ar.get<int>(1);
    double *raw = ar.get<double>((size_t)total * D);
    if (ar.failed || !src_d) return WM_ENOMEM;
    WM_CK(cudaMemcpyAsync(base_d, base.data(), sizeof(long long) * (k + 1), cudaMemcpyHostToDevice, st));
    WM_CK(cudaMemcpyAsync(eoff_d, eoff.data(), sizeof(long long) * (k + 1), cudaMemcpyHostToDevice, st));
    WM_CK(cudaMemcpyAsync(src_d, src.data(), sizeof(void *) * k, cudaMemcpyHostToDevice, st));
    WM_CK(cudaMemcpyAsync(dims_d, dims.data(), sizeof(int) * k, cudaMemcpyHostToDevice, st));
    WM_CK(cudaMemsetAsync(maxabs, 0, sizeof(unsigned), st));
    WM_CK(cudaMemsetAsync(bad, 0, sizeof(int), st));
    batch_gather(src_d, dims_d, base_d, k, total, d, x.dtype, x.layout, raw, maxabs, st);
    WM_CK(cudaMemcpyAsync(C.pin, maxabs, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    WM_CK(cudaStreamSynchronize(st));
    float mabs;
    memcpy(&mabs, C.pin, sizeof mabs);
    if (!(mabs <= 1.2e18f)) { set_detail("non-finite coordinate or |coordinate| > 2^60%s", ""); return WM_EINVAL; }
    // separation L: a power of two with L^2 / 4 above every squared distance inside an instance
    // (at most d (2 max|x|)^2), so the cap rho_cap = L^2 / 4 sits between the two kinds of pairs
    double L = 1.0;
    const double need = 4.0 * std::sqrt((double)D) * (double)mabs * (1.0 + 1e-6);
    while (L <= need) L *= 2.0;
    batch_scale(raw + (size_t)d * total, total, L, st);
    // ---- the joint problem
    Prepared S;
    WM_TRY(prepare(C, raw, total, D, WM_F64, WM_SOA, S));
    HdbState H;
    if (hdb) {
        Timer tc;
        WM_TRY(core_distances(S.P, S.T, x.min_pts, C.precision == WM_PREC_FP64, H, ar, st, C.pin, &C.stats));
        C.stats.ms_core_dist = tc.ms();
    }
    int *uf = ar.get<int>(n);
    unsigned long long *R = ar.get<unsigned long long>(4LL * n);
    EdgeK *E = ar.get<EdgeK>(n);
    if (ar.failed) return WM_ENOMEM;
    launch(init_uf_kernel, grid_for(n, 256), 256, 0, st, uf, R, n);
    WM_TRY(memogfk(C, S.P, S.T, hdb ? &H : nullptr, caps, E, uf, R, ovf, m, L * L / 4));
    if (*ovf) return 0;
    // ---- tree edges grouped by instance, K order inside each
    EdgeK *keys = ar.get<EdgeK>(m + 1), *ktmp = ar.get<EdgeK>(m + 1);
    int *local = ar.get<int>(m + 1);
    wm_edge *se = ar.get<wm_edge>(m + 1);
    if (ar.failed) return WM_ENOMEM;
    batch_edge_inst(E, (int)m, base_d, k, keys, st);
    EdgeK *grouped = keys;
    WM_TRY(radix_sort_edges(keys, ktmp, (int)m, st, ar, &grouped, C.pin + 4096));
    batch_edge_place(grouped, E, (int)m, base_d, local, se, bad, st);
    {
        std::vector<wm_edge *> dst(k);
        for (int j = 0; j < k; ++j) dst[j] = I(j).out_edges;
        WM_TRY(scatter_outputs<wm_edge>(C, se, eoff, eoff_d, dst));
    }
    if (!hdb) {
        double *tot = ar.get<double>(k);
        if (!tot) return WM_ENOMEM;
        batch_totals(se, base_d, k, tot, st);
        std::vector<double> ht(k);
        WM_CK(cudaMemcpyAsync(ht.data(), tot, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
        WM_CK(cudaStreamSynchronize(st));
        for (int j = 0; j < k; ++j)
            if (I(j).out_total_weight) *I(j).out_total_weight = ht[j];
    } else {
        double *scd = ar.get<double>(n);
        if (!scd) return WM_ENOMEM;
        batch_cd(H.cd64, S.P.pid, n, scd, st);
        {
            std::vector<double *> dst(k);
            for (int j = 0; j < k; ++j) dst[j] = I(j).out_core_dist;
            WM_TRY(scatter_outputs<double>(C, scd, base, base_d, dst));
        }
        bool want = false;
        for (int j = 0; j < k; ++j) want = want || I(j).out_dendro || I(j).out_order || I(j).out_reach;
        if (want) {
            Timer td;
            // the instances chained by bridges between consecutive start points
            std::vector<int> starts(k);
            for (int j = 0; j < k; ++j) starts[j] = (int)(base[j] + I(j).start);
            int *starts_d = ar.get<int>(k);
            EdgeK *Eall = ar.get<EdgeK>(n);
            wm_dnode *jd = ar.get<wm_dnode>(n), *sd = ar.get<wm_dnode>(m + 1);
            int *jo = ar.get<int>(n), *so = ar.get<int>(n);
            double *jr = ar.get<double>(n), *sr = ar.get<double>(n);
            if (ar.failed) return WM_ENOMEM;
            WM_CK(cudaMemcpyAsync(starts_d, starts.data(), sizeof(int) * k, cudaMemcpyHostToDevice, st));
            if (m > 0) WM_CK(cudaMemcpyAsync(Eall, E, sizeof(EdgeK) * m, cudaMemcpyDeviceToDevice, st));
            batch_bridges(starts_d, k, Eall + m, st);
            WM_TRY(dendrogram_impl(Eall, n, starts[0], 1, jd, jo, jr, ar, st, C.pin));
            batch_dendro(jd, E, (int)m, total, base_d, k, local, sd, bad, st);
            batch_order(jo, jr, total, base_d, k, so, sr, bad, st);
            std::vector<wm_dnode *> dd(k);
            std::vector<int *> od(k);
            std::vector<double *> rd(k);
            for (int j = 0; j < k; ++j) { dd[j] = I(j).out_dendro; od[j] = I(j).out_order; rd[j] = I(j).out_reach; }
            WM_TRY(scatter_outputs<wm_dnode>(C, sd, eoff, eoff_d, dd));
            WM_TRY(scatter_outputs<int>(C, so, base, base_d, od));
            WM_TRY(scatter_outputs<double>(C, sr, base, base_d, rd));
            C.stats.ms_dendrogram = td.ms();
        }
    }
    WM_CK(cudaMemcpyAsync(C.pin, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    WM_CK(cudaStreamSynchronize(st));
    if (C.pin[0]) {
        set_detail("batch: an output crossed two instances%s (flags %lld)", "", C.pin[0]);
        return WM_EINTERNAL;
    }
    return 0;
}

}  // namespace wm

// =========================================================================== C ABI
using namespace wm;

extern "C" {

int wm_emst(const void *pts, int64_t n, int32_t d, int32_t dtype, int32_t layout, wm_edge *out_edges,
            double *out_total_weight, const wm_opts *opts)
{
    g_detail.clear();
    if (!pts || n < 1 || n > 0x3fffffff || d < 1 || d > kMaxDim || (dtype != WM_F32 && dtype != WM_F64) ||
        (layout != WM_AOS && layout != WM_SOA) || (n > 1 && !out_edges && !out_total_weight)) {
        set_detail("invalid argument to wm_emst%s (n=%lld)", "", (long long)n);
        return WM_EINVAL;
    }
    EmstCtx c{pts, n, d, dtype, layout, out_edges, out_total_weight};
    return run_call(opts, n, d, 0, emst_body, &c);
}

int wm_hdbscan(const void *pts, int64_t n, int32_t d, int32_t dtype, int32_t layout, int32_t min_pts, wm_edge *out_mst,
               double *out_core_dist, wm_dnode *out_dendro, int32_t *out_order, double *out_reach, int32_t start,
               const wm_opts *opts)
{
    g_detail.clear();
    if (!pts || n < 1 || n > 0x3fffffff || d < 1 || d > kMaxDim || (dtype != WM_F32 && dtype != WM_F64) ||
        (layout != WM_AOS && layout != WM_SOA) || min_pts < 1 || min_pts > n || start < 0 || start >= n) {
        set_detail("invalid argument to wm_hdbscan%s (n=%lld)", "", (long long)n);
        return WM_EINVAL;
    }
    HdbCtx c{pts, n, d, dtype, layout, min_pts, start, out_mst, out_core_dist, out_dendro, out_order, out_reach};
    return run_call(opts, n, d, min_pts, hdbscan_body, &c);
}

int wm_single_linkage(const wm_edge *tree, int64_t n, int32_t start, wm_dnode *out_dendro, int32_t *out_order,
                      double *out_reach, const wm_opts *opts)
{
    g_detail.clear();
    if (n < 1 || n > 0x3fffffff || start < 0 || start >= n || (n > 1 && !tree)) {
        set_detail("invalid argument to wm_single_linkage%s (n=%lld)", "", (long long)n);
        return WM_EINVAL;
    }
    SlCtx c{tree, n, start, out_dendro, out_order, out_reach};
    return run_call(opts, n, 1, 1, sl_body, &c);
}

int wm_batch(const wm_instance *inst, int32_t count, int32_t dtype, int32_t layout, const wm_opts *opts)
{
    g_detail.clear();
    if (!inst || count < 1 || (dtype != WM_F32 && dtype != WM_F64) || (layout != WM_AOS && layout != WM_SOA)) {
        set_detail("invalid argument to wm_batch%s (count=%lld)", "", (long long)count);
        return WM_EINVAL;
    }
    // groups of equal minPts class (EMST instances form the class minPts <= 1); within a class,
    // the instances of one dimension form a group of their own when they hold at least
    // kBatchSplit points, the rest share one group in the dimension of its largest instance
    // (fewer groups, fewer rounds; at scale, the narrower arithmetic of one dimension wins)
    std::vector<std::pair<long long, int>> keyed;
    for (int i = 0; i < count; ++i) {
        const wm_instance &q = inst[i];
        const int mp = q.min_pts <= 1 ? 1 : q.min_pts;
        if (!q.pts || q.n < 1 || q.n > 0x3fffffff || q.d < 1 || q.d > kMaxDim - 1 || q.min_pts < 0 ||
            (mp > 1 && (mp > q.n || mp > 256 || q.start < 0 || q.start >= q.n))) {
            set_detail("wm_batch: invalid instance %s%lld", "", (long long)i);
            return WM_EINVAL;
        }
        keyed.push_back({(long long)mp * 64 + q.d, i});
    }
    {
        const long long kBatchSplit = 1 << 20;
        std::unordered_map<long long, long long> pts;
        for (auto &e : keyed) pts[e.first] += inst[e.second].n;
        for (auto &e : keyed)
            if (pts[e.first] < kBatchSplit) e.first = e.first / 64 * 64;   // merged: dimension 0 marks it
    }
    std::stable_sort(keyed.begin(), keyed.end(),
                     [](const std::pair<long long, int> &a, const std::pair<long long, int> &b) { return a.first < b.first; });
    // the groups (a run of one key, cut where it would exceed 2^30 points)
    std::vector<std::vector<int>> groups;
    for (size_t a = 0; a < keyed.size();) {
        size_t b = a;
        long long ptotal = 0;
        std::vector<int> part;
        while (b < keyed.size() && keyed[b].first == keyed[a].first) {
            const int i = keyed[b].second;
            if (!part.empty() && ptotal + inst[i].n > 0x3fffffff) {
                groups.push_back(part);
                part.clear();
                ptotal = 0;
            }
            part.push_back(i);
            ptotal += inst[i].n;
            ++b;
        }
        if (!part.empty()) groups.push_back(part);
        a = b;
    }
    struct GroupRun {
        int rc = WM_OK;
        wm_stats st{};
        std::string detail;
    };
    std::vector<GroupRun> res(groups.size());
    auto group_args = [&](size_t g, long long &ptotal, int &d, int &mp) {
        ptotal = 0;
        d = 0;
        for (int i : groups[g]) { ptotal += inst[i].n; d = std::max(d, (int)inst[i].d); }
        mp = inst[groups[g][0]].min_pts <= 1 ? 1 : inst[groups[g][0]].min_pts;
    };
    const bool caller_ws = opts && opts->workspace;
    const int kBatchThreads = 4;
    if (groups.size() == 1 || caller_ws) {
        for (size_t g = 0; g < groups.size(); ++g) {
            long long ptotal;
            int d, mp;
            group_args(g, ptotal, d, mp);
            BatchCtx c{inst, &groups[g], d, mp, dtype, layout};
            wm_opts o = opts ? *opts : wm_opts{};
            o.stats = &res[g].st;
            const long long extra = ptotal * (8LL * (d + 1) + 200) + (long long)groups[g].size() * 64;
            res[g].rc = run_call(&o, ptotal, d + 1, mp > 1 ? mp : 0, batch_body, &c, extra);
            res[g].detail = g_detail;
            if (res[g].rc) break;
        }
    } else {
        // groups run concurrently, each on a stream of its own with a workspace from the device's
        // stream-ordered pool; the streams wait for the caller's stream first
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return WM_ECUDA;
        cudaStream_t caller = opts ? (cudaStream_t)opts->stream : nullptr;
        cudaEvent_t ready;
        if (cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) != cudaSuccess) return WM_ECUDA;
        cudaEventRecord(ready, caller);
        cudaMemPool_t pool = batch_pool(dev);
        std::atomic<size_t> next{0};
        std::atomic<bool> failed{false};
        auto worker = [&]() {
            cudaSetDevice(dev);
            cudaStream_t st = nullptr;
            if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) { failed = true; return; }
            cudaStreamWaitEvent(st, ready, 0);
            for (size_t g; !failed && (g = next.fetch_add(1)) < groups.size();) {
                long long ptotal;
                int d, mp;
                group_args(g, ptotal, d, mp);
                BatchCtx c{inst, &groups[g], d, mp, dtype, layout};
                const long long extra = ptotal * (8LL * (d + 1) + 200) + (long long)groups[g].size() * 64;
                Caps cp = caps_for(ptotal, d + 1, mp > 1 ? mp : 0);
                cp.extra_bytes = extra;
                size_t bytes = estimate_bytes(ptotal, d + 1, mp > 1 ? mp : 0, cp);
                int rc = WM_ENOMEM;
                for (int attempt = 0; attempt < 4; ++attempt) {
                    void *ws = nullptr;
                    if (!pool || cudaMallocFromPoolAsync(&ws, bytes, pool, st) != cudaSuccess) {
                        cudaGetLastError();
                        set_detail("workspace of %s%lld bytes could not be allocated", "", (long long)bytes);
                        rc = WM_ENOMEM;
                        break;
                    }
                    wm_opts o = opts ? *opts : wm_opts{};
                    o.stream = st;
                    o.workspace = ws;
                    o.workspace_bytes = bytes;
                    o.stats = &res[g].st;
                    rc = run_call(&o, ptotal, d + 1, mp > 1 ? mp : 0, batch_body, &c, extra);
                    cudaFreeAsync(ws, st);
                    cudaStreamSynchronize(st);
                    if (rc != WM_ENOMEM) break;
                    bytes *= 2;   // the data needed more than the estimate
                }
                res[g].rc = rc;
                res[g].detail = g_detail;
                if (rc) failed = true;
            }
            cudaStreamDestroy(st);
        };
        std::vector<std::thread> threads;
        const int nt = (int)std::min<size_t>(kBatchThreads, groups.size());
        for (int t = 0; t < nt; ++t) threads.emplace_back(worker);
        for (auto &t : threads) t.join();
        cudaEventDestroy(ready);
    }
    wm_stats sum{};
    int rc = WM_OK;
    for (size_t g = 0; g < groups.size(); ++g) {
        const wm_stats &gs = res[g].st;
        if (rc == WM_OK && res[g].rc != WM_OK) {
            rc = res[g].rc;
            g_detail = res[g].detail;
        }
        sum.ms_total += gs.ms_total; sum.ms_ingest += gs.ms_ingest; sum.ms_build_tree += gs.ms_build_tree;
        sum.ms_core_dist += gs.ms_core_dist; sum.ms_wspd += gs.ms_wspd; sum.ms_bccp += gs.ms_bccp;
        sum.ms_kruskal += gs.ms_kruskal; sum.ms_dendrogram += gs.ms_dendrogram; sum.rounds += gs.rounds;
        sum.pairs_retrieved += gs.pairs_retrieved; sum.bccp_evals += gs.bccp_evals;
        sum.bccp_tile_evals += gs.bccp_tile_evals; sum.knn_evals += gs.knn_evals;
        sum.fp64_rechecks += gs.fp64_rechecks; sum.candidate_edges += gs.candidate_edges;
        sum.tree_nodes += gs.tree_nodes; sum.tree_depth = std::max(sum.tree_depth, gs.tree_depth);
        sum.workspace_bytes_used = std::max(sum.workspace_bytes_used, gs.workspace_bytes_used);
        sum.getpairs_visits += gs.getpairs_visits; sum.getrho_visits += gs.getrho_visits;
        sum.getpairs_launches += gs.getpairs_launches; sum.bccp_dual_evals += gs.bccp_dual_evals;
        sum.rho_shrinks += gs.rho_shrinks; sum.tile_launches += gs.tile_launches;
        sum.edge_batch_grown = std::max(sum.edge_batch_grown, gs.edge_batch_grown);
        sum.tie_overflow = std::max(sum.tie_overflow, gs.tie_overflow);
        sum.ms_knn_kernel += gs.ms_knn_kernel; sum.ms_tile_kernel += gs.ms_tile_kernel;
        sum.wspd_pairs += gs.wspd_pairs; sum.ms_getrho += gs.ms_getrho; sum.ms_bccp_group += gs.ms_bccp_group; sum.ms_bccp_dual += gs.ms_bccp_dual;
        sum.ms_getpairs += gs.ms_getpairs;
        sum.max_pending_pairs = std::max(sum.max_pending_pairs, gs.max_pending_pairs);
        sum.bccp_pairs_below += gs.bccp_pairs_below; sum.bccp_pairs_above += gs.bccp_pairs_above;
        sum.bccp_evals_outside += gs.bccp_evals_outside;
        sum.bccp_tile_evals_skipped += gs.bccp_tile_evals_skipped;
        sum.max_rel_screen_err = std::max(sum.max_rel_screen_err, gs.max_rel_screen_err);
    }
    if (opts && opts->stats) *opts->stats = sum;
    return rc;
}

int wm_get_tuning(int64_t n, int32_t d, int32_t min_pts, wm_tuning *out)
{
    if (!out || n < 0 || d < 1 || d > kMaxDim || min_pts < 0) return WM_EINVAL;
    if (n == 0) {   // the built-in defaults, before any table row or override
        wm_tuning t{};
        builtin_tuning(0, d, min_pts, &t);
        *out = t;
        return WM_OK;
    }
    *out = tuning_for(n, d, min_pts);
    return WM_OK;
}

int wm_set_tuning(const wm_tuning *t)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (!t) {
        g_tune_set = false;
        return WM_OK;
    }
    if (!tuning_valid(*t)) return WM_EINVAL;
    g_tune_override = *t;
    g_tune_set = true;
    return WM_OK;
}

int wm_query_footprint(int64_t n, int32_t d, int32_t min_pts, size_t *bytes)
{
    if (!bytes || n < 1 || d < 1 || d > kMaxDim || min_pts < 0) return WM_EINVAL;
    *bytes = estimate_bytes(n, d, min_pts, caps_for(n, d, min_pts));
    return WM_OK;
}

int wm_release_cache(void)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return WM_ECUDA;
    DevCache &dc = g_cache[dev & 63];
    std::lock_guard<std::mutex> lk(dc.mu);
    if (dc.ptr) {
        cudaDeviceSynchronize();
        cudaFree(dc.ptr);
    }
    dc.ptr = nullptr;
    dc.cap = 0;
    BatchPool &bp = g_batch_pool[dev & 63];
    std::lock_guard<std::mutex> lk2(bp.mu);
    if (bp.pool) {
        cudaDeviceSynchronize();
        cudaMemPoolTrimTo(bp.pool, 0);
    }
    return WM_OK;
}

const char *wm_strerror(int code)
{
    switch (code) {
    case WM_OK: return "success";
    case WM_EINVAL: return "invalid argument";
    case WM_ENOMEM: return "out of device memory or workspace";
    case WM_ETIMEOUT: return "a bounded device wait gave up";
    case WM_ECUDA: return "CUDA runtime error";
    case WM_EINTERNAL: return "internal consistency check failed";
    default: return "unknown error code";
    }
}

const char *wm_last_error_detail(void) { return g_detail.c_str(); }

int64_t wm_kernel_launch_count(void) { return (int64_t)g_launch_count.load(); }

int wm_fp32_fma_peak(double *tflops, double *ms)
{
    if (!tflops) return WM_EINVAL;
    g_detail.clear();
    const int blocks = num_sms() * 8, threads = 256, iters = 1 << 13;
    float *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    WM_CK(cudaMalloc((void **)&out, sizeof(float) * blocks));
    int rc = WM_OK;
    float best = 1e30f;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = WM_ECUDA;
    for (int rep = 0; rc == WM_OK && rep < 6; ++rep) {   // the first run warms up
        cudaEventRecord(e0, nullptr);
        launch(ffma_probe_kernel, blocks, threads, 0, nullptr, out, iters, 0.999999f, 1e-7f);
        cudaEventRecord(e1, nullptr);
        if (cudaEventSynchronize(e1) != cudaSuccess) { rc = WM_ECUDA; break; }
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        if (rep > 0) best = std::min(best, t);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (rc != WM_OK) {
        set_detail("FMA probe failed: %s%lld", cudaGetErrorString(cudaGetLastError()), 0);
        return rc;
    }
    const double flops = 2.0 * 8 * 4 * (double)iters * blocks * threads;
    *tflops = flops / (best * 1e-3) / 1e12;
    if (ms) *ms = best;
    return WM_OK;
}

const char *wm_version(void) { return "wspdmst 0.1 (sm_103a)"; }

}  // extern "C"

// =========================================================== no-allocation EMST entry point
// Device scratch for wm_emst_noalloc: one file-scope array per device, sized for
// WM_NOALLOC_MAX_POINTS points of up to 16 dimensions.  Host code must not use the symbol
// itself as a device address: its device address is looked up once per device below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[WM_NOALLOC_SCRATCH_BYTES];

namespace wm {

struct NoAllocDevice {
    std::mutex mu;
    void *scratch = nullptr;   // device address of g_noalloc_scratch on this device
};
static NoAllocDevice g_noalloc_dev[64];

// host-side readback buffer of the no-allocation path (ordinary host memory, one per thread)
static thread_local int g_noalloc_host[16384];

}  // namespace wm

extern "C" int wm_emst_noalloc(const void *pts, int64_t n, int32_t d, int32_t dtype, int32_t layout,
                               wm_edge *out_edges, double *out_total_weight, const wm_opts *opts)
{
    using namespace wm;
    g_detail.clear();
    if (!pts || n < 1 || d < 1 || d > kMaxDim || (dtype != WM_F32 && dtype != WM_F64) ||
        (layout != WM_AOS && layout != WM_SOA) || (n > 1 && !out_edges && !out_total_weight)) {
        set_detail("invalid argument to wm_emst_noalloc%s (n=%lld)", "", (long long)n);
        return WM_EINVAL;
    }
    if (n > WM_NOALLOC_MAX_POINTS) {
        set_detail("wm_emst_noalloc: n = %s%lld exceeds WM_NOALLOC_MAX_POINTS (32768); use wm_emst", "",
                   (long long)n);
        return WM_EINVAL;
    }
    const int precision = opts ? opts->precision : WM_PREC_FP32_SCREEN;
    if (precision != WM_PREC_FP32_SCREEN && precision != WM_PREC_FP64) {
        set_detail("bad precision%s %lld", "", precision);
        return WM_EINVAL;
    }
    Timer total;
    int dev = 0;
    WM_CK(cudaGetDevice(&dev));
    NoAllocDevice &nd = g_noalloc_dev[dev & 63];
    std::lock_guard<std::mutex> lk(nd.mu);
    if (!nd.scratch) {
        // once per device, with that device current
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_detail("wm_emst_noalloc: cudaGetSymbolAddress failed: %s%lld", cudaGetErrorString(e), 0);
            return WM_ECUDA;
        }
        nd.scratch = p;
    }
    Call C;
    C.st = opts ? (cudaStream_t)opts->stream : nullptr;
    C.precision = precision;
    C.timing = false;
    C.pin = g_noalloc_host;
    C.tune = tuning_for(n, d, 0);
    C.ar.base = (char *)nd.scratch;
    C.ar.cap = WM_NOALLOC_SCRATCH_BYTES;
    // Capacities sized for WM_NOALLOC_MAX_POINTS: traversal chunks of 4096 pairs and edge batches of
    // 4n + 65536; WSPD stack and pair lists follow from the chunk (see memogfk).  A capacity that
    // overflows is doubled and the call restarts, as wm_emst does, for as long as the array holds
    // the larger buffers.
    Caps caps;
    caps.chunk = 4096;
    caps.edges = 4 * n + 65536;
    caps.frontier_scale = 1;
    caps.extra_bytes = 0;
    EmstCtx c{pts, n, d, dtype, layout, out_edges, out_total_weight};
    int rc = 0;
    unsigned ovf = 0;
    size_t peak = 0;
    for (int attempt = 0; attempt < 6; ++attempt) {
        C.ar.off = 0;
        C.ar.peak = 0;
        C.ar.failed = false;
        C.stats = wm_stats{};
        ovf = 0;
        rc = emst_body(C, &c, caps, &ovf);
        // On every path (success, overflow, out of scratch, CUDA error) the GPU work of this attempt
        // must have finished before the array is reused by the next attempt or, once the lock is
        // released, by another call.
        const cudaError_t se = cudaStreamSynchronize(C.st);
        peak = std::max(peak, C.ar.peak);
        if (rc == 0 && se != cudaSuccess) {
            set_detail("CUDA error %s%lld", cudaGetErrorString(se), 0);
            rc = WM_ECUDA;
        }
        if (rc == 0 && C.ar.failed) rc = WM_ENOMEM;
        if (rc == WM_ENOMEM) {
            set_detail("wm_emst_noalloc: this input needs more than the %s%lld-byte static scratch; use wm_emst", "",
                       (long long)WM_NOALLOC_SCRATCH_BYTES);
            break;
        }
        if (rc == 0 && (ovf & 8u)) {
            set_detail("a BCCP traversal stack overflowed (internal error)%s", "");
            rc = WM_EINTERNAL;
        }
        if (rc != 0 || ovf == 0) break;
        if (ovf & 1u) caps.frontier_scale *= 2;
        if (ovf & 2u) caps.edges = std::min(kMaxEdgeCap, caps.edges * 2);
    }
    if (rc == 0 && ovf) {
        rc = WM_ENOMEM;
        set_detail("wm_emst_noalloc: the pair traversal or the edge batch still overflowed after %s%lld restarts "
                   "with doubled capacities; use wm_emst", "", 5LL);
    }
    cudaError_t le = cudaGetLastError();
    if (rc == 0 && le != cudaSuccess) {
        set_detail("CUDA error %s%lld", cudaGetErrorString(le), 0);
        rc = WM_ECUDA;
    }
    C.ar.peak = peak;
    C.stats.workspace_bytes_used = C.ar.peak;
    C.stats.ms_total = total.ms();
    if (opts && opts->stats) *opts->stats = C.stats;
    return rc;
}

// ======================================================================== serving loop
namespace wm {

struct ServerJob {
    wm_job spec;
    int64_t ticket = 0;
    int status = WM_JOB_QUEUED;
    size_t footprint = 0;
    std::chrono::steady_clock::time_point t_submit, t_done;
};

}  // namespace wm

struct wm_server {
    int device = 0;
    size_t budget = 0;
    size_t in_use = 0, peak = 0;
    int running = 0, peak_running = 0;
    int64_t finished = 0;
    int64_t next_ticket = 1;
    bool stop = false;
    std::mutex mu;
    std::condition_variable cv_work, cv_mem, cv_done;
    std::deque<wm::ServerJob *> queue;
    std::unordered_map<int64_t, wm::ServerJob *> jobs;
    std::vector<std::thread> threads;
    cudaMemPool_t pool = nullptr;
};

namespace wm {

static size_t job_footprint(const wm_job &j)
{
    size_t b = 0;
    wm_query_footprint(j.n, j.d, j.kind == WM_JOB_HDBSCAN ? j.min_pts : 0, &b);
    return b;
}

static int run_job(const wm_job &j, void *ws, size_t ws_bytes, cudaStream_t st)
{
    wm_opts o{};
    o.stream = st;
    o.precision = j.precision;
    o.workspace = ws;
    o.workspace_bytes = ws_bytes;
    if (j.kind == WM_JOB_EMST)
        return wm_emst(j.pts, j.n, j.d, j.dtype, j.layout, j.out_edges, j.out_total_weight, &o);
    return wm_hdbscan(j.pts, j.n, j.d, j.dtype, j.layout, j.min_pts, j.out_edges, j.out_core_dist, j.out_dendro,
                      j.out_order, j.out_reach, j.start, &o);
}

static void server_worker(wm_server *s)
{
    cudaSetDevice(s->device);
    cudaStream_t st = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    while (true) {
        ServerJob *job = nullptr;
        size_t fp = 0;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] { return s->stop || !s->queue.empty(); });
            if (s->queue.empty()) break;   // stop requested and nothing left
            job = s->queue.front();
            s->queue.pop_front();
            fp = job->footprint;
            // admission: wait until the job's workspace fits in the budget
            s->cv_mem.wait(lk, [&] { return s->in_use + fp <= s->budget; });
            s->in_use += fp;
            s->peak = std::max(s->peak, s->in_use);
            s->running += 1;
            s->peak_running = std::max(s->peak_running, s->running);
            job->status = WM_JOB_RUNNING;
        }
        int rc = WM_ENOMEM;
        for (int attempt = 0; attempt < 4; ++attempt) {
            void *ws = nullptr;
            if (cudaMallocFromPoolAsync(&ws, fp, s->pool, st) != cudaSuccess) {
                cudaGetLastError();
                rc = WM_ENOMEM;
                break;
            }
            rc = run_job(job->spec, ws, fp, st);
            cudaFreeAsync(ws, st);
            cudaStreamSynchronize(st);
            if (rc != WM_ENOMEM) break;
            // the data needed more workspace than estimated: grow within the budget and rerun
            std::unique_lock<std::mutex> lk(s->mu);
            size_t more = fp;
            if (fp + more > s->budget) break;
            s->cv_mem.wait(lk, [&] { return s->in_use + more <= s->budget; });
            s->in_use += more;
            s->peak = std::max(s->peak, s->in_use);
            fp += more;
        }
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->in_use -= fp;
            s->running -= 1;
            s->finished += 1;
            job->t_done = std::chrono::steady_clock::now();
            job->status = rc;
        }
        s->cv_mem.notify_all();
        s->cv_done.notify_all();
    }
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
}

}  // namespace wm

extern "C" {

int wm_server_create(int32_t device, size_t hbm_budget_bytes, int32_t workers, wm_server **out)
{
    using namespace wm;
    if (!out || workers < 1 || workers > 64 || hbm_budget_bytes == 0) return WM_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return WM_EINVAL;
    wm_server *s = new wm_server();
    s->device = device;
    s->budget = hbm_budget_bytes;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(device);
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    if (cudaMemPoolCreate(&s->pool, &props) != cudaSuccess) {
        cudaGetLastError();
        cudaSetDevice(prev);
        delete s;
        return WM_ECUDA;
    }
    uint64_t keep = hbm_budget_bytes;   // keep up to the budget cached in the pool between jobs
    cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    cudaSetDevice(prev);
    for (int i = 0; i < workers; ++i) s->threads.emplace_back(server_worker, s);
    *out = s;
    return WM_OK;
}

int wm_server_destroy(wm_server *s)
{
    if (!s) return WM_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto &t : s->threads) t.join();
    for (auto &kv : s->jobs) delete kv.second;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(s->device);
    cudaMemPoolDestroy(s->pool);
    cudaSetDevice(prev);
    delete s;
    return WM_OK;
}

int wm_submit(wm_server *s, const wm_job *job, int64_t *ticket)
{
    using namespace wm;
    if (!s || !job || !ticket || !job->pts || job->n < 1 || job->d < 1 || job->d > kMaxDim ||
        (job->kind != WM_JOB_EMST && job->kind != WM_JOB_HDBSCAN) ||
        (job->kind == WM_JOB_HDBSCAN && (job->min_pts < 1 || job->min_pts > job->n)))
        return WM_EINVAL;
    ServerJob *j = new ServerJob();
    j->spec = *job;
    j->footprint = job_footprint(*job);
    if (j->footprint > s->budget) {
        delete j;
        return WM_ENOMEM;   // admission rejection: can never fit the budget
    }
    j->t_submit = std::chrono::steady_clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        j->ticket = s->next_ticket++;
        s->jobs[j->ticket] = j;
        s->queue.push_back(j);
        *ticket = j->ticket;
    }
    s->cv_work.notify_one();
    return WM_OK;
}

int wm_poll(wm_server *s, int64_t ticket, int32_t *status, double *latency_ms)
{
    if (!s || !status) return WM_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return WM_EINVAL;
    *status = it->second->status;
    if (latency_ms) {
        *latency_ms = (it->second->status <= 0)
                          ? std::chrono::duration<double, std::milli>(it->second->t_done - it->second->t_submit).count()
                          : -1.0;
    }
    return WM_OK;
}

int wm_wait(wm_server *s, int64_t ticket, double *latency_ms)
{
    if (!s) return WM_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return WM_EINVAL;
    wm::ServerJob *j = it->second;
    s->cv_done.wait(lk, [&] { return j->status <= 0; });
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(j->t_done - j->t_submit).count();
    return j->status;
}

int wm_server_counters(wm_server *s, int64_t *finished, size_t *peak_bytes, int32_t *peak_running)
{
    if (!s) return WM_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (finished) *finished = s->finished;
    if (peak_bytes) *peak_bytes = s->peak;
    if (peak_running) *peak_running = s->peak_running;
    return WM_OK;
}

}  // extern "C"
