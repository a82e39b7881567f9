// wspd.cu -- the lazily traversed well-separated pair decomposition of MemoGFK (Sec. 3.2.1,
// Algorithm 1; Sec. 3.2.3, Algorithm 3) and the BCCP / BCCP* computations (Sec. 2.3, 3.2.2, 3.1.2).
//
// Per round the host runs, with the union-find state of the previous rounds:
//   comp labels  : every node gets the component id shared by all its points, or -1 (mixed);
//   GetRho       : a pruned breadth-first FindPair traversal that WriteMins, over well-separated
//                  unconnected pairs with |A|+|B| > beta, a lower bound of their BCCP;
//   GetPairs     : a second traversal retrieving the well-separated unconnected pairs whose BCCP
//                  can lie in [rho_lo, rho_hi); small pairs get their BCCP evaluated in place,
//                  larger ones are queued for the tile kernel;
//   BCCP tiles   : FP32 distance screen over A x B in warp tiles, then FP64 re-evaluation of every
//                  candidate inside the rigorous error band of the screened minimum, and the
//                  K-minimum edge is emitted when its FP64 w2 lies in [rho_lo, rho_hi).
//
// Recursion-free form: each traversal keeps a stack of pending node pairs in HBM; one kernel
// launch pops a chunk of it and every warp expands the pairs it takes depth first, on a stack of
// its own in shared memory, for a bounded number of rounds (see findpair_dfs_kernel).
//
// Well-separation tests use boxes (the nodes' bounding volumes).  Geometric separation is
// d(A,B) > max(diam A, diam B) with d and diam the box distance and box diagonal, made strict and
// rigorous so that every cross pair is strictly heavier than every pair inside A or inside B; for
// HDBSCAN* the disjunction with mutual unreachability (Sec. 3.1.2) is used.  Two single points
// always form a pair.
#include "wspd.cuh"

namespace wm {

namespace {

__device__ inline int nsize(const TravArgs &a, int x) { return a.end[x] - a.begin[x]; }

// threshold of the FP32 screen: any candidate whose screened value exceeds T cannot beat the
// screened minimum s once both are evaluated exactly in FP64.  With an exact FP32 copy (eta = 0)
// T = s (1 + 4 eps32) + 1.5e-42, bounded from above in FP32 with directed rounding (a float
// >= the exact value is >= its rounded-up value too); otherwise in FP64.
__device__ inline float screen_threshold(float s, const TravArgs &a)
{
    if (a.exact32) return __fadd_ru(__fmul_ru(s, 1.0f + 4.0f / 524288.0f), 1.6e-42f);
    const double eta = a.eta;
    double r = sqrt((double)s * (1.0 + 2.0 * kEps32)) + eta;
    double U = r * r * (1.0 + 2.0 * kGam64);
    double q = sqrt(U * (1.0 + 2.0 * kGam64)) + eta;
    return __double2float_ru(q * q * (1.0 + 2.0 * kEps32) + 1.5e-42);
}

// True when a screened value s proves that the exact FP64 weight of its point pair is at or above
// rho_hi, so that the pair's edge cannot belong to this round and needs no FP64 recheck: s is at
// least TravArgs::above_f, the smallest float whose rigorous lower bound on that weight reaches
// rho_hi (computed on the host, see above_threshold).
__device__ inline bool screened_above(float s, const TravArgs &a) { return s >= a.above_f; }

__device__ inline float dist32(const float *__restrict__ x32, int n, int d, int i, int j)
{
    float s = 0.f;
    for (int k = 0; k < d; ++k) {
        float t = x32[(size_t)k * n + i] - x32[(size_t)k * n + j];
        s = fmaf(t, t, s);
    }
    return s;
}

// dist32 with the dimension fixed at compile time (D > 0), the same operations in the same order
template <int D>
__device__ inline float dist32t(const float *__restrict__ x32, int n, int d, int i, int j)
{
    if (D <= 0) return dist32(x32, n, d, i, j);
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < (D > 0 ? D : 1); ++k) {
        float t = x32[(size_t)k * n + i] - x32[(size_t)k * n + j];
        s = fmaf(t, t, s);
    }
    return s;
}

// dist32 from the point-major copy: the same subtractions and fused multiply-adds in dimension
// order (a padded coordinate is 0 on both sides and adds exactly 0)
template <int D>
__device__ inline float dist32p(const float4 *__restrict__ x4, int i, int j)
{
    constexpr int Q = (D + 3) / 4;                          // float4s holding coordinates
    constexpr int S = Q <= 1 ? 1 : Q <= 2 ? 2 : 4;          // float4s per point (dp / 4)
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < Q; ++c) {
        const float4 p = x4[(size_t)i * S + c];
        const float4 q = x4[(size_t)j * S + c];
        const float pv[4] = {p.x, p.y, p.z, p.w}, qv[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            if (4 * c + r < D) {
                const float t = pv[r] - qv[r];
                s = fmaf(t, t, s);
            }
        }
    }
    return s;
}

__device__ inline double dist64(const double *__restrict__ x64, int n, int d, int i, int j)
{
    double s = 0.0;
    for (int k = 0; k < d; ++k) {
        double t = __dsub_rn(x64[(size_t)k * n + i], x64[(size_t)k * n + j]);
        s = __dadd_rn(s, __dmul_rn(t, t));
    }
    return s;
}

// max of two non-negative doubles through their bit patterns (integer compare, no FP64 op)
__device__ inline double pos_dmax(double x, double y)
{
    return __double_as_longlong(x) >= __double_as_longlong(y) ? x : y;
}

// exact FP64 weight of positions (i,j).  d32: the FP32 squared distance alone; c32: the larger
// FP32 core distance (HDBSCAN*).  When d32 is provably below the larger core distance (d32 is
// within 2^-19 of the true distance, a stored cd32 within 2^-24 of its FP64 value), the weight
// is that core distance and the FP64 distance is skipped.
__device__ inline double exact_w2(const TravArgs &a, int i, int j, float d32, float c32)
{
    if (a.cd64) {
        double c = pos_dmax(a.cd64[i], a.cd64[j]);
        if (a.exact32 && d32 * (1.0f + 1.0f / 131072.0f) < c32 * (1.0f - 1.0f / 4194304.0f)) return c;
        return pos_dmax(c, dist64(a.x64, a.n, a.d, i, j));
    }
    return dist64(a.x64, a.n, a.d, i, j);
}

// exact_w2, also noting the relative error of the FP32 screened value (sd, or for HDBSCAN* its
// maximum with the FP32 core distances c32) against the exact weight in err
__device__ inline double checked_w2(const TravArgs &a, int i, int j, float sd, float c32, float &err)
{
    const double w = exact_w2(a, i, j, sd, c32);
    if (w > 0.0) {   // the ratio in FP32 with outward rounding (a single FP64 subtraction)
        const double sv = a.cd64 ? pos_dmax((double)sd, (double)c32) : (double)sd;
        err = fmaxf(err, __fdiv_ru(__double2float_ru(fabs(sv - w)), __double2float_rd(w)));
    }
    return w;
}

// the largest relative screen error of a warp into stat[12] (bits of a non-negative float)
__device__ inline void err_flush(const TravArgs &a, float err)
{
    for (int o = 16; o; o >>= 1) err = fmaxf(err, __shfl_xor_sync(0xffffffffu, err, o));
    if ((threadIdx.x & 31) == 0 && err > 0.f) atomicMax(a.stat + 12, (unsigned long long)__float_as_uint(err));
}

// a recheck candidate held back so that the FP64 work of several lanes runs in one instruction
struct Deferred {
    int i = -1, j = 0;
    float sd = 0.f, c32 = 0.f;
};

__device__ inline float screen_value(const Deferred &c, bool hdb) { return hdb ? fmaxf(c.sd, c.c32) : c.sd; }

struct KMin {
    unsigned long long hi, lo;   // w2 bits, (min id << 32) | max id
};
__device__ inline void kmin_update(KMin &m, double w2, int pu, int pv)
{
    unsigned long long h = (unsigned long long)__double_as_longlong(w2);
    unsigned a = (unsigned)min(pu, pv), b = (unsigned)max(pu, pv);
    unsigned long long l = ((unsigned long long)a << 32) | b;
    if (h < m.hi || (h == m.hi && l < m.lo)) { m.hi = h; m.lo = l; }
}

// warp-aggregated append of `cnt` items (0..2) per lane; returns this lane's first slot
__device__ inline int warp_append(int *counter, int cnt)
{
    const int lane = threadIdx.x & 31;
    int x = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    int total = __shfl_sync(0xffffffffu, x, 31);
    int base = 0;
    if (lane == 31 && total) base = atomicAdd(counter, total);
    base = __shfl_sync(0xffffffffu, base, 31);
    return base + x - cnt;
}

__device__ inline bool in_range(const TravArgs &a, const KMin &m)
{
    // non-negative doubles (and +inf) order like their bit patterns
    return m.hi != ~0ull && m.hi >= (unsigned long long)__double_as_longlong(a.rho_lo) &&
           m.hi < (unsigned long long)__double_as_longlong(a.rho_hi);
}

// outcome of a BCCP against the round's range: -1 below rho_lo, 0 inside, 1 at or above rho_hi
__device__ inline int range_side(const TravArgs &a, const KMin &m)
{
    if (m.hi == ~0ull || m.hi >= (unsigned long long)__double_as_longlong(a.rho_hi)) return 1;
    return m.hi < (unsigned long long)__double_as_longlong(a.rho_lo) ? -1 : 0;
}

// per-thread tallies of BCCP outcomes outside the round's range (stat[8..10])
struct Waste {
    unsigned long long below = 0, above = 0, ev = 0;
    __device__ void add(int side, unsigned long long evals)
    {
        if (side < 0) ++below;
        if (side > 0) ++above;
        if (side != 0) ev += evals;
    }
};

__device__ inline unsigned long long warp_sum_u64(unsigned long long v)
{
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ inline void waste_flush(const TravArgs &a, Waste w)
{
    w.below = warp_sum_u64(w.below);
    w.above = warp_sum_u64(w.above);
    w.ev = warp_sum_u64(w.ev);
    if ((threadIdx.x & 31) == 0 && (w.below | w.above)) {
        atomicAdd(a.stat + 8, w.below);
        atomicAdd(a.stat + 9, w.above);
        atomicAdd(a.stat + 10, w.ev);
    }
}

// warp-aggregated append of one edge per lane that has one
__device__ inline void warp_emit(const TravArgs &a, bool has, const KMin &m)
{
    int slot = warp_append(a.edge_count, has ? 1 : 0);
    if (has) {
        if (slot < a.edge_cap) {
            EdgeK e;
            e.hi = m.hi;
            e.lo = m.lo;
            a.edges[slot] = e;
        } else {
            atomicOr(a.overflow, 2u);
        }
    }
}


// ------------------------------------------------------------------ packed node records
// rec[node] = {l = {begin, end, left, comp label}, m = {diam2 bound, cdmin, cdmax, 0}} (the right
// child is always left + 1, and the label of the round is what a visit tests first, with the
// sizes); box[node][2*DP] holds the bounds in groups of four dimensions (box_lo / box_hi).  A visit
// reads each node's record and box with 256-bit loads, 1 + DP / 4 of them per node.
__device__ inline void box_terms(const float4 &plo, const float4 &phi, const float4 &qlo, const float4 &qhi, float &s,
                                 float &t)
{
    const float al[4] = {plo.x, plo.y, plo.z, plo.w}, ah[4] = {phi.x, phi.y, phi.z, phi.w};
    const float bl[4] = {qlo.x, qlo.y, qlo.z, qlo.w}, bh[4] = {qhi.x, qhi.y, qhi.z, qhi.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float g = fmaxf(fmaxf(bl[k] - ah[k], al[k] - bh[k]), 0.f);
        float m = fmaxf(bh[k] - al[k], ah[k] - bl[k]);
        s = fmaf(g, g, s);
        t = fmaf(m, m, t);
    }
}

// g0 = the first four-dimension group of both boxes {P lo, P hi, Q lo, Q hi}, loaded by the caller
// together with the records so that the two loads overlap
template <int DP>
__device__ inline void pair_bounds_packed(const TravArgs &a, int P, int Q, const int4 &lp, const int4 &lq,
                                          const float4 &mp, const float4 &mq, const float4 (&g0)[4], float &lbB,
                                          float &ubB, bool &ws, float &dP, float &dQ)
{
    const float *bp = a.box + (size_t)P * 2 * DP;
    const float *bq = a.box + (size_t)Q * 2 * DP;
    float s = 0.f, t = 0.f;   // squared gap and squared extent, dimension by dimension in order
    box_terms(g0[0], g0[1], g0[2], g0[3], s, t);
#pragma unroll
    for (int c = 1; c < DP / 4; ++c) {
        float4 plo, phi, qlo, qhi;
        ldg256(bp + 8 * c, plo, phi);
        ldg256(bq + 8 * c, qlo, qhi);
        box_terms(plo, phi, qlo, qhi, s, t);
    }
    float lb = lower_w2(s), ub = upper_w2(t);
    dP = mp.x;
    dQ = mq.x;
    float dm = fmaxf(dP, dQ);
    ws = lb > dm;
    lbB = lb;
    ubB = ub;
    if (a.cdmin) {
        float lhs = fmaxf(lb, fmaxf(mp.y, mq.y));
        float rhs = fmaxf(dm, fmaxf(mp.z, mq.z));
        if (a.disjunctive) ws = ws || lhs >= rhs;   // or mutually unreachable (Sec. 3.1.2)
        lbB = lhs;
        ubB = fmaxf(ub, fmaxf(mp.z, mq.z));
    }
    if (lp.z < 0 && lq.z < 0) ws = true;   // two single points
}

// pair-size classes of a retrieved well-separated pair (by |A||B|)
constexpr int kTinyMax = 8;      // one thread per pair
constexpr int kSmallMax = 64;    // 8 lanes per pair
// (larger pairs: one warp per pair up to TravArgs::medium_max, warp tiles (brute force) up to
// big_max, the pruned dual-tree BCCP above)

// One FindPair visit of the node pair me (Algorithm 1's recursion body).  MODE 0 = GetRho
// (WriteMin candidates into rho_cand, pruned by rho_now), MODE 1 = GetPairs (classifies a
// retrieved pair into cls), MODE 2 = both in one pass: rho_now is the running GetRho minimum R,
// a well-separated pair of more than beta points lowers it, and a smaller one is retrieved when
// its lower bound is below R (R only falls, so every pair GetPairs would take with the final R is
// taken, plus some the final R excludes, whose edges the host drops).  Sets push = 2 with the
// two child pairs when the pair is split.
template <int MODE, int DP>
__device__ inline void visit_pair(const TravArgs &a, int2 me, float rho_now, int &push, int2 &c0, int2 &c1, int &cls,
                                  float &rho_cand, float &lb_out)
{
    const int P = me.x, Q = me.y;
    // the records and the first box group of both nodes in one round trip (a pair that the
    // checks below reject has read its box group for nothing; the overlap pays for that)
    float4 g0[4];
    ldg256(a.box + (size_t)P * 2 * DP, g0[0], g0[1]);
    ldg256(a.box + (size_t)Q * 2 * DP, g0[2], g0[3]);
    int4 lp, lq;
    float4 mp, mq;
    load_rec(a.rec, P, lp, mp);
    load_rec(a.rec, Q, lq, mq);
    const int sp = lp.y - lp.x, sq = lq.y - lq.x;
    if (MODE == 0 && sp + sq <= a.beta) return;
    if (lp.w >= 0 && lp.w == lq.w) return;   // all points already connected
    float lbB, ubB, dP, dQ;
    bool ws;
    pair_bounds_packed<DP>(a, P, Q, lp, lq, mp, mq, g0, lbB, ubB, ws, dP, dQ);
    // (double)x >= r  <=>  x >= (smallest float >= r), for a float x; likewise for <
    if (MODE == 0) {
        // pairs whose BCCP is certainly below rho_lo were handled by earlier rounds
        if (lbB >= rho_now || ubB < a.rho_lo_f) return;
        if (ws) { rho_cand = fminf(rho_cand, lbB); return; }
    } else if (MODE == 2) {
        if (lbB >= rho_now || ubB < a.rho_lo_f) return;
        if (ws) {
            if (sp + sq > a.beta) { rho_cand = fminf(rho_cand, lbB); return; }
            long long prod = (long long)sp * sq;
            cls = prod <= kTinyMax ? 0 : prod <= kSmallMax ? 1 : prod <= a.medium_max ? 2 : prod <= a.big_max ? 3 : 4;
            lb_out = lbB;
            return;
        }
    } else {
        if (lbB >= a.rho_hi_f || ubB < a.rho_lo_f) return;
        if (ws) {
            long long prod = (long long)sp * sq;
            cls = a.collect_all ? 0
                                : prod <= kTinyMax ? 0 : prod <= kSmallMax ? 1 : prod <= a.medium_max ? 2 : prod <= a.big_max ? 3 : 4;
            lb_out = lbB;
            return;
        }
    }
    // split the node with the larger diameter (a leaf cannot be split)
    const bool splitP = lp.z >= 0 && (lq.z < 0 || dP >= dQ);
    const int O = splitP ? Q : P;
    c0 = make_int2(splitP ? lp.z : lq.z, O);
    c1 = make_int2((splitP ? lp.z : lq.z) + 1, O);
    push = 2;
}

// One traversal step.  The pending pairs form a logical stack: the global stack S[0, top) with the
// previous step's output xin[0, xin_count) on top of it.  The step pops the top min(size, chunk)
// pairs; warps take them 32 at a time and visit each (breadth first over the popped pairs), keeping
// the children on a stack of their own in shared memory (spilled to the step output xout when it
// is full); when the popped pairs are exhausted, every warp expands its own stack depth first for
// at most `budget` rounds and then writes what is left to xout.  Pairs of xin beyond one chunk are
// moved onto S.  The last block to finish sets the new stack size and clears the counters it owns.
template <int MODE, int DP>
__global__ void __launch_bounds__(256) findpair_dfs_kernel(TravArgs a, DfsArgs s)
{
    __shared__ int2 wst[kDfsWarpsPerBlock][kDfsWarpCap];
    // GetPairs: retrieved pairs gathered per warp and size class, reserved in the global lists 32
    // at a time
    __shared__ int2 rbuf[MODE != 0 ? kDfsWarpsPerBlock : 1][5][32];
    __shared__ float rlb[MODE != 0 ? kDfsWarpsPerBlock : 1][5][32];   // their lower bounds
    const int lane = threadIdx.x & 31;
    int2 *ws = wst[threadIdx.x >> 5];
    int2 (*rb)[32] = rbuf[MODE != 0 ? threadIdx.x >> 5 : 0];
    float (*rl)[32] = rlb[MODE != 0 ? threadIdx.x >> 5 : 0];
    int rcnt[5] = {0, 0, 0, 0, 0};   // warp-uniform fill of each class buffer
    // moves class c's buffer to its global list
    auto flush_class = [&](int c) {
        int base = 0;
        if (lane == 0) base = atomicAdd(a.list_count + c, rcnt[c]);
        base = __shfl_sync(0xffffffffu, base, 0);
        for (int i = lane; i < rcnt[c]; i += 32) {
            if (base + i < a.list_cap[c]) {
                a.list[c][base + i] = rb[c][i];
                a.list_lb[c][base + i] = rl[c][i];
            } else {
                atomicOr(a.overflow, 4u);
            }
        }
        rcnt[c] = 0;
        __syncwarp();
    };
    // counts are clamped to the capacities, so that no access leaves the buffers even after an
    // overflow (the host then discards the traversal)
    const int tp = min(*s.top, a.frontier_cap), xc = min(*s.xin_count, s.xcap);
    const int mx = xc < s.chunk ? xc : s.chunk;   // pairs taken from xin (its top part)
    const int excess = xc - mx;                   // the rest of xin goes onto S
    const int ms = excess > 0 ? 0 : (tp < s.chunk - mx ? tp : s.chunk - mx);   // pairs taken from S
    const int m = mx + ms;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < excess; i += gridDim.x * blockDim.x) {
        if (tp + i < a.frontier_cap) s.S[tp + i] = s.xin[i];
        else atomicOr(a.overflow, 1u);
    }
    auto input = [&](int i) -> int2 { return i < mx ? s.xin[xc - mx + i] : s.S[tp - ms + (i - mx)]; };
    const bool stop = __shfl_sync(0xffffffffu, (int)(*(volatile unsigned *)a.overflow != 0), 0) != 0;
    unsigned n_vis = 0, n_ret = 0;   // per warp and launch: far below 2^32
    float rho_w = INFINITY;    // GetRho: smallest candidate this warp has written
    float rho_g = INFINITY;    // GetRho: the shared minimum as last read (refreshed every 4 rounds)
    int refresh = 0;
    int sp = 0, it = 0;        // warp stack size (warp-uniform), rounds on the warp's own stack
    bool fed = stop;           // no more input for this warp
    // every popped pair costs one visit in the breadth-first phase: a contiguous share per warp
    // (m <= chunk <= 2^24 and gw * share < m + nw: 32-bit arithmetic suffices)
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int share = (m + nw - 1) / nw;
    int in_next = gw * share;
    const int in_end = min(m, in_next + share);
    while (!stop) {
        // one round: the next 32 popped pairs while there are any (every popped pair is visited
        // in this step, breadth first), then up to `budget` rounds of the warp's own stack
        int2 me = make_int2(0, 0);
        int k = 0;
        bool from_input = false;
        if (!fed) {
            const int base = in_next;
            k = base < in_end ? min(32, in_end - base) : 0;
            if (k == 0) fed = true;
            else {
                from_input = true;
                in_next += 32;
                if (lane < k) me = input(base + lane);
            }
        }
        if (!from_input) {
            if (sp == 0 || it == s.budget) break;
            k = sp < 32 ? sp : 32;
            sp -= k;
            if (lane < k) me = ws[sp + lane];
            __syncwarp();
            ++it;
        }
        const bool has = lane < k;
        int push = 0, cls = -1;
        int2 c0 = make_int2(0, 0), c1 = c0;
        float rho_cand = INFINITY, lb = 0.f;
        // the shared GetRho minimum only prunes: a stale (larger) copy is safe, so it is read from
        // L2 every fourth round and this warp's own minimum is used in between
        if (MODE != 1 && (refresh++ & 3) == 0) rho_g = __uint_as_float(*(volatile unsigned *)a.rho_bits);
        if (has) {
            ++n_vis;
            float rho_now = 0.f;
            if (MODE != 1) rho_now = fminf(rho_g, rho_w);
            visit_pair<MODE, DP>(a, me, rho_now, push, c0, c1, cls, rho_cand, lb);
        }
        int x = push;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        const int total = __shfl_sync(0xffffffffu, x, 31);
        // children onto the warp stack while it has room, else into the step output
        if (sp + total <= kDfsWarpCap) {
            if (push) { ws[sp + x - 2] = c0; ws[sp + x - 1] = c1; }
            sp += total;
        } else {
            int base = 0;
            if (lane == 0) base = atomicAdd(s.xout_count, total);
            base = __shfl_sync(0xffffffffu, base, 0);
            if (push) {
                if (base + x <= s.xcap) { s.xout[base + x - 2] = c0; s.xout[base + x - 1] = c1; }
                else atomicOr(a.overflow, 1u);
            }
        }
        __syncwarp();
        if (MODE != 1) {
            for (int o = 16; o; o >>= 1) rho_cand = fminf(rho_cand, __shfl_xor_sync(0xffffffffu, rho_cand, o));
            if (rho_cand < rho_w) {
                rho_w = rho_cand;
                // non-negative floats order like their bit patterns
                if (lane == 0) atomicMin(a.rho_bits, __float_as_uint(rho_cand));
            }
        }
        if (MODE != 0) {
            if (__any_sync(0xffffffffu, cls >= 0)) {
#pragma unroll
                for (int c = 0; c < 5; ++c) {
                    const unsigned bal = __ballot_sync(0xffffffffu, cls == c);
                    const int nc = __popc(bal);
                    if (nc == 0) continue;
                    if (rcnt[c] + nc > 32) flush_class(c);
                    if (cls == c) {
                        ++n_ret;
                        rb[c][rcnt[c] + __popc(bal & lanemask_lt())] = me;
                        rl[c][rcnt[c] + __popc(bal & lanemask_lt())] = lb;
                    }
                    rcnt[c] += nc;
                }
                __syncwarp();
            }
        }
    }
    if (MODE != 0) {
#pragma unroll
        for (int c = 0; c < 5; ++c)
            if (rcnt[c] > 0) flush_class(c);
    }
    // what is left on the warp stack goes to the step output (every popped pair was visited)
    if (!stop && sp > 0) {
        int base = 0;
        if (lane == 0) base = atomicAdd(s.xout_count, sp);
        base = __shfl_sync(0xffffffffu, base, 0);
        for (int i = lane; i < sp; i += 32) {
            if (base + i < s.xcap) s.xout[base + i] = ws[i];
            else atomicOr(a.overflow, 1u);
        }
    }
    const unsigned long long t_vis = warp_sum_u64(n_vis), t_ret = warp_sum_u64(n_ret);
    if (lane == 0 && t_vis) {
        atomicAdd(a.stat + (MODE == 0 ? 5 : 4), t_vis);
        if (t_ret) atomicAdd(a.stat + 0, t_ret);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned t = atomicAdd(s.done, 1u);
        if (t == gridDim.x - 1) {
            const int nt = tp + excess - ms;
            *s.top = nt < a.frontier_cap ? nt : a.frontier_cap;
            atomicMax(a.stat + 7, (unsigned long long)nt + (unsigned long long)*(volatile int *)s.xout_count);
            *s.xin_count = 0;   // xin is the next step's output buffer
            *s.next = 0;
            *s.done = 0;
            __threadfence();
        }
    }
}

// ------------------------------------------------------------- BCCP of tiny/small/medium pairs
// A group of G lanes evaluates one pair: lane g takes the evaluations e = g, g+G, ... of the
// |A| x |B| product (a = e / |B|, b = e % |B|).  FP32 screen, group minimum, band threshold,
// FP64 recheck of every candidate inside the band, group K-minimum; the group leader emits the
// edge when its FP64 w2 lies in [rho_lo, rho_hi).
template <int G, int D>
__global__ void __launch_bounds__(256) bccp_group_kernel(TravArgs a, const int2 *__restrict__ pairs,
                                                         const float *__restrict__ lbs, const int *__restrict__ count)
{
    const int m = *count;
    const int lane = threadIdx.x & 31, g = lane & (G - 1);
    constexpr int PPW = 32 / G;   // pairs per warp
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
    const int n = a.n, d = a.d;
    unsigned long long n_ev = 0, n_re = 0;
    float serr = 0.f;   // largest relative screen error of this thread's rechecks
    Waste waste;
    for (int base = warp * PPW; base < m; base += nwarps * PPW) {
        const int pi = base + lane / G;
        const bool valid = pi < m;
        int pb = 0, qb = 0, na = 0, nb = 0;
        // a pair retrieved under a larger bound than this flush's rho_hi (one-pass rounds, or an
        // edge-batch overflow) has no edge in the range: it is skipped
        int2 pr = make_int2(0, 0);
        float plb = 0.f;
        if (valid) {   // the pair and its bound are independent loads
            pr = pairs[pi];
            plb = lbs[pi];
        }
        if (valid && plb < a.rho_hi_f) {
            int4 lp = a.rec[pr.x].l, lq = a.rec[pr.y].l;
            pb = lp.x; na = lp.y - lp.x; qb = lq.x; nb = lq.y - lq.x;
        }
        const int tot = na * nb;
        KMin best{~0ull, ~0ull};
        if (a.fp64) {
            for (int e = g; e < tot; e += G) {
                int i = pb + e / nb, j = qb + e % nb;
                double w = dist64(a.x64, n, d, i, j);
                if (a.cd64) w = pos_dmax(w, pos_dmax(a.cd64[i], a.cd64[j]));
                kmin_update(best, w, a.pid[i], a.pid[j]);
            }
        } else {
            // lane g visits e = g, g + G, ... of the na x nb grid; (i, j) advance without division.
            // The classes using this kernel have |A||B| <= kPer G, so a lane's screened values
            // stay in registers for the band test (no second evaluation).
            constexpr int kPer = 8;
            static_assert(kTinyMax <= kPer && kSmallMax <= 8 * kPer, "group kernel: a class exceeds kPer per lane");
            float sv[kPer];
            float smin = INFINITY;
            {
                int i = pb + (nb > 0 ? g / nb : 0), j = qb + (nb > 0 ? g % nb : 0);
#pragma unroll
                for (int t = 0; t < kPer; ++t) {
                    sv[t] = INFINITY;
                    if (g + t * G < tot) {
                        const float sd = D > 0 ? dist32p<D>(a.x4, i, j) : dist32t<D>(a.x32, n, d, i, j);
                        sv[t] = a.cd32 ? fmaxf(sd, fmaxf(a.cd32[i], a.cd32[j])) : sd;
                        smin = fminf(smin, sv[t]);
                        j += G;
                        while (j >= qb + nb) { j -= nb; ++i; }
                    }
                }
            }
#pragma unroll
            for (int o = G / 2; o; o >>= 1) smin = fminf(smin, __shfl_xor_sync(0xffffffffu, smin, o));
            // a pair whose screened minimum already proves its BCCP above the round's range
            // gets no recheck (its edge belongs to a later round, if any)
            const float T = screened_above(smin, a) ? -1.f : screen_threshold(smin, a);
            // the candidates (few) are evaluated again for the recheck.  A lane's first candidate is
            // rechecked after the loop, where the lanes run together (an FP64 instruction costs the
            // same however few lanes are active); later ones inline
            Deferred df;
#pragma unroll
            for (int t = 0; t < kPer; ++t) {
                if (g + t * G < tot && sv[t] <= T) {
                    const int e = g + t * G;
                    const int i = pb + e / nb, j = qb + e % nb;
                    const float sd = D > 0 ? dist32p<D>(a.x4, i, j) : dist32t<D>(a.x32, n, d, i, j);
                    const float c32 = a.cd32 ? fmaxf(a.cd32[i], a.cd32[j]) : 0.f;
                    if (df.i < 0) df = Deferred{i, j, sd, c32};
                    else kmin_update(best, checked_w2(a, i, j, sd, c32, serr), a.pid[i], a.pid[j]);
                    ++n_re;
                }
            }
            __syncwarp();
            if (df.i >= 0) kmin_update(best, checked_w2(a, df.i, df.j, df.sd, df.c32, serr), a.pid[df.i], a.pid[df.j]);
        }
#pragma unroll
        for (int o = G / 2; o; o >>= 1) {
            unsigned long long oh = __shfl_xor_sync(0xffffffffu, best.hi, o);
            unsigned long long ol = __shfl_xor_sync(0xffffffffu, best.lo, o);
            if (oh < best.hi || (oh == best.hi && ol < best.lo)) { best.hi = oh; best.lo = ol; }
        }
        if (g == 0) n_ev += (unsigned long long)tot;
        if (valid && g == 0) waste.add(range_side(a, best), (unsigned long long)tot);
        warp_emit(a, valid && g == 0 && in_range(a, best), best);
    }
    waste_flush(a, waste);
    err_flush(a, serr);
    n_ev = warp_sum_u64(n_ev);
    n_re = warp_sum_u64(n_re);
    if (lane == 0 && n_ev) {
        atomicAdd(a.stat + 1, n_ev);
        atomicAdd(a.stat + 2, n_re);
    }
}

__global__ void pack_nodes_kernel(int N, int d, int DP, const float *__restrict__ lo, const float *__restrict__ hi,
                                  const int *__restrict__ begin, const int *__restrict__ end,
                                  const int *__restrict__ left, const int *__restrict__ right,
                                  const float *__restrict__ diam2, const float *__restrict__ cdmin,
                                  const float *__restrict__ cdmax, NodeRec *__restrict__ rec, float *__restrict__ box)
{
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < N; x += gridDim.x * blockDim.x) {
        NodeRec r;
        r.l = make_int4(begin[x], end[x], left[x], -1);   // right[x] == left[x] + 1
        r.m = make_float4(diam2[x], cdmin ? cdmin[x] : 0.f, cdmax ? cdmax[x] : 0.f, 0.f);
        rec[x] = r;
        for (int k = 0; k < DP; ++k) {
            box[(size_t)x * 2 * DP + box_lo(k)] = k < d ? lo[(size_t)k * N + x] : 0.f;
            box[(size_t)x * 2 * DP + box_hi(k)] = k < d ? hi[(size_t)k * N + x] : 0.f;
        }
    }
}

// Initial frontier: (left(A), right(A)) for every internal node A whose points are not all
// connected (and, for GetRho, |A| > beta).
__global__ void frontier_init_kernel(TravArgs a, int mode, int2 *__restrict__ out, int *out_count)
{
    __shared__ int sh[32];
    // GetRho (and the combined pass, mode 2) reads the previous round's node list (every node in
    // the first round) and writes the survivors; GetPairs reads the survivors
    const int *in = mode != 1 ? a.node_in : a.node_out;
    const int m = in ? *(mode != 1 ? a.node_in_n : a.node_out_n) : a.N;
    for (int b0 = blockIdx.x * blockDim.x; b0 < m; b0 += gridDim.x * blockDim.x) {
        const int t = b0 + threadIdx.x;
        const int x = t < m ? (in ? in[t] : t) : -1;
        const bool cand = x >= 0 && a.left[x] >= 0 && a.comp[x] < 0;
        if (mode != 1 && a.node_out) {
            const int s = block_append(a.node_out_n, cand ? 1 : 0, sh);
            if (cand) a.node_out[s] = x;
        }
        // GetRho may start from a sample of the frontier: the minimum over fewer pairs is an
        // upper bound of the exact one, which is still a valid split of the weight range
        const int push = cand && (mode != 0 || (nsize(a, x) > a.beta && t % a.rho_sample == 0)) ? 1 : 0;
        const int slot = block_append(out_count, push, sh);
        if (push) {
            if (slot < a.frontier_cap) out[slot] = make_int2(a.left[x], a.right[x]);
            else atomicOr(a.overflow, 1u);
        }
    }
}

// ------------------------------------------------------------------------ component labels
__global__ void uf_flatten_kernel(int *uf, int n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int r = i;
        for (int it = 0; it < n && uf[r] != r; ++it) r = uf[r];
        uf[i] = r;
    }
}

// Component labels.  A node's points are the tree positions [begin, end); they all lie in one
// component iff the per-position label (the union-find root of the point) does not change inside
// the range.  With chg[i] = (lab[i] != lab[i-1]) and E its exclusive prefix sum, node x is in one
// component iff E[end] == E[begin + 1].
__global__ void pos_labels_kernel(const int *__restrict__ pid, const int *__restrict__ uf, int n, int *__restrict__ lab,
                                  int *__restrict__ chg)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int l = uf[pid[i]];
        lab[i] = l;
        chg[i] = i > 0 && l != uf[pid[i - 1]];
    }
}

__global__ void node_labels_kernel(int N, NodeRec *__restrict__ rec, const int *__restrict__ lab,
                                   const int *__restrict__ E, int *__restrict__ comp)
{
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < N; x += gridDim.x * blockDim.x) {
        const int4 L = rec[x].l;
        const int c = E[L.y] == E[L.x + 1] ? lab[L.x] : -1;
        comp[x] = c;
        rec[x].l.w = c;
    }
}

// ------------------------------------------------------------------------- BCCP tile kernel
constexpr int kItems = 2;              // points of the larger side per lane
constexpr int kTileA = 32 * kItems;
// points of the smaller side staged per warp (8 warps per block, static shared memory < 48 KB)
__host__ __device__ constexpr int tile_q(int dd) { return dd <= 8 ? 128 : 64; }

__global__ void huge_items_kernel(const TravArgs a, const int2 *__restrict__ pairs, const float *__restrict__ lbs, int m,
                                  long long *__restrict__ items)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < m) {
        int P = pairs[j].x, Q = pairs[j].y;
        int4 lp = a.rec[P].l, lq = a.rec[Q].l;
        int small = min(lp.y - lp.x, lq.y - lq.x);   // the query side
        // no work for a pair retrieved under a larger bound than this flush's rho_hi
        items[j] = lbs[j] < a.rho_hi_f ? (small + 31) / 32 : 0;
        EdgeK none;
        none.hi = ~0ull;
        none.lo = ~0ull;
        a.huge_best[j] = none;
        a.huge_sbest[j] = 0x7f800000u;   // +inf
    }
}

template <int DP, int DM, bool HDB, bool FP64>
__global__ void __launch_bounds__(256) bccp_dual_kernel(TravArgs a, const int2 *__restrict__ pairs, int m,
                                                        const long long *__restrict__ item_off,
                                                        const long long *__restrict__ total_items)
{
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    int *stk = a.stack + (size_t)gw * a.stack_cap;
    const long long TI = *total_items;
    const int n = a.n, d = a.d;
    const float rho_hi_f = a.rho_hi_f;
    unsigned long long n_ev = 0, n_re = 0;
    float serr = 0.f;
    for (long long item = gw; item < TI; item += nw) {
        int lo = 0, hi = m - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (item_off[mid] <= item) lo = mid; else hi = mid - 1;
        }
        const int j = lo;
        const int P = pairs[j].x, Q = pairs[j].y;
        const int4 lp = a.rec[P].l, lq = a.rec[Q].l;
        // queries: the smaller side; its points far from the other side are pruned at the other
        // tree's root, the rest run a nearest-first descent into it
        const bool pq = lp.y - lp.x <= lq.y - lq.x;   // P is the query side
        const int Aend = pq ? lp.y : lq.y;
        const int Broot = pq ? Q : P;
        const int i = (pq ? lp.x : lq.x) + (int)(item - item_off[j]) * 32 + lane;
        const bool valid = i < Aend;
        const int ii = valid ? i : (pq ? lp.x : lq.x);
        float qx[DM];
        double qx64[DM];
#pragma unroll
        for (int k = 0; k < DM; ++k) {
            if (k < d) {
                qx[k] = a.x32[(size_t)k * n + ii];
                if (FP64) qx64[k] = a.x64[(size_t)k * n + ii];
            }
        }
        const float qcd = HDB ? a.cd32[ii] : 0.f;
        const int qpid = a.pid[ii];
        KMin best{~0ull, ~0ull};
        // threshold (screened scale) and its reload from the shared WriteMin
        auto cur_thr = [&]() -> float {
            float t;
            if (FP64) {
                unsigned long long hb = ((volatile unsigned long long *)&a.huge_best[j].hi)[0];
                t = hb == ~0ull ? INFINITY : __double2float_ru(__longlong_as_double((long long)hb));
            } else {
                float sb = __uint_as_float(((volatile unsigned *)a.huge_sbest)[j]);
                t = sb == INFINITY ? INFINITY : screen_threshold(sb, a);
            }
            return fminf(t, rho_hi_f);
        };
        float thr = cur_thr();
        int sp = 0;
        if (lane == 0) stk[0] = Broot;
        sp = 1;
        __syncwarp();
        for (int guard = 0; sp > 0 && guard < 2 * a.N + 2; ++guard) {
            const int node = stk[sp - 1];
            __syncwarp();
            --sp;
            const int4 ln = a.rec[node].l;
            const float *bx = a.box + (size_t)node * 2 * DP;
            float lb = 0.f;
#pragma unroll
            for (int k = 0; k < DM; ++k) {
                if (k < d) {
                    float g = fmaxf(fmaxf(bx[box_lo(k)] - qx[k], qx[k] - bx[box_hi(k)]), 0.f);
                    lb = fmaf(g, g, lb);
                }
            }
            float lbw = lower_w2(lb);
            if (HDB) lbw = fmaxf(lbw, fmaxf(qcd * (1.0f - 1.0f / 4194304.0f), a.rec[node].m.y));
            const bool need = valid && lbw <= thr * (1.0f + 1.0f / 131072.0f);
            if (!__any_sync(0xffffffffu, need)) continue;
            const int bsz = ln.y - ln.x;
            if (bsz <= 32) {
                const int b0 = ln.x;
                float px[DM];
                double px64[DM];
#pragma unroll
                for (int k = 0; k < DM; ++k) {
                    if (k < d) {
                        px[k] = lane < bsz ? a.x32[(size_t)k * n + b0 + lane] : 0.f;
                        if (FP64) px64[k] = lane < bsz ? a.x64[(size_t)k * n + b0 + lane] : 0.0;
                    }
                }
                const float pcd = (HDB && lane < bsz) ? a.cd32[b0 + lane] : 0.f;
                const int ppid = lane < bsz ? a.pid[b0 + lane] : 0;
                if (FP64) {
                    for (int p = 0; p < bsz; ++p) {
                        double acc = 0.0;
#pragma unroll
                        for (int k = 0; k < DM; ++k) {
                            if (k < d) {
                                double t = __dsub_rn(qx64[k], __shfl_sync(0xffffffffu, px64[k], p));
                                acc = __dadd_rn(acc, __dmul_rn(t, t));
                            }
                        }
                        int bp = __shfl_sync(0xffffffffu, ppid, p);
                        if (HDB) acc = pos_dmax(acc, pos_dmax(a.cd64[ii], a.cd64[b0 + p]));
                        if (valid) kmin_update(best, acc, qpid, bp);
                    }
                    n_ev += (unsigned long long)bsz;
                    // publish this warp's best so other items prune against it
                    KMin wb = best;
                    for (int o = 16; o; o >>= 1) {
                        unsigned long long oh = __shfl_xor_sync(0xffffffffu, wb.hi, o);
                        unsigned long long ol = __shfl_xor_sync(0xffffffffu, wb.lo, o);
                        if (oh < wb.hi || (oh == wb.hi && ol < wb.lo)) { wb.hi = oh; wb.lo = ol; }
                    }
                    if (lane == 0 && wb.hi != ~0ull) {
                        EdgeK *slot = a.huge_best + j;
                        EdgeK mine;
                        mine.hi = wb.hi;
                        mine.lo = wb.lo;
                        EdgeK cur = *slot;
                        for (int it = 0; it < (1 << 20) && edge_less(mine, cur); ++it) {
                            EdgeK old = atomicCAS(slot, cur, mine);
                            if (old.hi == cur.hi && old.lo == cur.lo) break;
                            cur = old;
                        }
                    }
                    __syncwarp();
                } else {
                    float smin = INFINITY;
                    for (int p = 0; p < bsz; ++p) {
                        float acc = 0.f;
#pragma unroll
                        for (int k = 0; k < DM; ++k) {
                            if (k < d) {
                                float t = qx[k] - __shfl_sync(0xffffffffu, px[k], p);
                                acc = fmaf(t, t, acc);
                            }
                        }
                        if (HDB) acc = fmaxf(acc, fmaxf(qcd, __shfl_sync(0xffffffffu, pcd, p)));
                        if (valid) smin = fminf(smin, acc);
                    }
                    for (int o = 16; o; o >>= 1) smin = fminf(smin, __shfl_xor_sync(0xffffffffu, smin, o));
                    if (lane == 0 && smin < INFINITY) atomicMin(a.huge_sbest + j, __float_as_uint(smin));
                    thr = fminf(thr, fminf(screen_threshold(smin, a), rho_hi_f));
                    thr = fminf(thr, cur_thr());
                    for (int p = 0; p < bsz; ++p) {
                        float acc = 0.f;
#pragma unroll
                        for (int k = 0; k < DM; ++k) {
                            if (k < d) {
                                float t = qx[k] - __shfl_sync(0xffffffffu, px[k], p);
                                acc = fmaf(t, t, acc);
                            }
                        }
                        const float c32 = HDB ? fmaxf(qcd, __shfl_sync(0xffffffffu, pcd, p)) : 0.f;
                        const float sd = acc;
                        if (HDB) acc = fmaxf(acc, c32);
                        int bp = __shfl_sync(0xffffffffu, ppid, p);
                        if (valid && acc <= thr) {
                            kmin_update(best, checked_w2(a, ii, b0 + p, sd, c32, serr), qpid, bp);
                            ++n_re;
                        }
                    }
                    n_ev += (unsigned long long)bsz;
                }
                if (FP64) thr = cur_thr();
            } else {
                // push the farther child first so the nearer one is visited next
                const int c0 = ln.z, c1 = ln.z + 1;
                const float *b0x = a.box + (size_t)c0 * 2 * DP, *b1x = a.box + (size_t)c1 * 2 * DP;
                float l0 = 0.f, l1 = 0.f;
#pragma unroll
                for (int k = 0; k < DM; ++k) {
                    if (k < d) {
                        float g0 = fmaxf(fmaxf(b0x[box_lo(k)] - qx[k], qx[k] - b0x[box_hi(k)]), 0.f);
                        float g1 = fmaxf(fmaxf(b1x[box_lo(k)] - qx[k], qx[k] - b1x[box_hi(k)]), 0.f);
                        l0 = fmaf(g0, g0, l0);
                        l1 = fmaf(g1, g1, l1);
                    }
                }
                if (!valid) { l0 = 0.f; l1 = 0.f; }
                for (int o = 16; o; o >>= 1) {
                    l0 += __shfl_xor_sync(0xffffffffu, l0, o);
                    l1 += __shfl_xor_sync(0xffffffffu, l1, o);
                }
                if (sp + 2 > a.stack_cap) {   // cannot happen: cap = tree depth + 4; reported, not ignored
                    if (lane == 0) atomicOr(a.overflow, 8u);
                    break;
                }
                if (lane == 0) {
                    stk[sp] = l0 <= l1 ? c1 : c0;
                    stk[sp + 1] = l0 <= l1 ? c0 : c1;
                }
                __syncwarp();
                sp += 2;
            }
        }
        // fold this item's K-minimum into the pair's slot
        for (int o = 16; o; o >>= 1) {
            unsigned long long oh = __shfl_xor_sync(0xffffffffu, best.hi, o);
            unsigned long long ol = __shfl_xor_sync(0xffffffffu, best.lo, o);
            if (oh < best.hi || (oh == best.hi && ol < best.lo)) { best.hi = oh; best.lo = ol; }
        }
        if (lane == 0 && best.hi != ~0ull) {
            EdgeK *slot = a.huge_best + j;
            EdgeK mine;
            mine.hi = best.hi;
            mine.lo = best.lo;
            EdgeK cur = *slot;
            for (int it = 0; it < (1 << 20) && edge_less(mine, cur); ++it) {
                EdgeK old = atomicCAS(slot, cur, mine);
                if (old.hi == cur.hi && old.lo == cur.lo) break;
                cur = old;
            }
        }
        __syncwarp();
    }
    err_flush(a, serr);
    n_ev = warp_sum_u64(n_ev);
    n_re = warp_sum_u64(n_re);
    if (lane == 0 && n_ev) {
        atomicAdd(a.stat + 1, n_ev);
        atomicAdd(a.stat + 2, n_re);
        atomicAdd(a.stat + 6, n_ev);
    }
}

__global__ void huge_emit_kernel(TravArgs a, int m)
{
    const int lane = threadIdx.x & 31;
    Waste waste;
    const int limit = (m + 31) & ~31;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j - lane < limit; j += gridDim.x * blockDim.x) {
        KMin b{~0ull, ~0ull};
        if (j < m) { b.hi = a.huge_best[j].hi; b.lo = a.huge_best[j].lo; }
        // (a BCCP above the range may be a partial minimum here: the dual-tree search prunes at rho_hi)
        if (j < m) waste.add(range_side(a, b), 0);
        warp_emit(a, j < m && in_range(a, b), b);
    }
    waste_flush(a, waste);
}

// BCCP of one medium or big pair per warp (pairs handed out in small chunks): the larger side A
// on the lanes (kItems points each), the smaller side B staged in shared memory in chunks of
// kTileQ.  FP32 screen against a running warp minimum, FP64 re-evaluation of every candidate
// inside the band of the running minimum (the threshold only decreases, so every candidate of
// the final band is re-evaluated), warp K-minimum, emitted when its FP64 w2 lies in
// [rho_lo, rho_hi).
template <int D, bool HDB, bool FP64>
__global__ void __launch_bounds__(256) bccp_pair_tile_kernel(TravArgs a, const int2 *__restrict__ pairs,
                                                             const float *__restrict__ lbs, int m, int *next, int chunk)
{
    constexpr int DD = D > 0 ? D : kMaxDim;
    constexpr int kTileQ = tile_q(DD);
    __shared__ float qs[8][kTileQ * (DD + 1)];
    __shared__ EdgeK ebuf[8][32];   // per warp: emitted edges, appended to the batch 32 at a time
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    float *q = qs[wib];
    EdgeK *eb = ebuf[wib];
    int ecnt = 0;   // warp-uniform
    auto flush_edges = [&]() {
        int base = 0;
        if (lane == 0) base = atomicAdd(a.edge_count, ecnt);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (lane < ecnt) {
            if (base + lane < a.edge_cap) a.edges[base + lane] = eb[lane];
            else atomicOr(a.overflow, 2u);
        }
        ecnt = 0;
        __syncwarp();
    };
    const int d = D > 0 ? D : a.d;
    const int n = a.n;
    unsigned long long n_ev = 0, n_re = 0, n_skip = 0;
    float serr = 0.f;
    Waste waste;
    // pairs handed out `chunk` at a time (sizes vary too much for a static deal; on long lists
    // one counter increment per pair would serialise the warps on it)
    int j = 0, jend = 0;
    while (true) {
        if (j == jend) {
            int base = 0;
            if (lane == 0) base = atomicAdd(next, chunk);
            base = __shfl_sync(0xffffffffu, base, 0);
            if (base >= m) break;
            j = base;
            jend = min(base + chunk, m);
        }
        const int2 pr = pairs[j];
        if (lbs[j++] >= a.rho_hi_f) {   // retrieved under a larger bound: no edge in the range
            if (lane == 0) waste.add(1, 0);
            continue;
        }
        const int4 lp = a.rec[pr.x].l, lq = a.rec[pr.y].l;
        const bool pa = lp.y - lp.x >= lq.y - lq.x;   // A: the larger side, on the lanes
        const int abeg = pa ? lp.x : lq.x, aend = pa ? lp.y : lq.y;
        const int bbeg = pa ? lq.x : lp.x, bend = pa ? lq.y : lp.y;
        KMin best{~0ull, ~0ull};
        Deferred df;                // this lane's first candidate, rechecked at the end of the pair
        float run_min = INFINITY;   // screened minimum over the chunks done so far
        for (int a0 = abeg; a0 < aend; a0 += kTileA) {
            const int a1 = min(a0 + kTileA, aend);
            float ax[kItems][DD];
            float acd[kItems];
            bool av[kItems];
#pragma unroll
            for (int it = 0; it < kItems; ++it) {
                const int i = a0 + lane + 32 * it;
                av[it] = i < a1;
                const int ii = av[it] ? i : a0;
#pragma unroll
                for (int k = 0; k < DD; ++k)
                    if (D > 0 || k < d) ax[it][k] = a.x32[(size_t)k * n + ii];
                acd[it] = HDB ? a.cd32[ii] : 0.f;
            }
            for (int b0 = bbeg; b0 < bend; b0 += kTileQ) {
                const int nb = min(kTileQ, bend - b0);
                __syncwarp();
                // stage the B chunk: q[jj*(DD+1) + k], last slot = cd (HDB); gather its bounding box
                // and smallest core distance on the way
                float blo[DD], bhi[DD];
#pragma unroll
                for (int k = 0; k < DD; ++k) { blo[k] = INFINITY; bhi[k] = -INFINITY; }
                float bcd = INFINITY;
                for (int jj = lane; jj < nb; jj += 32) {
#pragma unroll
                    for (int k = 0; k < DD; ++k)
                        if (D > 0 || k < d) {
                            const float v = a.x32[(size_t)k * n + b0 + jj];
                            q[jj * (DD + 1) + k] = v;
                            blo[k] = fminf(blo[k], v);
                            bhi[k] = fmaxf(bhi[k], v);
                        }
                    const float c = HDB ? a.cd32[b0 + jj] : 0.f;
                    q[jj * (DD + 1) + DD] = c;
                    bcd = fminf(bcd, c);
                }
                // Chunk pruning: an A point skips the chunk when a rigorous lower bound of its
                // FP64 w2 to every point of the chunk exceeds both the band threshold of the
                // running screened minimum (then none of them can be a candidate) and rho_hi
                // (then none of them can give this round's edge), with the margins the dual-tree
                // kernel uses.  The box is widened by delta so that it holds the FP64 points.
                float thr_now;
                if (FP64) {
                    thr_now = best.hi == ~0ull ? INFINITY : __double2float_ru(__longlong_as_double((long long)best.hi));
                    for (int o = 16; o; o >>= 1) thr_now = fminf(thr_now, __shfl_xor_sync(0xffffffffu, thr_now, o));
                } else {
                    thr_now = run_min == INFINITY ? INFINITY : screen_threshold(run_min, a);
                }
                thr_now = fminf(thr_now, a.rho_hi_f) * (1.0f + 1.0f / 131072.0f);
                bool live[kItems];
                bool any_live = false;
                if (thr_now < INFINITY) {
#pragma unroll
                    for (int k = 0; k < DD; ++k) {
                        if (D > 0 || k < d) {
                            for (int o = 16; o; o >>= 1) {
                                blo[k] = fminf(blo[k], __shfl_xor_sync(0xffffffffu, blo[k], o));
                                bhi[k] = fmaxf(bhi[k], __shfl_xor_sync(0xffffffffu, bhi[k], o));
                            }
                            if (!a.exact32) {
                                blo[k] = __fsub_rd(blo[k], a.delta32);
                                bhi[k] = __fadd_ru(bhi[k], a.delta32);
                            }
                        }
                    }
                    if (HDB) for (int o = 16; o; o >>= 1) bcd = fminf(bcd, __shfl_xor_sync(0xffffffffu, bcd, o));
#pragma unroll
                    for (int it = 0; it < kItems; ++it) {
                        float g2 = 0.f;
#pragma unroll
                        for (int k = 0; k < DD; ++k) {
                            if (D > 0 || k < d) {
                                const float g = fmaxf(fmaxf(blo[k] - ax[it][k], ax[it][k] - bhi[k]), 0.f);
                                g2 = fmaf(g, g, g2);
                            }
                        }
                        float lbw = lower_w2(g2);
                        if (HDB) lbw = fmaxf(lbw, fmaxf(acd[it], bcd) * (1.0f - 1.0f / 4194304.0f));
                        live[it] = av[it] && lbw <= thr_now;
                        any_live = any_live || live[it];
                    }
                } else {
#pragma unroll
                    for (int it = 0; it < kItems; ++it) { live[it] = av[it]; any_live = any_live || live[it]; }
                }
                if (!__any_sync(0xffffffffu, any_live)) {
                    n_skip += (unsigned long long)((a1 - a0) * nb);
                    continue;
                }
                if (!FP64) {
                    float mn[kItems];
#pragma unroll
                    for (int it = 0; it < kItems; ++it) mn[it] = INFINITY;
                    for (int jj = 0; jj < nb; ++jj) {
                        const float *qq = q + jj * (DD + 1);
                        float qv[DD];
#pragma unroll
                        for (int k = 0; k < DD; ++k)
                            if (D > 0 || k < d) qv[k] = qq[k];
#pragma unroll
                        for (int it = 0; it < kItems; ++it) {
                            float s = 0.f;
#pragma unroll
                            for (int k = 0; k < DD; ++k) {
                                if (D > 0 || k < d) {
                                    float t = ax[it][k] - qv[k];
                                    s = fmaf(t, t, s);
                                }
                            }
                            if (HDB) s = fmaxf(s, fmaxf(acd[it], qq[DD]));
                            mn[it] = fminf(mn[it], s);
                        }
                    }
                    float wmn = INFINITY;
#pragma unroll
                    for (int it = 0; it < kItems; ++it) {
                        if (!live[it]) mn[it] = INFINITY;   // pruned: no candidate in this chunk
                        wmn = fminf(wmn, mn[it]);
                    }
                    for (int o = 16; o; o >>= 1) wmn = fminf(wmn, __shfl_xor_sync(0xffffffffu, wmn, o));
                    run_min = fminf(run_min, wmn);
                    // nothing to recheck while the running minimum proves the pair above the range
                    const float T = screened_above(run_min, a) ? -1.f : screen_threshold(run_min, a);
                    int nre = 0;
#pragma unroll
                    for (int it = 0; it < kItems; ++it) {
                        if (!live[it] || mn[it] > T) continue;
                        const int i = a0 + lane + 32 * it;
                        for (int jj = 0; jj < nb; ++jj) {
                            const float *qq = q + jj * (DD + 1);
                            float s = 0.f;
#pragma unroll
                            for (int k = 0; k < DD; ++k) {
                                if (D > 0 || k < d) {
                                    float t = ax[it][k] - qq[k];
                                    s = fmaf(t, t, s);
                                }
                            }
                            const float c32 = HDB ? fmaxf(acd[it], qq[DD]) : 0.f;
                            const float sd = s;
                            if (HDB) s = fmaxf(s, c32);
                            if (s <= T) {
                                if (df.i < 0) df = Deferred{i, b0 + jj, sd, c32};
                                else kmin_update(best, checked_w2(a, i, b0 + jj, sd, c32, serr), a.pid[i], a.pid[b0 + jj]);
                                ++nre;
                            }
                        }
                    }
                    n_re += (unsigned long long)nre;
                } else {
#pragma unroll
                    for (int it = 0; it < kItems; ++it) {
                        if (!live[it]) continue;
                        const int i = a0 + lane + 32 * it;
                        for (int jj = 0; jj < nb; ++jj) {
                            double w = dist64(a.x64, n, d, i, b0 + jj);
                            if (HDB) w = pos_dmax(w, pos_dmax(a.cd64[i], a.cd64[b0 + jj]));
                            kmin_update(best, w, a.pid[i], a.pid[b0 + jj]);
                        }
                    }
                }
                n_ev += (unsigned long long)((a1 - a0) * nb);
            }
        }
        __syncwarp();
        if (!FP64 && df.i >= 0 && !screened_above(run_min, a) && screen_value(df, HDB) <= screen_threshold(run_min, a))
            kmin_update(best, checked_w2(a, df.i, df.j, df.sd, df.c32, serr), a.pid[df.i], a.pid[df.j]);
        // warp K-minimum of the pair
        for (int o = 16; o; o >>= 1) {
            unsigned long long oh = __shfl_xor_sync(0xffffffffu, best.hi, o);
            unsigned long long ol = __shfl_xor_sync(0xffffffffu, best.lo, o);
            if (oh < best.hi || (oh == best.hi && ol < best.lo)) { best.hi = oh; best.lo = ol; }
        }
        if (lane == 0) waste.add(range_side(a, best), (unsigned long long)(aend - abeg) * (unsigned long long)(bend - bbeg));
        if (in_range(a, best)) {   // best is the same on every lane
            if (lane == 0) {
                EdgeK e;
                e.hi = best.hi;
                e.lo = best.lo;
                eb[ecnt] = e;
            }
            __syncwarp();
            if (++ecnt == 32) flush_edges();
        }
    }
    if (ecnt > 0) flush_edges();
    waste_flush(a, waste);
    err_flush(a, serr);
    n_re = warp_sum_u64(n_re);
    if (lane == 0 && n_ev) {
        atomicAdd(a.stat + 1, n_ev);
        atomicAdd(a.stat + 3, n_ev);
        atomicAdd(a.stat + 2, n_re);
    }
    if (lane == 0 && n_skip) atomicAdd(a.stat + 11, n_skip);
}

}  // namespace

// ----------------------------------------------------------------------------- host side

int launch_comp_labels(const Tree &T, const Points &P, int *uf, NodeRec *rec, int *scratch,
                       Arena &ar, cudaStream_t st)
{
    const int n = P.n;
    int *lab = scratch, *E = scratch + n;   // E holds n + 1 entries
    launch(uf_flatten_kernel, grid_for(n, 256), 256, 0, st, uf, n);
    launch(pos_labels_kernel, grid_for(n, 256), 256, 0, st, P.pid, uf, n, lab, E);
    int rc = scan_exclusive_i32(E, E, n, E + n, st, ar);
    if (rc) return rc;
    launch(node_labels_kernel, grid_for(T.N, 256), 256, 0, st, T.N, rec, lab, E, T.comp);
    return 0;
}

// ----------------------------------------------------------- bounded-memory traversal
// The pending pairs form a stack (S plus the previous step's output on top of it).  One step pops
// at most `chunk` pairs and pushes back at most chunk + warps * kDfsWarpCap, so the stack grows by
// a bounded amount per step while the traversal goes depth first.
void traversal_init(int mode, TravArgs &a, int2 *stack, int *cnt, cudaStream_t st)
{
    cudaMemsetAsync(cnt, 0, sizeof(int) * kTravCounters, st);
    if (mode != 1 && a.node_out_n) cudaMemsetAsync(a.node_out_n, 0, sizeof(int), st);
    launch(frontier_init_kernel, grid_for(a.N, 256), 256, 0, st, a, mode, stack, cnt + 0);
}

// Warps of a step: at most 2 chunk / (64 budget + kDfsWarpCap), so that a step's output
// (children of at most chunk + warps * 32 * budget visits, plus every warp's full stack) fits
// in 4 * chunk pairs.
int dfs_warps(int chunk, int budget)
{
    long long w = 2LL * chunk / (64 * budget + kDfsWarpCap);
    const long long wmax = (long long)num_sms() * 4 * kDfsWarpsPerBlock;
    w = w > wmax ? wmax : w;
    w = w / kDfsWarpsPerBlock * kDfsWarpsPerBlock;
    return (int)(w < kDfsWarpsPerBlock ? kDfsWarpsPerBlock : w);
}

long long dfs_out_cap(int chunk, int budget)
{
    return 2LL * chunk + (long long)dfs_warps(chunk, budget) * (64 * budget + kDfsWarpCap);
}

long long dfs_step_visits(int chunk, int budget)
{
    return (long long)chunk + (long long)dfs_warps(chunk, budget) * 32 * budget;
}

void traversal_step(int mode, TravArgs &a, int2 *stack, int2 *const xbuf[2], int *cnt, int step, int chunk,
                    cudaStream_t st)
{
    DfsArgs s;
    const int cur = step & 1;
    s.S = stack;
    s.top = cnt + 0;
    s.xin = xbuf[cur];
    s.xin_count = cnt + (cur ? 2 : 1);
    s.xout = xbuf[cur ^ 1];
    s.xout_count = cnt + (cur ? 1 : 2);
    s.next = cnt + 3;
    s.done = (unsigned *)(cnt + 4);
    s.chunk = chunk;
    s.xcap = (int)std::min<long long>(dfs_out_cap(chunk, a.dfs_budget), 4LL * chunk);   // the output buffers hold 4 * chunk pairs
    s.budget = a.dfs_budget;
    const int grid = dfs_warps(chunk, a.dfs_budget) / kDfsWarpsPerBlock;
#define WM_FP(DPV)                                                                                \
    do {                                                                                          \
        if (mode == 0) launch(findpair_dfs_kernel<0, DPV>, grid, 32 * kDfsWarpsPerBlock, 0, st, a, s); \
        else if (mode == 2) launch(findpair_dfs_kernel<2, DPV>, grid, 32 * kDfsWarpsPerBlock, 0, st, a, s); \
        else launch(findpair_dfs_kernel<1, DPV>, grid, 32 * kDfsWarpsPerBlock, 0, st, a, s);           \
    } while (0)
    if (a.dp == 4) WM_FP(4);
    else if (a.dp == 8) WM_FP(8);
    else WM_FP(16);
#undef WM_FP
}

// GetRho: the whole traversal, polling emptiness every 3 steps.
int run_traversal(TravArgs &a, int2 *stack, int2 *const xbuf[2], int *cnt, int chunk, cudaStream_t st, int *pinned,
                  unsigned *overflow_out, int *steps_out)
{
    traversal_init(0, a, stack, cnt, st);
    int steps = 0;
    while (true) {
        for (int b = 0; b < 3; ++b, ++steps) traversal_step(0, a, stack, xbuf, cnt, steps, chunk, st);
        cudaMemcpyAsync(pinned, cnt, sizeof(int) * kTravCounters, cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(pinned + kTravCounters, a.overflow, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) return WM_ECUDA;
        if (pinned[kTravCounters]) { *overflow_out = (unsigned)pinned[kTravCounters]; return 0; }
        if (pinned[0] == 0 && pinned[1] == 0 && pinned[2] == 0) break;
        if (steps > 10000000) {
            set_error_detail("WSPD traversal did not terminate");
            return WM_EINTERNAL;
        }
    }
    *overflow_out = 0;
    if (steps_out) *steps_out = steps;
    return 0;
}

// ------------------------------------------------------------- shrinking rho_hi in a round
// Deterministic split of an edge batch for a smaller rho_hi: the largest w2 (bits WriteMax), then
// a histogram of the weights over [lo, largest] in kSplitBins equal bins.  Both depend only on the
// multiset of weights, not on the order in which the edges were appended.
__global__ void w2_max_kernel(const EdgeK *__restrict__ e, int m, unsigned long long *out)
{
    unsigned long long mx = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) mx = max(mx, e[i].hi);
    for (int o = 16; o; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx) atomicMax(out, mx);
}

__global__ void w2_hist_kernel(const EdgeK *__restrict__ e, int m, double lo, const unsigned long long *__restrict__ maxbits,
                               int *hist)
{
    const double hi = __longlong_as_double((long long)*maxbits);
    const double scale = hi > lo ? (double)kSplitBins / (hi - lo) : 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        const double w = edge_w2(e[i]);
        int b = (int)((w - lo) * scale);
        b = b < 0 ? 0 : b >= kSplitBins ? kSplitBins - 1 : b;
        atomicAdd(hist + b, 1);
    }
}

__global__ void keep_below_kernel(const EdgeK *__restrict__ in, int m, double bound, EdgeK *__restrict__ out, int *count)
{
    const int lane = threadIdx.x & 31;
    const int limit = (m + 31) & ~31;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t - lane < limit; t += gridDim.x * blockDim.x) {
        bool keep = false;
        EdgeK e;
        if (t < m) { e = in[t]; keep = edge_w2(e) < bound; }
        unsigned b = __ballot_sync(0xffffffffu, keep);
        int base = 0;
        if (lane == 0 && b) base = atomicAdd(count, __popc(b));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (keep) out[base + __popc(b & lanemask_lt())] = e;
    }
}

void w2_histogram(const EdgeK *e, int m, double lo, unsigned long long *maxbits, int *hist, cudaStream_t st)
{
    cudaMemsetAsync(maxbits, 0, sizeof(unsigned long long), st);
    cudaMemsetAsync(hist, 0, sizeof(int) * kSplitBins, st);
    if (m <= 0) return;
    launch(w2_max_kernel, grid_for(m, 256), 256, 0, st, e, m, maxbits);
    launch(w2_hist_kernel, grid_for(m, 256), 256, 0, st, e, m, lo, maxbits, hist);
}

void keep_below(const EdgeK *in, int m, double bound, EdgeK *out, int *count, cudaStream_t st)
{
    cudaMemsetAsync(count, 0, sizeof(int), st);
    if (m > 0) launch(keep_below_kernel, grid_for(m, 256), 256, 0, st, in, m, bound, out, count);
}

// BCCP of the tiny, small and medium pair lists (counts read back by the host).
template <int D>
static void run_bccp_groups_d(TravArgs &a, const int *counts_host, cudaStream_t st)
{
    if (counts_host[0] > 0)
        launch(bccp_group_kernel<1, D>, grid_for((long long)counts_host[0], 256), 256, 0, st, a, a.list[0],
               a.list_lb[0], a.list_count + 0);
    if (counts_host[1] > 0)
        launch(bccp_group_kernel<8, D>, grid_for((long long)counts_host[1] * 8, 256), 256, 0, st, a, a.list[1],
               a.list_lb[1], a.list_count + 1);
}

void run_bccp_groups(TravArgs &a, const int *counts_host, cudaStream_t st)
{
    switch (a.d) {
    case 2: run_bccp_groups_d<2>(a, counts_host, st); break;
    case 3: run_bccp_groups_d<3>(a, counts_host, st); break;
    case 5: run_bccp_groups_d<5>(a, counts_host, st); break;
    case 7: run_bccp_groups_d<7>(a, counts_host, st); break;
    default: run_bccp_groups_d<0>(a, counts_host, st); break;
    }
}

__global__ void point_major_kernel(const float *__restrict__ x32, int n, int d, int dq, float4 *__restrict__ x4)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)n * dq;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t / dq), c = (int)(t % dq);
        float v[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) v[r] = 4 * c + r < d ? x32[(size_t)(4 * c + r) * n + i] : 0.f;
        x4[t] = make_float4(v[0], v[1], v[2], v[3]);
    }
}

void point_major(const float *x32, int n, int d, int dp, float4 *x4, cudaStream_t st)
{
    launch(point_major_kernel, grid_for((long long)n * (dp / 4), 256), 256, 0, st, x32, n, d, dp / 4, x4);
}

void pack_nodes(const Tree &T, int d, int dp, NodeRec *rec, float *box, cudaStream_t st)
{
    launch(pack_nodes_kernel, grid_for(T.N, 256), 256, 0, st, T.N, d, dp, T.lo, T.hi, T.begin, T.end, T.left, T.right,
           T.diam2, T.cdmin, T.cdmax, rec, box);
}

// Pruned BCCP of the pairs of a list (the huge pairs, or a short list of big pairs that the
// tile kernel would give to a few warps only): one warp per 32 points of a pair's smaller side.
int run_bccp_huge(TravArgs &a, const int2 *pairs, const float *lbs, int m, long long *items, long long *total,
                  cudaStream_t st, Arena &ar, bool hdb, bool fp64, int stack_warps)
{
    if (m <= 0) return 0;
    launch(huge_items_kernel, grid_for(m, 256, 1 << 20), 256, 0, st, a, pairs, lbs, m, items);
    int rc = scan_exclusive_i64(items, items, m, total, st, ar);
    if (rc) return rc;
    const int blocks = stack_warps / 8;
#define WM_DUAL(DPV, DMV)                                                                                     \
    do {                                                                                                      \
        if (fp64) {                                                                                           \
            if (hdb) launch(bccp_dual_kernel<DPV, DMV, true, true>, blocks, 256, 0, st, a, pairs, m, items, total);   \
            else launch(bccp_dual_kernel<DPV, DMV, false, true>, blocks, 256, 0, st, a, pairs, m, items, total);      \
        } else {                                                                                              \
            if (hdb) launch(bccp_dual_kernel<DPV, DMV, true, false>, blocks, 256, 0, st, a, pairs, m, items, total);  \
            else launch(bccp_dual_kernel<DPV, DMV, false, false>, blocks, 256, 0, st, a, pairs, m, items, total);     \
        }                                                                                                     \
    } while (0)
    if (a.d <= 2) WM_DUAL(4, 2);
    else if (a.d <= 3) WM_DUAL(4, 3);
    else if (a.d <= 4) WM_DUAL(4, 4);
    else if (a.d <= 8) WM_DUAL(8, 8);
    else WM_DUAL(16, 16);
#undef WM_DUAL
    launch(huge_emit_kernel, grid_for(m, 256), 256, 0, st, a, m);
    return 0;
}

// BCCP of the medium and big pair lists: one warp per pair.  next: two device counters.
void run_bccp_tiles(TravArgs &a, const int *counts_host, int *next, cudaStream_t st, bool hdb, bool fp64)
{
    cudaMemsetAsync(next, 0, 2 * sizeof(int), st);
    for (int c = 2; c <= 3; ++c) {
        const int m = counts_host[c];
        if (m <= 0) continue;
        const int grid = (int)std::min<long long>((long long)num_sms() * 4, ((long long)m + 7) / 8);
        const int2 *pl = a.list[c];
        const float *pb = a.list_lb[c];
        int *nx = next + (c - 2);
        const int chunk = (long long)m > 128LL * grid * 8 ? 4 : 1;   // long lists: fewer counter increments
#define WM_TILE(DV)                                                                                    \
    do {                                                                                               \
        if (fp64) {                                                                                    \
            if (hdb) launch(bccp_pair_tile_kernel<DV, true, true>, grid, 256, 0, st, a, pl, pb, m, nx, chunk);   \
            else launch(bccp_pair_tile_kernel<DV, false, true>, grid, 256, 0, st, a, pl, pb, m, nx, chunk);      \
        } else {                                                                                       \
            if (hdb) launch(bccp_pair_tile_kernel<DV, true, false>, grid, 256, 0, st, a, pl, pb, m, nx, chunk);  \
            else launch(bccp_pair_tile_kernel<DV, false, false>, grid, 256, 0, st, a, pl, pb, m, nx, chunk);     \
        }                                                                                              \
    } while (0)
        switch (a.d) {
        case 2: WM_TILE(2); break;
        case 3: WM_TILE(3); break;
        case 5: WM_TILE(5); break;
        case 7: WM_TILE(7); break;
        default: WM_TILE(0); break;
        }
#undef WM_TILE
    }
}

}  // namespace wm
