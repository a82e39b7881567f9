// kdtree.cu -- ingest of the input points and the spatial-median k-d tree (Sec. 2.3 "k-d tree";
// Sec. 3.2.1: spatial-median splits down to one point per leaf).
//
// A node splits its tight bounding box at the midpoint of the widest dimension.  If every point
// falls on one side (all points equal, or an extent of one float ulp) the node splits its points
// by count instead, so every leaf holds exactly one point and the tree has 2n-1 nodes.
//
// Build: nodes with more than 32 points are split level by level over the whole GPU; each level
// computes boxes with warp work-units of 256 points, counts the left side, and partitions the
// FP32 coordinates and ids between two ping-pong buffers (a child that leaves the top levels is
// written to the final arrays directly); the FP64 coordinates are gathered once at the end.  A node of 2..32 points is finished by one warp, which
// holds its points in registers and splits recursively with ballots and shuffles.
#include <cstring>
#include <utility>

#include "wm_internal.cuh"

namespace wm {

namespace {

// ---------------------------------------------------------------------------------- ingest
__global__ void ingest_kernel(const void *__restrict__ src, int n, int d, int dtype, int layout,
                              float *__restrict__ x32, double *__restrict__ x64, int *__restrict__ pid,
                              unsigned *__restrict__ bad, unsigned *__restrict__ delta_bits)
{
    float dmax = 0.f;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)n * d;
         t += (long long)gridDim.x * blockDim.x) {
        // t indexes the SoA output: k = t / n, i = t % n
        int k = (int)(t / n), i = (int)(t % n);
        size_t sidx = layout == WM_SOA ? (size_t)t : (size_t)i * d + k;
        double v;
        float f;
        if (dtype == WM_F32) {
            f = ((const float *)src)[sidx];
            v = (double)f;
        } else {
            v = ((const double *)src)[sidx];
            f = __double2float_rn(v);
            float e = (float)fabs(v - (double)f);
            // round the error bound up
            e = __fmul_ru(e, 1.0f + 1.0f / 8388608.0f);
            dmax = fmaxf(dmax, e);
        }
        if (!isfinite(v) || fabs(v) > 1152921504606846976.0) atomicOr(bad, 1u);
        x32[t] = f;
        x64[t] = v;
        if (k == 0) pid[i] = i;
    }
    for (int o = 16; o; o >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    if ((threadIdx.x & 31) == 0 && dmax > 0.f) atomicMax(delta_bits, __float_as_uint(dmax));
}

// ------------------------------------------------------------------------ top-level build
constexpr int kUnit = 256;   // points per warp work-unit

struct Level {
    const int *act;      // active node ids (size > 32)
    const int *unit_off; // [A] prefix of work-units per node
    const long long *tot;   // (A << 32) | total work-units, on the device
};

// Per-level scalars kept on the device, so that several levels run between host syncs:
// [0] first node id of the level's children, [1] offset of its small roots in the small list,
// [2] 2 A (length of the child flag arrays), [3] A.
__global__ void level_begin_kernel(const long long *__restrict__ tot, const int *__restrict__ tsmall, int *state)
{
    state[0] += state[2];
    state[1] += *tsmall;
    const int A = (int)(*tot >> 32);
    state[3] = A;
    state[2] = 2 * A;
}

__device__ inline int find_unit_node(const int *__restrict__ unit_off, int A, int u)
{
    int lo = 0, hi = A - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (unit_off[mid] <= u) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ inline void init_node_box(int nd, int N, int d, float *lo, float *hi, int *cnt)
{
    for (int k = 0; k < d; ++k) { lo[(size_t)k * N + nd] = INFINITY; hi[(size_t)k * N + nd] = -INFINITY; }
    cnt[nd] = 0;
}

// the root as the first level's only active node
__global__ void level0_kernel(int n, int N, int d, float *lo, float *hi, int *cnt, int *act, int *unit_off,
                              long long *tot)
{
    init_node_box(0, N, d, lo, hi, cnt);
    act[0] = 0;
    unit_off[0] = 0;
    *tot = (1LL << 32) | (long long)((n + kUnit - 1) / kUnit);
}

// True for the warp whose unit of node nd completed the node's units (one per node and phase);
// the counter is left at 0 for the next phase.  The caller's global writes of the phase precede.
__device__ inline bool last_unit(int *ucnt, int nd, int nunits)
{
    const int lane = threadIdx.x & 31;
    __threadfence();
    int done = 0;
    if (lane == 0) {
        done = atomicAdd(&ucnt[nd], 1) == nunits - 1;
        if (done) ucnt[nd] = 0;
    }
    done = __shfl_sync(0xffffffffu, done, 0);
    if (done) __threadfence();
    return done;
}

// Box of every active node from its units; the unit that completes a node picks the split: the
// midpoint of the widest dimension.
__global__ void box_units_kernel(Level L, const int *__restrict__ nbegin, const int *__restrict__ nend,
                                 const float *__restrict__ x32, int n, int N, int d, float *lo, float *hi, int *ucnt,
                                 int *__restrict__ sdim, float *__restrict__ sval)
{
    const int lane = threadIdx.x & 31;
    const int TU = (int)(*L.tot & 0xffffffffLL), A = (int)(*L.tot >> 32);
    for (int u = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < TU; u += (gridDim.x * blockDim.x) >> 5) {
        int j = find_unit_node(L.unit_off, A, u);
        int nd = L.act[j];
        const int nb = nbegin[nd], ne = nend[nd];
        int b = nb + (u - L.unit_off[j]) * kUnit;
        int e = min(b + kUnit, ne);
        for (int k = 0; k < d; ++k) {
            float mn = INFINITY, mx = -INFINITY;
            for (int i = b + lane; i < e; i += 32) {
                float v = x32[(size_t)k * n + i];
                mn = fminf(mn, v);
                mx = fmaxf(mx, v);
            }
            for (int o = 16; o; o >>= 1) {
                mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
                mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            }
            if (lane == 0) {
                atomicMinF(&lo[(size_t)k * N + nd], mn);
                atomicMaxF(&hi[(size_t)k * N + nd], mx);
            }
        }
        if (last_unit(ucnt, nd, (ne - nb + kUnit - 1) / kUnit) && lane == 0) {
            int best = 0;
            float ext = -1.f;
            for (int k = 0; k < d; ++k) {
                float ee = *(volatile float *)&hi[(size_t)k * N + nd] - *(volatile float *)&lo[(size_t)k * N + nd];
                if (ee > ext) { ext = ee; best = k; }
            }
            float l = *(volatile float *)&lo[(size_t)best * N + nd], h = *(volatile float *)&hi[(size_t)best * N + nd];
            sdim[j] = best;
            sval[j] = l + (h - l) * 0.5f;
        }
    }
}

// Left-side counts from the units; the unit that completes a node creates its two children and
// the flags of the next level's lists: bigu[2j + s] = (child is active) << 32 | its work-units,
// is_small[2j + s] = child has 2..32 points.
__global__ void count_units_kernel(Level L, const int *__restrict__ state, int *nbegin, int *nend, int *nleft, int *nright, int *nparent,
                                   int *__restrict__ ndepth, const float *__restrict__ x32, int n,
                                   const int *__restrict__ sdim, const float *__restrict__ sval, int *cnt, int *ucnt,
                                   int *__restrict__ count_split, long long *__restrict__ bigu,
                                   int *__restrict__ is_small)
{
    const int lane = threadIdx.x & 31;
    const int TU = (int)(*L.tot & 0xffffffffLL), A = (int)(*L.tot >> 32);
    for (int u = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < TU; u += (gridDim.x * blockDim.x) >> 5) {
        int j = find_unit_node(L.unit_off, A, u);
        int nd = L.act[j];
        const int nb = nbegin[nd], ne = nend[nd];
        int b = nb + (u - L.unit_off[j]) * kUnit;
        int e = min(b + kUnit, ne);
        int k = sdim[j];
        float s = sval[j];
        int c = 0;
        for (int i = b + lane; i < e; i += 32) c += x32[(size_t)k * n + i] < s ? 1 : 0;
        for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (lane == 0 && c) atomicAdd(&cnt[nd], c);
        if (last_unit(ucnt, nd, (ne - nb + kUnit - 1) / kUnit) && lane == 0) {
            const int sz = ne - nb;
            int Lc = *(volatile int *)&cnt[nd];
            int cs = 0;
            if (Lc == 0 || Lc == sz) { Lc = sz / 2; cs = 1; }   // all points on one side: split by count
            count_split[j] = cs;
            cnt[nd] = Lc;
            const int l = state[0] + 2 * j, r = l + 1;
            nleft[nd] = l; nright[nd] = r;
            nbegin[l] = nb; nend[l] = nb + Lc; nbegin[r] = nb + Lc; nend[r] = ne;
            nparent[l] = nd; nparent[r] = nd;
            nleft[l] = nright[l] = nleft[r] = nright[r] = -1;
            ndepth[l] = ndepth[r] = ndepth[nd] + 1;
            const int sl = Lc, sr = sz - Lc;
            bigu[2 * j] = sl > 32 ? (1LL << 32) | (long long)((sl + kUnit - 1) / kUnit) : 0;
            bigu[2 * j + 1] = sr > 32 ? (1LL << 32) | (long long)((sr + kUnit - 1) / kUnit) : 0;
            is_small[2 * j] = sl > 1 && sl <= 32;
            is_small[2 * j + 1] = sr > 1 && sr <= 32;
        }
    }
}

// The next level's lists from the flags and their prefixes; a new active node gets its work-unit
// offset and an empty box.
__global__ void next_level_kernel(const long long *__restrict__ bigu, const long long *__restrict__ prebigu,
                                  const int *__restrict__ is_small, const int *__restrict__ presmall,
                                  const int *__restrict__ state, int N, int d, int *__restrict__ act,
                                  int *__restrict__ unit_off, int *__restrict__ small, float *lo, float *hi, int *cnt)
{
    const int m = state[2], next_id = state[0];
    small += state[1];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        const int id = next_id + i;
        if (bigu[i]) {
            const long long pre = prebigu[i];
            const int k = (int)(pre >> 32);
            act[k] = id;
            unit_off[k] = (int)(pre & 0xffffffffLL);
            init_node_box(id, N, d, lo, hi, cnt);
        }
        if (is_small[i]) small[presmall[i]] = id;
    }
}

// Partition of each active node's points by its split.  The points of a child that stays active
// (more than 32 points) go to the other ping-pong buffer (w32, wpid); those of a child that leaves
// the top levels go straight to their final place (f32, fpid), which no active node reads.
__global__ void scatter_units_kernel(Level L, const int *__restrict__ nbegin,
                                     const int *__restrict__ nend, const float *__restrict__ x32,
                                     const int *__restrict__ pid, int n, int d, const int *__restrict__ sdim,
                                     const float *__restrict__ sval, const int *__restrict__ count_split,
                                     const int *__restrict__ cnt, int *__restrict__ curl, int *__restrict__ curr,
                                     float *__restrict__ w32, int *__restrict__ wpid, float *__restrict__ f32,
                                     int *__restrict__ fpid)
{
    const int lane = threadIdx.x & 31;
    const int TU = (int)(*L.tot & 0xffffffffLL), A = (int)(*L.tot >> 32);
    for (int u = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < TU; u += (gridDim.x * blockDim.x) >> 5) {
        int j = find_unit_node(L.unit_off, A, u);
        int nd = L.act[j];
        int nb = nbegin[nd], ne = nend[nd];
        int b = nb + (u - L.unit_off[j]) * kUnit;
        int e = min(b + kUnit, ne);
        int k = sdim[j];
        float s = sval[j];
        int cs = count_split[j];
        int Lc = cnt[nd];
        const bool lbig = Lc > 32, rbig = ne - nb - Lc > 32;
        for (int i0 = b; i0 < e; i0 += 32) {
            int i = i0 + lane;
            bool valid = i < e;
            int dst = i;
            bool fl;
            if (!cs) {
                fl = valid && x32[(size_t)k * n + i] < s;
                unsigned bl = __ballot_sync(0xffffffffu, fl);
                unsigned br = __ballot_sync(0xffffffffu, valid && !fl);
                int bsl = 0, bsr = 0;
                if (lane == 0) {
                    if (bl) bsl = atomicAdd(&curl[nd], __popc(bl));
                    if (br) bsr = atomicAdd(&curr[nd], __popc(br));
                }
                bsl = __shfl_sync(0xffffffffu, bsl, 0);
                bsr = __shfl_sync(0xffffffffu, bsr, 0);
                if (fl) dst = nb + bsl + __popc(bl & lanemask_lt());
                else dst = nb + Lc + bsr + __popc(br & lanemask_lt());
            } else {
                fl = i < nb + Lc;
            }
            if (valid) {
                const bool big = fl ? lbig : rbig;
                float *o32 = big ? w32 : f32;
                for (int kk = 0; kk < d; ++kk) o32[(size_t)kk * n + dst] = x32[(size_t)kk * n + i];
                (big ? wpid : fpid)[dst] = pid[i];
            }
        }
    }
}

// FP64 coordinates in tree order: x64[k][p] = src[k][pid[p]]
__global__ void gather64_kernel(const double *__restrict__ src, const int *__restrict__ pid, int n, int d,
                                double *__restrict__ x64)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)n * d;
         t += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(t / n), p = (int)(t % n);
        x64[t] = src[(size_t)k * n + pid[p]];
    }
}

// ------------------------------------------------------------------ warp-local small subtrees
// float <-> unsigned key of the same order, for the warp min/max reductions on integers
__device__ inline unsigned f2key(float f)
{
    const unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : u | 0x80000000u;
}
__device__ inline float key2f(unsigned k) { return __uint_as_float((k & 0x80000000u) ? k & 0x7fffffffu : ~k); }

// One warp per node of 2..32 points.  Node ids of the subtree: base + 0 .. base + 2m - 3.  The
// points stay in registers (lane = position in the node's range); a split permutes them through
// the warp's shared-memory slots.
template <int DM>
__global__ void __launch_bounds__(256) small_subtree_kernel(const int *__restrict__ small,
                                                            const int *__restrict__ small_base, int S, int *nbegin,
                                                            int *nend, int *nleft, int *nright, int *nparent,
                                                            int *ndepth, float *lo, float *hi, float *x32, int *pid,
                                                            int n, int N, int d, int *max_depth)
{
    __shared__ float shx[8][DM * 32];
    __shared__ int shid[8][32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (wid >= S) return;
    float *sx = shx[wib];
    int *sid = shid[wib];
    const int root = small[wid];
    int next = small_base[wid];
    const int b0 = nbegin[root];
    const int m = nend[root] - b0;
    float c32[DM];
    int myid = -1;
#pragma unroll
    for (int k = 0; k < DM; ++k) c32[k] = 0.f;
    if (lane < m) {
#pragma unroll
        for (int k = 0; k < DM; ++k)
            if (k < d) c32[k] = x32[(size_t)k * n + b0 + lane];
        myid = pid[b0 + lane];
    }
    // explicit stack of (lo_lane, hi_lane, node)
    int st_lo[32], st_hi[32], st_nd[32];
    int sp = 0;
    st_lo[0] = 0; st_hi[0] = m; st_nd[0] = root; sp = 1;
    int mdepth = 0;
    while (sp > 0) {
        --sp;
        int rl = st_lo[sp], rh = st_hi[sp], nd = st_nd[sp];
        int sz = rh - rl;
        bool in = lane >= rl && lane < rh;
        int dep = ndepth[nd];
        mdepth = max(mdepth, dep);
        // box over the lanes in range
        int best = 0;
        float ext = -1.f, bl = 0.f, bh = 0.f, cv = 0.f;
#pragma unroll
        for (int k = 0; k < DM; ++k) {
            if (k >= d) break;
            const unsigned key = f2key(c32[k]);
            const float mn = key2f(__reduce_min_sync(0xffffffffu, in ? key : 0xffffffffu));
            const float mx = key2f(__reduce_max_sync(0xffffffffu, in ? key : 0u));
            if (lane == 0) { lo[(size_t)k * N + nd] = mn; hi[(size_t)k * N + nd] = mx; }
            if (mx - mn > ext) { ext = mx - mn; best = k; bl = mn; bh = mx; cv = c32[k]; }
        }
        if (sz == 1) continue;   // leaf: box = the point
        float sv = bl + (bh - bl) * 0.5f;
        bool fl = in && cv < sv;
        unsigned bal = __ballot_sync(0xffffffffu, fl);
        int Lc = __popc(bal);
        bool cs = (Lc == 0 || Lc == sz);
        if (cs) { Lc = sz / 2; fl = in && (lane - rl) < Lc; bal = __ballot_sync(0xffffffffu, fl); }
        unsigned bar = __ballot_sync(0xffffffffu, in && !fl);
        if (!cs) {
            // permute the lanes in range: this lane's point moves to position dst
            const int dst = fl ? rl + __popc(bal & lanemask_lt()) : rl + Lc + __popc(bar & lanemask_lt());
            if (in) {
#pragma unroll
                for (int k = 0; k < DM; ++k)
                    if (k < d) sx[k * 32 + dst] = c32[k];
                sid[dst] = myid;
            }
            __syncwarp();
            if (in) {
#pragma unroll
                for (int k = 0; k < DM; ++k)
                    if (k < d) c32[k] = sx[k * 32 + lane];
                myid = sid[lane];
            }
            __syncwarp();
        }
        int l = next, r = next + 1;
        next += 2;
        if (lane == 0) {
            nleft[nd] = l; nright[nd] = r;
            nbegin[l] = b0 + rl; nend[l] = b0 + rl + Lc;
            nbegin[r] = b0 + rl + Lc; nend[r] = b0 + rh;
            nparent[l] = nd; nparent[r] = nd;
            nleft[l] = nright[l] = nleft[r] = nright[r] = -1;
            ndepth[l] = ndepth[r] = dep + 1;
        }
        __syncwarp();
        // push right then left (left processed first)
        st_lo[sp] = rl + Lc; st_hi[sp] = rh; st_nd[sp] = r; ++sp;
        st_lo[sp] = rl; st_hi[sp] = rl + Lc; st_nd[sp] = l; ++sp;
    }
    if (lane < m) {
#pragma unroll
        for (int k = 0; k < DM; ++k)
            if (k < d) x32[(size_t)k * n + b0 + lane] = c32[k];
        pid[b0 + lane] = myid;
    }
    if (lane == 0) atomicMax(max_depth, mdepth);
}

// Leaves created by the top levels (single points): box = the point.  Then widen every box by
// delta (rounding outward) and store the rigorous diameter bound.
__global__ void finish_boxes_kernel(int N, int n, int d, const int *__restrict__ nbegin, const int *__restrict__ nleft,
                                    const float *__restrict__ x32, float *lo, float *hi, float delta,
                                    float *__restrict__ diam2, const int *__restrict__ ndepth, int *max_depth)
{
    int dmax = 0;
    for (int nd = blockIdx.x * blockDim.x + threadIdx.x; nd < N; nd += gridDim.x * blockDim.x) {
        bool leaf = nleft[nd] < 0;
        float s = 0.f;
        for (int k = 0; k < d; ++k) {
            float l, h;
            if (leaf) { l = h = x32[(size_t)k * n + nbegin[nd]]; }
            else { l = lo[(size_t)k * N + nd]; h = hi[(size_t)k * N + nd]; }
            if (delta > 0.f) { l = __fsub_rd(l, delta); h = __fadd_ru(h, delta); }
            lo[(size_t)k * N + nd] = l;
            hi[(size_t)k * N + nd] = h;
            float e = __fsub_ru(h, l);
            s = __fmaf_ru(e, e, s);
        }
        diam2[nd] = upper_w2(s);
        dmax = max(dmax, ndepth[nd]);
    }
    for (int o = 16; o; o >>= 1) dmax = max(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    if ((threadIdx.x & 31) == 0) atomicMax(max_depth, dmax);
}

// Tighter diameter bounds.  The box diagonal can be far above the largest distance between the
// points of a node, most of all in high dimension, where a few points set the box's extent in each
// coordinate, and a smaller bound lets node pairs pass the geometric separation test of the WSPD
// higher up the tree (fewer, larger pairs).  Any rigorous upper bound of the diameter keeps the
// MST argument valid, so every internal node takes the smallest of
//   - its box diagonal (finish_boxes_kernel),
//   - m <= 32 points: the largest pairwise distance of its points,
//   - m > 32: 2 r, r an upper bound of the distance from the box centre c to any of its points;
//     for m <= kDiamDirect r is found from the points, above it from the children's radii
//     (every point of child i is within r_i + |c - c_i| of c), bottom-up.
// Point distances are evaluated in FP32 (relative error <= 2^-19 for exactly representable
// operands, covered by the 2^-18 margin) and widened by the FP32 copy's absolute error delta per
// coordinate into bounds on the FP64 points; the centre distances in FP64 with a margin.
constexpr int kDiamDirect = 4096;

template <int DM>
__global__ void __launch_bounds__(256) tight_diam_kernel(int N, int n, int d, const int *__restrict__ nbegin,
                                                         const int *__restrict__ nend, const int *__restrict__ nleft,
                                                         const float *__restrict__ x32, const float *__restrict__ lo,
                                                         const float *__restrict__ hi, float delta,
                                                         float *__restrict__ diam2, float *__restrict__ rad)
{
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const double dsq = (double)delta * sqrt((double)d) * (1.0 + 1e-6);
    // a warp reads the records of 32 consecutive nodes and then works through those with
    // 3..kDiamDirect points together (a leaf's radius is only needed for composition above
    // kDiamDirect points, and two points' box diagonal is already their distance)
    for (int base = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; base < N; base += nw * 32) {
        const int mine = base + lane;
        int mb = 0, mm = 0;
        if (mine < N && nleft[mine] >= 0) {
            mb = nbegin[mine];
            mm = nend[mine] - mb;
        }
        unsigned todo = __ballot_sync(0xffffffffu, mm >= 3 && mm <= kDiamDirect);
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1;
            const int nd = base + src;
            const int b = __shfl_sync(0xffffffffu, mb, src), m = __shfl_sync(0xffffffffu, mm, src);
            float c[DM];
#pragma unroll
            for (int k = 0; k < DM; ++k) c[k] = k < d ? 0.5f * (lo[(size_t)k * N + nd] + hi[(size_t)k * N + nd]) : 0.f;
            float mr = 0.f;
            for (int i = b + lane; i < b + m; i += 32) {
                float s = 0.f;
#pragma unroll
                for (int k = 0; k < DM; ++k) {
                    if (k < d) {
                        const float t = x32[(size_t)k * n + i] - c[k];
                        s = fmaf(t, t, s);
                    }
                }
                mr = fmaxf(mr, s);
            }
            for (int o = 16; o; o >>= 1) mr = fmaxf(mr, __shfl_xor_sync(0xffffffffu, mr, o));
            const double r = sqrt((double)mr * (1.0 + 1.0 / 262144.0)) * (1.0 + 1e-12) + dsq;
            double bound = 4.0 * r * r;
            if (m <= 32) {
                float p[DM];
#pragma unroll
                for (int k = 0; k < DM; ++k) p[k] = (k < d && lane < m) ? x32[(size_t)k * n + b + lane] : 0.f;
                float mx = 0.f;
                for (int j = 1; j < m; ++j) {
                    float s = 0.f;
#pragma unroll
                    for (int k = 0; k < DM; ++k) {
                        if (k < d) {
                            const float t = p[k] - __shfl_sync(0xffffffffu, p[k], j);
                            s = fmaf(t, t, s);
                        }
                    }
                    if (lane < j) mx = fmaxf(mx, s);
                }
                for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
                const double q = sqrt((double)mx * (1.0 + 1.0 / 262144.0)) * (1.0 + 1e-12) + 2.0 * dsq;
                bound = fmin(bound, q * q);
            }
            if (lane == 0) {
                rad[nd] = __double2float_ru(r);
                const float f = __double2float_ru(bound * (1.0 + 1.0 / 1099511627776.0) + 1e-300);
                if (f < diam2[nd]) diam2[nd] = f;
            }
        }
    }
}

// Radii of the nodes above kDiamDirect points, bottom-up with arrival counters: each node whose
// parent is above the limit starts a climb; the second child to arrive at a parent composes it.
__global__ void diam_up_kernel(int N, int d, const int *__restrict__ nbegin, const int *__restrict__ nend,
                               const int *__restrict__ nleft, const int *__restrict__ nright,
                               const int *__restrict__ nparent, const float *__restrict__ lo,
                               const float *__restrict__ hi, float *diam2, float *rad, int *arrive)
{
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < N; x += gridDim.x * blockDim.x) {
        const int px = nparent[x];
        if (nend[x] - nbegin[x] > kDiamDirect || px < 0 || nend[px] - nbegin[px] <= kDiamDirect) continue;
        int cur = x;
        for (int it = 0; it < 128; ++it) {   // at most the tree depth
            const int p = nparent[cur];
            if (p < 0) break;
            __threadfence();
            if (atomicAdd(&arrive[p], 1) == 0) break;   // the sibling composes the parent
            __threadfence();
            double r = 0.0;
            for (int side = 0; side < 2; ++side) {
                const int ch = side ? nright[p] : nleft[p];
                double cc = 0.0;
                for (int k = 0; k < d; ++k) {
                    const double cp = 0.5 * ((double)lo[(size_t)k * N + p] + (double)hi[(size_t)k * N + p]);
                    const double ci = 0.5 * ((double)lo[(size_t)k * N + ch] + (double)hi[(size_t)k * N + ch]);
                    const double t = cp - ci;
                    cc += t * t;
                }
                // nodes of one or two points have no radius of their own: every point lies in the
                // box, within half its (rounded-up) diagonal of the centre
                const double rc = nend[ch] - nbegin[ch] < 3 ? 0.5 * sqrt((double)diam2[ch]) * (1.0 + 1e-12)
                                                             : (double)((volatile float *)rad)[ch];
                r = fmax(r, (sqrt(cc) * (1.0 + 1e-12) + rc) * (1.0 + 1e-12));
            }
            rad[p] = __double2float_ru(r);
            const float f = __double2float_ru(4.0 * r * r * (1.0 + 1.0 / 1099511627776.0) + 1e-300);
            if (f < diam2[p]) diam2[p] = f;
            cur = p;
        }
    }
}

__global__ void inverse_perm_kernel(const int *__restrict__ pid, int *__restrict__ pos, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) pos[pid[i]] = i;
}

__global__ void small_sizes_kernel(const int *small, int S, const int *nbegin, const int *nend, int *out)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < S) out[j] = 2 * (nend[small[j]] - nbegin[small[j]]) - 2;
}

__global__ void add_const_kernel(int *p, int m, int c)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < m) p[j] += c;
}

}  // namespace

// --------------------------------------------------------------------------- host drivers

int ingest_points(const void *dev_src, int n, int d, int dtype, int layout, Points &P, Arena &ar,
                  cudaStream_t st, unsigned *pinned)
{
    P.n = n; P.d = d;
    P.x32 = ar.get<float>((size_t)n * d);
    P.x64 = ar.get<double>((size_t)n * d);
    P.pid = ar.get<int>(n);
    P.pos = ar.get<int>(n);
    unsigned *flags = ar.get<unsigned>(2);
    if (ar.failed) return WM_ENOMEM;
    cudaMemsetAsync(flags, 0, 2 * sizeof(unsigned), st);
    launch(ingest_kernel, grid_for((long long)n * d, 256), 256, 0, st, dev_src, n, d, dtype, layout, P.x32, P.x64, P.pid,
                                                                     flags, flags + 1);
    cudaMemcpyAsync(pinned, flags, 2 * sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return WM_ECUDA;
    if (pinned[0]) return WM_EINVAL;
    unsigned db = pinned[1];
    float dl;
    memcpy(&dl, &db, sizeof(float));
    P.delta = dl;
    return 0;
}

int build_tree(Points &P, Tree &T, Arena &ar, cudaStream_t st, int *pinned, bool tight_diameters)
{
    const int n = P.n, d = P.d;
    const int N = 2 * n - 1;
    T.N = N;
    T.lo = ar.get<float>((size_t)N * d);
    T.hi = ar.get<float>((size_t)N * d);
    T.begin = ar.get<int>(N);
    T.end = ar.get<int>(N);
    T.left = ar.get<int>(N);
    T.right = ar.get<int>(N);
    T.parent = ar.get<int>(N);
    T.diam2 = ar.get<float>(N);
    T.comp = ar.get<int>(N);
    T.arrive = ar.get<int>(N);
    int *depth = ar.get<int>(N);
    int *maxdep = ar.get<int>(1);
    // final (tree-order) point arrays; the ingest arrays (input order) become the first
    // ping-pong buffer of the top levels
    float *f32 = ar.get<float>((size_t)n * d);
    int *fpid = ar.get<int>(n);
    double *f64 = ar.get<double>((size_t)n * d);
    if (ar.failed) return WM_ENOMEM;
    // root
    int h0[6] = {0, n, -1, -1, -1, 0};
    cudaMemcpyAsync(T.begin, &h0[0], sizeof(int), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(T.end, &h0[1], sizeof(int), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(T.left, &h0[2], sizeof(int), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(T.right, &h0[3], sizeof(int), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(T.parent, &h0[4], sizeof(int), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(depth, &h0[5], sizeof(int), cudaMemcpyHostToDevice, st);
    cudaMemsetAsync(maxdep, 0, sizeof(int), st);

    size_t mark = ar.off;
    // scratch
    int *act = ar.get<int>(n / 16 + 2), *act2 = ar.get<int>(n / 16 + 2);
    int *uoff = ar.get<int>(n / 16 + 2), *uoff2 = ar.get<int>(n / 16 + 2);
    long long *tot = ar.get<long long>(2);
    int *tsmall = ar.get<int>(2), *lstate = ar.get<int>(4);
    int *sdim = ar.get<int>(n / 16 + 2);
    float *sval = ar.get<float>(n / 16 + 2);
    int *csplit = ar.get<int>(n / 16 + 2);
    long long *bigu = ar.get<long long>(n / 8 + 4), *prebigu = ar.get<long long>(n / 8 + 4);
    int *issmall = ar.get<int>(n / 8 + 4), *presmall = ar.get<int>(n / 8 + 4);
    int *cnt = ar.get<int>(N), *curl = ar.get<int>(N), *curr = ar.get<int>(N), *ucnt = ar.get<int>(N);
    int *small = ar.get<int>(n / 2 + 2), *small_sz = ar.get<int>(n / 2 + 2), *small_base = ar.get<int>(n / 2 + 2);
    float *t32 = ar.get<float>((size_t)n * d);
    int *tpid = ar.get<int>(n);
    if (ar.failed) return WM_ENOMEM;
    float *r32 = P.x32, *w32 = t32;   // level buffers: read, write
    int *rpid = P.pid, *wpid = tpid;

    int A = 0, S = 0, next_id = 1;
    if (n > 32) {
        launch(level0_kernel, 1, 1, 0, st, n, N, d, T.lo, T.hi, cnt, act, uoff, tot);
        A = 1;
    } else if (n > 1) {
        cudaMemsetAsync(small, 0, sizeof(int), st);
        S = 1;
    }
    if (A == 0) {   // no top level: the points go to their final arrays as they are
        cudaMemcpyAsync(f32, P.x32, sizeof(float) * n * d, cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(fpid, P.pid, sizeof(int) * n, cudaMemcpyDeviceToDevice, st);
    }
    cudaMemsetAsync(curl, 0, sizeof(int) * N, st);
    cudaMemsetAsync(curr, 0, sizeof(int) * N, st);
    cudaMemsetAsync(ucnt, 0, sizeof(int) * N, st);
    {
        const int init[4] = {1, 0, 0, 0};   // pageable source: copied before the call returns
        cudaMemcpyAsync(lstate, init, sizeof init, cudaMemcpyHostToDevice, st);
        cudaMemsetAsync(tsmall, 0, sizeof(int), st);
    }
    // Levels run kLevelsPerSync at a time with their counts on the device; the host sizes the
    // launches from a bound on A (at most doubling per level, at most n / 33) and learns the
    // real A at each sync.  Levels after the last active one find A = 0 and do nothing.
    constexpr int kLevelsPerSync = 4;
    const int amax = n / 33 + 1;
    long long *tcur = tot, *tnext = tot + 1;
    int abound = A;
    while (A > 0) {
        for (int g = 0; g < kLevelsPerSync; ++g) {
            launch(level_begin_kernel, 1, 1, 0, st, tcur, tsmall, lstate);
            const Level L{act, uoff, tcur};
            const int gw = num_sms() * 8;   // blocks of 256 threads, 8 warps each
            launch(box_units_kernel, gw, 256, 0, st, L, T.begin, T.end, r32, n, N, d, T.lo, T.hi, ucnt, sdim, sval);
            launch(count_units_kernel, gw, 256, 0, st, L, lstate, T.begin, T.end, T.left, T.right, T.parent, depth, r32,
                                                    n, sdim, sval, cnt, ucnt, csplit, bigu, issmall);
            launch(scatter_units_kernel, gw, 256, 0, st, L, T.begin, T.end, r32, rpid, n, d, sdim, sval, csplit, cnt,
                                                      curl, curr, w32, wpid, f32, fpid);
            std::swap(r32, w32);
            std::swap(rpid, wpid);
            // next lists
            int rc = scan_exclusive_i64_dev(bigu, prebigu, lstate + 2, 2 * abound, tnext, st, ar);
            if (rc) return rc;
            rc = scan_exclusive_i32_dev(issmall, presmall, lstate + 2, 2 * abound, tsmall, st, ar);
            if (rc) return rc;
            launch(next_level_kernel, grid_for(2 * abound, 256, 1 << 20), 256, 0, st, bigu, prebigu, issmall, presmall,
                                                                                 lstate, N, d, act2, uoff2, small, T.lo,
                                                                                 T.hi, cnt);
            std::swap(act, act2);
            std::swap(uoff, uoff2);
            std::swap(tcur, tnext);
            abound = std::min(2 * abound, amax);
        }
        cudaMemcpyAsync(pinned, tcur, sizeof(long long), cudaMemcpyDeviceToHost, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) return WM_ECUDA;
        long long tn;
        memcpy(&tn, pinned, sizeof tn);
        A = (int)(tn >> 32);
        abound = A;
    }
    if (n > 32) {
        // fold the last level's children and small roots into the totals
        launch(level_begin_kernel, 1, 1, 0, st, tcur, tsmall, lstate);
        cudaMemcpyAsync(pinned, lstate, 2 * sizeof(int), cudaMemcpyDeviceToHost, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) return WM_ECUDA;
        next_id = pinned[0];
        S = pinned[1];
    }
    // sizes of the small roots and their node-id bases
    if (S > 0) {
        launch(small_sizes_kernel, grid_for(S, 256, 1 << 20), 256, 0, st, small, S, T.begin, T.end, small_sz);
        int rc = scan_exclusive_i32(small_sz, small_base, S, tsmall + 1, st, ar);
        if (rc) return rc;
        launch(add_const_kernel, grid_for(S, 256, 1 << 20), 256, 0, st, small_base, S, next_id);
        int blocks = (S + 7) / 8;
#define WM_SMALL(DM) launch(small_subtree_kernel<DM>, blocks, 256, 0, st, small, small_base, S, T.begin, T.end, T.left, \
        T.right, T.parent, depth, T.lo, T.hi, f32, fpid, n, N, d, maxdep)
        if (d <= 2) WM_SMALL(2);
        else if (d <= 3) WM_SMALL(3);
        else if (d <= 4) WM_SMALL(4);
        else if (d <= 5) WM_SMALL(5);
        else if (d <= 8) WM_SMALL(8);
        else WM_SMALL(16);
#undef WM_SMALL
    }
    if (n == 1) {
        int m1 = -1;
        cudaMemcpyAsync(T.left, &m1, sizeof(int), cudaMemcpyHostToDevice, st);
    }
    launch(gather64_kernel, grid_for((long long)n * d, 256), 256, 0, st, P.x64, fpid, n, d, f64);
    P.x32 = f32;
    P.pid = fpid;
    P.x64 = f64;
    launch(finish_boxes_kernel, grid_for(N, 256), 256, 0, st, N, n, d, T.begin, T.left, P.x32, T.lo, T.hi, P.delta, T.diam2,
                                                         depth, maxdep);
    if (tight_diameters) {
        // a warp handles 32 consecutive nodes per iteration
        const int blocks = (int)std::min<long long>(((long long)N + 255) / 256, (long long)num_sms() * 16);
        float *rad = ar.get<float>(N);
        if (!rad) return WM_ENOMEM;
#define WM_TD(DM) launch(tight_diam_kernel<DM>, blocks, 256, 0, st, N, n, d, T.begin, T.end, T.left, P.x32, T.lo, T.hi, \
                         P.delta, T.diam2, rad)
        if (d <= 2) WM_TD(2);
        else if (d <= 3) WM_TD(3);
        else if (d <= 4) WM_TD(4);
        else if (d <= 5) WM_TD(5);
        else if (d <= 8) WM_TD(8);
        else WM_TD(16);
#undef WM_TD
        if (n > kDiamDirect) {
            cudaMemsetAsync(T.arrive, 0, sizeof(int) * N, st);
            launch(diam_up_kernel, grid_for(N, 256), 256, 0, st, N, d, T.begin, T.end, T.left, T.right, T.parent, T.lo,
                   T.hi, T.diam2, rad, T.arrive);
        }
    }
    launch(inverse_perm_kernel, grid_for(n, 256, 1 << 20), 256, 0, st, P.pid, P.pos, n);
    cudaMemcpyAsync(pinned, maxdep, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return WM_ECUDA;
    T.depth = pinned[0] + 1;
    ar.off = mark;   // release build scratch
    return 0;
}

}  // namespace wm
