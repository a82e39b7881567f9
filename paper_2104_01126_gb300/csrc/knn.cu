// knn.cu -- core distances for HDBSCAN* (Sec. 2.1: cd(p) = distance to the minPts-th nearest
// neighbour, p itself counted; Sec. 2.3 / 3.1.3: computed with k-NN queries, k = minPts), the
// per-node cd_min / cd_max bounds (Table 1) and the repair edges that make the returned MST the
// canonical one under the key K.
//
// k-NN: one warp answers 32 consecutive tree positions (spatially close queries) with a shared
// depth-first traversal of the k-d tree.  A subtree of at most 32 points is scanned directly:
// its points are loaded once and broadcast with shuffles.  Each lane keeps the KL = minPts + 8
// smallest screened values in a sorted list in shared memory (slot-major, one bank per lane).
// A node is skipped for a lane when its box is provably farther than the lane's KL-th value.
// FP32 screen: the k-th screened value s_k gives the band threshold T(s_k); when the list
// provably holds every point with screened value <= T (its KL-th value exceeds T), those
// candidates are re-evaluated in FP64 and sorted, giving the exact k-th squared distance.  A
// query whose band overflows the list (ties, duplicates) is answered by an exact FP64 scan.
//
// Repair edges: R = {(p,q), q != p : w2(p,q) <= cd2(p)}, weighted by the mutual reachability
// distance.  Under general position every edge of the K-minimum spanning tree of G_MR either has
// a weight no other edge has (then every MST contains it, the WSPD-derived candidates too) or has
// d(p,q) <= max(cd(p), cd(q)) (then it is in R); adding R to the MemoGFK batches of their weight
// range therefore yields the K-minimum tree itself.
#include <algorithm>
#include <cstring>
#include <type_traits>

#include "hdb.cuh"
#include "wspd.cuh"

namespace wm {

namespace {

struct KnnArgs {
    int N, n, d, k, KL;
    const float *lo, *hi;
    const int *begin, *end, *left, *right;
    const NodeRec *rec;  // packed node records (right child = left + 1)
    const float *box;    // packed boxes, 2 DMP floats per node (DMP = d rounded up to 4, 8, 16) in groups of
                         // four dimensions: lo[4c..4c+3], hi[4c..4c+3]
    const float *x32;
    const double *x64;
    double eta;
    int stack_cap;       // entries of a warp's traversal stack (in shared memory): depth + 4
    double *wscratch;    // [warps][KL][32] FP64 candidate values
    double *cd64;
    float *cd32;
    int *rep_q;          // [n][KL-1] tree positions
    double *rep_d;       // [n][KL-1] FP64 squared distances
    int *rep_cnt;        // [n]
    int *slow;           // slow query list
    int *slow_cnt;
    int *next_group;     // dispenser of 32-query groups
    int *err;            // set when a traversal stack would overflow (an internal error)
    unsigned long long *stat;   // [0] evals, [1] fp64 rechecks, [2] bits of the largest relative
                                //     error of a screened k-th value against the exact one
};

__device__ inline double d64(const double *__restrict__ x64, int n, int d, int i, int j)
{
    double s = 0.0;
    for (int k = 0; k < d; ++k) {
        double t = __dsub_rn(x64[(size_t)k * n + i], x64[(size_t)k * n + j]);
        s = __dadd_rn(s, __dmul_rn(t, t));
    }
    return s;
}

__device__ inline float knn_threshold(float s, double eta)
{
    double t;
    if (eta == 0.0) {
        t = (double)s * (1.0 + 4.0 * kEps32) + 1.5e-42;
    } else {
        double r = sqrt((double)s * (1.0 + 2.0 * kEps32)) + eta;
        double U = r * r * (1.0 + 2.0 * kGam64);
        double q = sqrt(U * (1.0 + 2.0 * kGam64)) + eta;
        t = q * q * (1.0 + 2.0 * kEps32) + 1.5e-42;
    }
    return __double2float_ru(t);
}

// Upper bound of knn_threshold(s, 0) in FP32 with directed rounding: s (1 + 2^-17) + 1.6e-42, both
// steps rounded up (1.6e-42 as a float exceeds 1.5e-42).  Any float >= the exact threshold is
// >= its rounded-up value as well, so it can stand in for it as a pruning bound.
__device__ inline float knn_threshold_fast(float s)
{
    return __fadd_ru(__fmul_ru(s, 1.0f + 4.0f / 524288.0f), 1.6e-42f);
}

// coordinates per leaf point in the shared-memory broadcast buffer (d rounded up to 4, 8 or 16:
// the stride of the packed boxes as well)
template <int DM> constexpr int knn_dmp() { return DM <= 4 ? 4 : DM <= 8 ? 8 : 16; }

// shared memory of one warp of the k-NN kernel: leaf points, screened lists, indices, stack,
// rounded up to 16 bytes so that the next warp's region starts float4-aligned
__host__ __device__ inline size_t knn_warp_smem(int dmp, int KL, size_t vsize, int stack_cap)
{
    const size_t b = (size_t)32 * dmp * sizeof(float) + (size_t)KL * 32 * (vsize + sizeof(int)) +
                     (size_t)stack_cap * sizeof(int);
    return (b + 15) & ~(size_t)15;
}

template <int DM, bool FP64>
__global__ void __launch_bounds__(256) knn_fast_kernel(KnnArgs a)
{
    using V = typename std::conditional<FP64, double, float>::type;
    extern __shared__ unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nwb = blockDim.x >> 5;
    const int KL = a.KL;
    // per-warp shared region: float4 leaf[32][DMP/4] (the scanned subtree's points, read as
    // broadcasts); V sv[KL][32]; int sj[KL][32] (slot-major, one bank per lane); int stk[stack_cap]
    // (the warp's traversal stack); the FP64 candidate values of the epilogue live in global
    // scratch: double sw[KL][32]
    constexpr int DMP = knn_dmp<DM>(), DQ = DMP / 4;
    size_t per_warp = knn_warp_smem(DMP, KL, sizeof(V), a.stack_cap);
    unsigned char *base = smem_raw + per_warp * wib;
    float4 *leaf = (float4 *)base;
    V *sv = (V *)(base + (size_t)32 * DMP * sizeof(float));
    int *sj = (int *)((unsigned char *)sv + (size_t)KL * 32 * sizeof(V));
    int *stk = sj + (size_t)KL * 32;
    const int gw = blockIdx.x * nwb + wib;
    double *sw = a.wscratch + (size_t)gw * KL * 32;
    const int n = a.n, d = a.d;
    const bool exact32 = a.eta == 0.0;   // FP32 copy is exact: threshold in FP32
    unsigned long long n_ev = 0, n_re = 0;
    float kerr = 0.f;   // largest relative error of a screened k-th value (FP32 screen)
    // 32-query groups handed out dynamically: their costs differ too much for a static deal
    while (true) {
        int q0 = 0;
        if (lane == 0) q0 = atomicAdd(a.next_group, 32);
        q0 = __shfl_sync(0xffffffffu, q0, 0);
        if (q0 >= n) break;
        const int i = q0 + lane;
        const bool valid = i < n;
        float qx[DMP];
        double qx64[DM];
#pragma unroll
        for (int k = 0; k < DMP; ++k) qx[k] = k < d && valid ? a.x32[(size_t)k * n + i] : 0.f;
#pragma unroll
        for (int k = 0; k < DM; ++k) {
            if (k < d) {
                if (FP64) qx64[k] = valid ? a.x64[(size_t)k * n + i] : 0.0;
            }
        }
        // the group's centroid orders the children of a visited node (nearer first) without a
        // reduction over the lanes at every node
        float cent[DMP];
        {
            const float nv = (float)__popc(__ballot_sync(0xffffffffu, valid));
#pragma unroll
            for (int k = 0; k < DMP; ++k) {
                float v = valid ? qx[k] : 0.f;
                for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                cent[k] = v / nv;
            }
        }
        int cnt = 0;
        V thr = (V)INFINITY;   // KL-th kept value (list full) or +inf
        // cut: the band threshold of the current k-th value; a point screened above it can never
        // be a candidate, and a node is skipped when its box bound exceeds cut (1 + 2^-17)
        // (the bound is a rigorous lower bound of the true distance and a screened value is
        // within 2^-19 of the true one, so every skipped point screens above cut as well).
        // cut only decreases, so the final threshold T(s_k) is below every cut used.
        V cut = (V)INFINITY;
        int sp = 0;
        if (lane == 0) stk[0] = 0;
        sp = 1;
        __syncwarp();
        for (int guard = 0; sp > 0 && guard < 2 * a.N + 2; ++guard) {
            int node = stk[sp - 1];
            __syncwarp();
            --sp;
            const int4 L = a.rec[node].l;
            const int b = L.x, e = L.y;
            // prune test for each lane (packed box: groups of four dimensions, lo then hi, padding 0)
            float lb = 0.f;
            {
                const float4 *bx = (const float4 *)(a.box + (size_t)node * 2 * DMP);
#pragma unroll
                for (int c = 0; c < DQ; ++c) {
                    const float4 l4 = bx[2 * c], h4 = bx[2 * c + 1];
                    const float lv[4] = {l4.x, l4.y, l4.z, l4.w}, hv[4] = {h4.x, h4.y, h4.z, h4.w};
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const float g = fmaxf(fmaxf(lv[r] - qx[4 * c + r], qx[4 * c + r] - hv[r]), 0.f);
                        lb = fmaf(g, g, lb);
                    }
                }
            }
            bool need = valid && (V)lower_w2(lb) <= cut * (V)(1.0f + 1.0f / 131072.0f) &&
                        (cnt < KL || (V)lower_w2(lb) <= thr);
            if (!__any_sync(0xffffffffu, need)) continue;
            if (e - b <= 32) {
                // scan the subtree's points
                const int m = e - b;
                double px64[DM];
                if (FP64) {
#pragma unroll
                    for (int k = 0; k < DM; ++k)
                        if (k < d) px64[k] = lane < m ? a.x64[(size_t)k * n + b + lane] : 0.0;
                } else {
                    if (lane < m) {
#pragma unroll
                        for (int c = 0; c < DQ; ++c) {
                            float v[4];
#pragma unroll
                            for (int r = 0; r < 4; ++r)
                                v[r] = 4 * c + r < d ? a.x32[(size_t)(4 * c + r) * n + b + lane] : 0.f;
                            leaf[lane * DQ + c] = make_float4(v[0], v[1], v[2], v[3]);
                        }
                    }
                    __syncwarp();
                }
                for (int p = 0; p < m; ++p) {
                    V s;
                    if (FP64) {
                        double acc = 0.0;
#pragma unroll
                        for (int k = 0; k < DM; ++k) {
                            if (k < d) {
                                double t = __dsub_rn(qx64[k], __shfl_sync(0xffffffffu, px64[k], p));
                                acc = __dadd_rn(acc, __dmul_rn(t, t));
                            }
                        }
                        s = (V)acc;
                    } else {
                        // padded coordinates are 0 on both sides and add nothing
                        float acc = 0.f;
#pragma unroll
                        for (int c = 0; c < DQ; ++c) {
                            const float4 v = leaf[p * DQ + c];
                            const float pv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                            for (int r = 0; r < 4; ++r) {
                                float t = qx[4 * c + r] - pv[r];
                                acc = fmaf(t, t, acc);
                            }
                        }
                        s = (V)acc;
                    }
                    if (valid && s <= cut && (cnt < KL || s < thr)) {
                        int pos = cnt < KL ? cnt : KL - 1;
                        while (pos > 0 && sv[(pos - 1) * 32 + lane] > s) {
                            sv[pos * 32 + lane] = sv[(pos - 1) * 32 + lane];
                            sj[pos * 32 + lane] = sj[(pos - 1) * 32 + lane];
                            --pos;
                        }
                        sv[pos * 32 + lane] = s;
                        sj[pos * 32 + lane] = b + p;
                        if (cnt < KL) ++cnt;
                        if (cnt >= a.k && pos < a.k) {
                            V sk = sv[(a.k - 1) * 32 + lane];
                            cut = FP64 ? sk : exact32 ? (V)knn_threshold_fast((float)sk) : (V)knn_threshold((float)sk, a.eta);
                            // entries above the cut can never be candidates again: drop them
                            while (cnt > a.k && sv[(cnt - 1) * 32 + lane] > cut) --cnt;
                        }
                        thr = cnt == KL ? sv[(KL - 1) * 32 + lane] : (V)INFINITY;
                    }
                }
                if (!FP64) __syncwarp();   // the leaf buffer is reused by the next scan
                n_ev += (unsigned long long)m;
            } else {
                // push the farther child (from the group's centroid) first so the nearer one is
                // visited next
                const int c0 = L.z, c1 = L.z + 1;
                const float4 *b0 = (const float4 *)(a.box + (size_t)c0 * 2 * DMP);
                const float4 *b1 = (const float4 *)(a.box + (size_t)c1 * 2 * DMP);
                float l0 = 0.f, l1 = 0.f;
#pragma unroll
                for (int c = 0; c < DQ; ++c) {
                    const float4 lo0 = b0[2 * c], hi0 = b0[2 * c + 1], lo1 = b1[2 * c], hi1 = b1[2 * c + 1];
                    const float a0[4] = {lo0.x, lo0.y, lo0.z, lo0.w}, z0[4] = {hi0.x, hi0.y, hi0.z, hi0.w};
                    const float a1[4] = {lo1.x, lo1.y, lo1.z, lo1.w}, z1[4] = {hi1.x, hi1.y, hi1.z, hi1.w};
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const float g0 = fmaxf(fmaxf(a0[r] - cent[4 * c + r], cent[4 * c + r] - z0[r]), 0.f);
                        const float g1 = fmaxf(fmaxf(a1[r] - cent[4 * c + r], cent[4 * c + r] - z1[r]), 0.f);
                        l0 = fmaf(g0, g0, l0);
                        l1 = fmaf(g1, g1, l1);
                    }
                }
                int first = l0 <= l1 ? c1 : c0, second = l0 <= l1 ? c0 : c1;
                if (sp + 2 > a.stack_cap) {   // cannot happen: cap = depth + 4; reported, not ignored
                    if (lane == 0) atomicOr(a.err, 1);
                    sp = 0;
                    break;
                }
                if (lane == 0) { stk[sp] = first; stk[sp + 1] = second; }
                __syncwarp();
                sp += 2;
            }
        }
        if (!valid) continue;
        // ---- exact k-th value and repair candidates
        const int k = a.k;
        double cd2;
        int ncand;
        bool complete;
        if (FP64) {
            cd2 = (double)sv[(k - 1) * 32 + lane];
            complete = cnt < KL || (double)sv[(KL - 1) * 32 + lane] > cd2;
            ncand = 0;
            while (ncand < cnt && (double)sv[ncand * 32 + lane] <= cd2) {
                sw[ncand * 32 + lane] = (double)sv[ncand * 32 + lane];
                ++ncand;
            }
        } else {
            const float sk = (float)sv[(k - 1) * 32 + lane];
            const float T = exact32 ? knn_threshold_fast(sk) : knn_threshold(sk, a.eta);
            complete = cnt < KL || (float)sv[(KL - 1) * 32 + lane] > T;
            ncand = 0;
            while (ncand < cnt && (float)sv[ncand * 32 + lane] <= T) ++ncand;
            if (complete) {
                for (int c = 0; c < ncand; ++c) {
                    int j = sj[c * 32 + lane];
                    double w = j == i ? 0.0 : d64(a.x64, n, d, i, j);
                    // insertion sort by w (non-negative doubles compared through their bit patterns)
                    int pos = c;
                    while (pos > 0 && __double_as_longlong(sw[(pos - 1) * 32 + lane]) > __double_as_longlong(w)) {
                        sw[pos * 32 + lane] = sw[(pos - 1) * 32 + lane];
                        sj[pos * 32 + lane] = sj[(pos - 1) * 32 + lane];
                        --pos;
                    }
                    sw[pos * 32 + lane] = w;
                    sj[pos * 32 + lane] = j;
                }
                n_re += (unsigned long long)ncand;
            }
            cd2 = complete ? sw[(k - 1) * 32 + lane] : 0.0;
        }
        if (!complete) {
            int s = atomicAdd(a.slow_cnt, 1);
            a.slow[s] = i;
            continue;
        }
        if (!FP64 && cd2 > 0.0) {   // the ratio in FP32 with outward rounding
            const double sk = (double)sv[(k - 1) * 32 + lane];
            kerr = fmaxf(kerr, __fdiv_ru(__double2float_ru(fabs(sk - cd2)), __double2float_rd(cd2)));
        }
        a.cd64[i] = cd2;
        a.cd32[i] = __double2float_rn(cd2);
        int r = 0;
        for (int c = 0; c < ncand && r < KL - 1; ++c) {
            int j = sj[c * 32 + lane];
            double w = sw[c * 32 + lane];
            if (j != i && __double_as_longlong(w) <= __double_as_longlong(cd2)) {
                a.rep_q[(size_t)i * (KL - 1) + r] = j;
                a.rep_d[(size_t)i * (KL - 1) + r] = w;
                ++r;
            }
        }
        a.rep_cnt[i] = r;
    }
    for (int o = 16; o; o >>= 1) {
        n_ev += __shfl_xor_sync(0xffffffffu, n_ev, o);
        n_re += __shfl_xor_sync(0xffffffffu, n_re, o);
        kerr = fmaxf(kerr, __shfl_xor_sync(0xffffffffu, kerr, o));
    }
    if (lane == 0) {
        atomicAdd(a.stat + 0, n_ev);
        atomicAdd(a.stat + 1, n_re);
        if (kerr > 0.f) atomicMax(a.stat + 2, (unsigned long long)__float_as_uint(kerr));
    }
}

// Exact FP64 answer for one query per warp (ties or duplicates overflowed the list): each lane
// keeps the k smallest w2 of its strided share, the warp merges the 32 lists, then a second
// scan collects every q with w2 <= cd2 as repair edges.
__global__ void __launch_bounds__(32) knn_slow_kernel(KnnArgs a, const int *__restrict__ slow, int nslow,
                                                      int *extra_q, int *extra_p, double *extra_d, int *extra_cnt,
                                                      int extra_cap, int *tie_overflow)
{
    extern __shared__ unsigned char smem_raw[];
    const int lane = threadIdx.x;
    const int k = a.k, n = a.n, d = a.d;
    double *lw = (double *)smem_raw;            // [k][32]
    int *head = (int *)(lw + (size_t)k * 32);   // [32]
    for (int t = blockIdx.x; t < nslow; t += gridDim.x) {
        const int i = slow[t];
        int cnt = 0;
        for (int j = lane; j < n; j += 32) {
            double w = j == i ? 0.0 : d64(a.x64, n, d, i, j);
            if (cnt < k || w < lw[(k - 1) * 32 + lane]) {
                int pos = cnt < k ? cnt : k - 1;
                while (pos > 0 && lw[(pos - 1) * 32 + lane] > w) { lw[pos * 32 + lane] = lw[(pos - 1) * 32 + lane]; --pos; }
                lw[pos * 32 + lane] = w;
                if (cnt < k) ++cnt;
            }
        }
        head[lane] = 0;
        __syncwarp();
        double kth = 0.0;
        for (int r = 0; r < k; ++r) {
            double mine = head[lane] < cnt ? lw[head[lane] * 32 + lane] : INFINITY;
            double mn = mine;
            for (int o = 16; o; o >>= 1) mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
            unsigned who = __ballot_sync(0xffffffffu, mine == mn);
            if (lane == __ffs(who) - 1) head[lane]++;
            __syncwarp();
            kth = mn;
        }
        if (lane == 0) {
            a.cd64[i] = kth;
            a.cd32[i] = __double2float_rn(kth);
            a.rep_cnt[i] = 0;
        }
        for (int j = lane; j < n; j += 32) {
            if (j == i) continue;
            double w = d64(a.x64, n, d, i, j);
            if (w <= kth) {
                int s = atomicAdd(extra_cnt, 1);
                if (s < extra_cap) { extra_p[s] = i; extra_q[s] = j; extra_d[s] = w; }
                else atomicOr(tie_overflow, 1);
            }
        }
        __syncwarp();
    }
}

// node bounds of cd2, bottom-up with arrival counters
__global__ void cd_bounds_kernel(int N, const int *__restrict__ left, const int *__restrict__ right,
                                 const int *__restrict__ parent, const int *__restrict__ begin,
                                 const double *__restrict__ cd64, double *nmin, double *nmax, float *cdmin,
                                 float *cdmax, int *arrive)
{
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < N; x += gridDim.x * blockDim.x) {
        if (left[x] >= 0) continue;
        double c = cd64[begin[x]];
        nmin[x] = c; nmax[x] = c;
        cdmin[x] = __double2float_rd(c);
        cdmax[x] = __double2float_ru(c);
        int cur = x;
        for (int it = 0; it < N; ++it) {
            int p = parent[cur];
            if (p < 0) break;
            __threadfence();
            if (atomicAdd(&arrive[p], 1) == 0) break;
            __threadfence();
            double a0 = ((volatile double *)nmin)[left[p]], a1 = ((volatile double *)nmin)[right[p]];
            double b0 = ((volatile double *)nmax)[left[p]], b1 = ((volatile double *)nmax)[right[p]];
            double mn = fmin(a0, a1), mx = fmax(b0, b1);
            nmin[p] = mn; nmax[p] = mx;
            cdmin[p] = __double2float_rd(mn);
            cdmax[p] = __double2float_ru(mx);
            cur = p;
        }
    }
}

// A pair (p, q) whose distance is within both core distances is in both points' lists: only the
// endpoint with the smaller input id emits it, so every repair edge appears once.
__device__ inline bool rep_keep(int i, int j, double D, const double *__restrict__ cd64, const int *__restrict__ pid)
{
    return !(__double_as_longlong(D) <= __double_as_longlong(cd64[j]) && pid[j] < pid[i]);
}

__global__ void rep_flags_kernel(const int *__restrict__ rep_q, const double *__restrict__ rep_d,
                                 const int *__restrict__ rep_cnt, int n, int KL, const double *__restrict__ cd64,
                                 const int *__restrict__ pid, int *__restrict__ out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int k = 0;
        for (int r = 0; r < rep_cnt[i]; ++r)
            k += rep_keep(i, rep_q[(size_t)i * (KL - 1) + r], rep_d[(size_t)i * (KL - 1) + r], cd64, pid);
        out[i] = k;
    }
}

// repair edge of positions (i, j) with FP64 squared distance D: weight max(cd2 i, cd2 j, D)
__global__ void rep_emit_kernel(const int *__restrict__ rep_q, const double *__restrict__ rep_d,
                                const int *__restrict__ rep_cnt, const int *__restrict__ off, int n, int KL,
                                const double *__restrict__ cd64, const int *__restrict__ pid, EdgeK *__restrict__ out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int o = off[i];
        for (int r = 0; r < rep_cnt[i]; ++r) {
            const int j = rep_q[(size_t)i * (KL - 1) + r];
            const double D = rep_d[(size_t)i * (KL - 1) + r];
            if (!rep_keep(i, j, D, cd64, pid)) continue;
            const double c = __double_as_longlong(cd64[i]) >= __double_as_longlong(cd64[j]) ? cd64[i] : cd64[j];
            out[o++] = make_edge(__double_as_longlong(c) >= __double_as_longlong(D) ? c : D, pid[i], pid[j]);
        }
    }
}

// the exact lists of the slow queries, appended after the others (count: running total)
__global__ void rep_emit_extra_kernel(const int *__restrict__ ep, const int *__restrict__ eq,
                                      const double *__restrict__ ed, const int *__restrict__ cnt, int cap,
                                      const double *__restrict__ cd64, const int *__restrict__ pid, EdgeK *__restrict__ out,
                                      int *count)
{
    __shared__ int sh[32];
    const int m = min(*cnt, cap);
    for (int b0 = blockIdx.x * blockDim.x; b0 < m; b0 += gridDim.x * blockDim.x) {
        const int t = b0 + threadIdx.x;
        bool keep = false;
        int i = 0, j = 0;
        double D = 0.0;
        if (t < m) {
            i = ep[t];
            j = eq[t];
            D = ed[t];
            keep = rep_keep(i, j, D, cd64, pid);
        }
        const int slot = block_append(count, keep ? 1 : 0, sh);
        if (keep) {
            const double c = __double_as_longlong(cd64[i]) >= __double_as_longlong(cd64[j]) ? cd64[i] : cd64[j];
            out[slot] = make_edge(__double_as_longlong(c) >= __double_as_longlong(D) ? c : D, pid[i], pid[j]);
        }
    }
}

__global__ void core_out_kernel(const double *__restrict__ cd64, const int *__restrict__ pid, int n, double *out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[pid[i]] = sqrt(cd64[i]);
}

}  // namespace

int core_distances(Points &P, Tree &T, int min_pts, bool fp64, HdbState &H, Arena &ar, cudaStream_t st, int *pin,
                   wm_stats *stats)
{
    const int n = P.n, d = P.d, N = T.N;
    if (min_pts > kMaxMinPts) return WM_EINVAL;
    const int KL = std::min(min_pts + 8, n);
    H.cd64 = ar.get<double>(n);
    H.cd32 = ar.get<float>(n);
    H.cdmin = ar.get<float>(N);
    H.cdmax = ar.get<float>(N);
    if (ar.failed) return WM_ENOMEM;
    // persistent output of this function: repair edges (allocated before the scratch)
    const int RQ = KL > 1 ? KL - 1 : 1;
    const int extra_cap = 4 * n + 1024;
    EdgeK *rep = ar.get<EdgeK>((size_t)n * RQ + extra_cap);
    if (!rep) return WM_ENOMEM;
    size_t mark = ar.off;
    KnnArgs a;
    a.N = N; a.n = n; a.d = d; a.k = min_pts; a.KL = KL;
    a.lo = T.lo; a.hi = T.hi; a.begin = T.begin; a.end = T.end; a.left = T.left; a.right = T.right;
    a.x32 = P.x32; a.x64 = P.x64;
    a.eta = fp64 ? 0.0 : 2.0 * (double)P.delta * sqrt((double)d) * (1.0 + 1e-6);
    a.stack_cap = T.depth + 4;
    a.cd64 = H.cd64; a.cd32 = H.cd32;
    a.rep_q = ar.get<int>((size_t)n * RQ);
    a.rep_d = ar.get<double>((size_t)n * RQ);
    a.rep_cnt = ar.get<int>(n + 1);
    a.slow = ar.get<int>(n);
    int *cnts = ar.get<int>(8);
    a.slow_cnt = cnts;
    a.stat = ar.get<unsigned long long>(4);
    int *ex_p = ar.get<int>(extra_cap), *ex_q = ar.get<int>(extra_cap);
    double *ex_d = ar.get<double>(extra_cap);
    double *nmin = ar.get<double>(N), *nmax = ar.get<double>(N);
    int *off = ar.get<int>(n + 1);
    if (ar.failed) return WM_ENOMEM;
    cudaMemsetAsync(cnts, 0, 8 * sizeof(int), st);
    cudaMemsetAsync(a.stat, 0, 4 * sizeof(unsigned long long), st);
    // launch shape: warps per block limited by shared memory; the grid fills the SMs
    const int dmp = d <= 3 ? 4 : d <= 7 ? 8 : 16;   // = knn_dmp<DM> of the instantiation used
    size_t per_warp = knn_warp_smem(dmp, KL, fp64 ? 8 : 4, a.stack_cap);
    int wpb = (int)std::min<size_t>(8, std::max<size_t>(1, (48u << 10) / per_warp));
    size_t smem = per_warp * wpb;
    int blocks = num_sms() * std::max(1, 32 / wpb);
    int total_warps = blocks * wpb;
    a.next_group = cnts + 6;
    a.err = cnts + 5;
    a.wscratch = ar.get<double>((size_t)total_warps * KL * 32);
    // packed node records and boxes (the traversal reads a node with two or three vector loads)
    NodeRec *rec = ar.get<NodeRec>(N);
    float *box = ar.get<float>((size_t)N * 2 * dmp);
    if (!a.wscratch || !rec || !box) return WM_ENOMEM;
    pack_nodes(T, d, dmp, rec, box, st);
    a.rec = rec;
    a.box = box;
#define WM_KNN(DM)                                                                                           \
    do {                                                                                                     \
        if (fp64) {                                                                                          \
            cudaFuncSetAttribute(knn_fast_kernel<DM, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
            launch(knn_fast_kernel<DM, true>, blocks, 32 * wpb, smem, st, a);                                    \
        } else {                                                                                             \
            cudaFuncSetAttribute(knn_fast_kernel<DM, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
            launch(knn_fast_kernel<DM, false>, blocks, 32 * wpb, smem, st, a);                                   \
        }                                                                                                    \
    } while (0)
    cudaEvent_t k0, k1;
    cudaEventCreate(&k0);
    cudaEventCreate(&k1);
    cudaEventRecord(k0, st);
    if (d <= 2) WM_KNN(2);
    else if (d <= 3) WM_KNN(3);
    else if (d <= 5) WM_KNN(5);
    else if (d <= 7) WM_KNN(7);
    else WM_KNN(16);
#undef WM_KNN
    cudaEventRecord(k1, st);
    cudaMemcpyAsync(pin, cnts, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) {
        cudaEventDestroy(k0);
        cudaEventDestroy(k1);
        return WM_ECUDA;
    }
    if (stats) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, k0, k1);
        stats->ms_knn_kernel = ms;
    }
    cudaEventDestroy(k0);
    cudaEventDestroy(k1);
    const int nslow = pin[0];
    if (nslow > 0) {
        size_t sm2 = (size_t)min_pts * 32 * 8 + 32 * 4;
        cudaFuncSetAttribute(knn_slow_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2);
        launch(knn_slow_kernel, std::min(nslow, num_sms() * 8), 32, sm2, st, a, a.slow, nslow, ex_q, ex_p, ex_d, cnts + 1,
                                                                     extra_cap, cnts + 2);
    }
    // node bounds
    cudaMemsetAsync(T.arrive, 0, sizeof(int) * N, st);
    launch(cd_bounds_kernel, grid_for(N, 256), 256, 0, st, N, T.left, T.right, T.parent, T.begin, H.cd64, nmin, nmax,
                                                       H.cdmin, H.cdmax, T.arrive);
    // repair edges: one copy of each, weighted, in no particular order (each MemoGFK round takes
    // those of its weight range)
    launch(rep_flags_kernel, grid_for(n, 256), 256, 0, st, a.rep_q, a.rep_d, a.rep_cnt, n, KL, H.cd64, P.pid, off);
    int rc = scan_exclusive_i32(off, off, n, cnts + 3, st, ar);
    if (rc) return rc;
    launch(rep_emit_kernel, grid_for(n, 256), 256, 0, st, a.rep_q, a.rep_d, a.rep_cnt, off, n, KL, H.cd64, P.pid, rep);
    launch(rep_emit_extra_kernel, grid_for(extra_cap, 256), 256, 0, st, ex_p, ex_q, ex_d, cnts + 1, extra_cap, H.cd64,
           P.pid, rep, cnts + 3);
    cudaMemcpyAsync(pin, cnts, 8 * sizeof(int), cudaMemcpyDeviceToHost, st);
    unsigned long long hs[3];
    cudaMemcpyAsync(pin + 8, a.stat, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return WM_ECUDA;
    memcpy(hs, pin + 8, sizeof hs);
    if (pin[5]) {
        set_error_detail("k-NN: a traversal stack overflowed (internal error)");
        return WM_EINTERNAL;
    }
    const int nrep = pin[3];
    if (stats) {
        stats->knn_evals = (int64_t)hs[0];
        stats->fp64_rechecks += (int64_t)hs[1];
        stats->tie_overflow = pin[2] ? 1 : 0;
        float ke;
        const unsigned kb = (unsigned)hs[2];
        memcpy(&ke, &kb, sizeof ke);
        stats->max_rel_screen_err = std::max(stats->max_rel_screen_err, (double)ke);
    }
    H.rep = rep;
    H.nrep = nrep;
    ar.off = mark;
    // keep the cd arrays and node bounds (allocated before mark); drop the scratch
    return 0;
}

int write_core_distances(const Points &P, const HdbState &H, double *out, Arena &ar, cudaStream_t st)
{
    if (!out) return 0;
    cudaPointerAttributes at;
    bool dev = cudaPointerGetAttributes(&at, out) == cudaSuccess &&
               (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    double *dst = out;
    if (!dev) {
        dst = ar.get<double>(P.n);
        if (!dst) return WM_ENOMEM;
    }
    launch(core_out_kernel, grid_for(P.n, 256), 256, 0, st, H.cd64, P.pid, P.n, dst);
    if (!dev) cudaMemcpyAsync(out, dst, sizeof(double) * P.n, cudaMemcpyDeviceToHost, st);
    return cudaStreamSynchronize(st) == cudaSuccess ? 0 : WM_ECUDA;
}

}  // namespace wm
