// wm_internal.cuh -- internal declarations shared by the CUDA translation units of libwspdmst.
//
// Data layout in HBM (all arrays are device-resident for the whole call):
//   points  : SoA, permuted into k-d tree order.  x32[k*n + i] (float, the FP32 screen copy),
//             x64[k*n + i] (double, the exact copy), pid[i] = input row of tree position i.
//   tree    : one record per node, stored as parallel arrays indexed by node id (BFS order):
//             box lo/hi [k*N + node] (float, rounded outward so they contain the FP64 points),
//             begin/end (point range in tree order), left/right children (-1 at a leaf),
//             parent, plus per-round comp label and, for HDBSCAN*, cd bounds.
//   edges   : 16-byte records EdgeK {hi = bits of the FP64 w2, lo = (min id << 32) | max id},
//             which compare as 128-bit unsigned integers exactly like the key K (w2 >= 0).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include <atomic>
#include <utility>

#include "../../include/wspdmst.h"

namespace wm {

constexpr int kMaxDim = 16;

// ------------------------------------------------------------------ error bounds of the screen
// Relative error bound of an FP32 sum of d <= 16 squared differences of exactly representable
// inputs: each subtract, square and add contributes at most one half-ulp, (d+2)*2^-24 <= 2^-19.
constexpr double kEps32 = 1.0 / 524288.0;                  // 2^-19
// Relative error bound of the FP64 evaluation of w2 (same operation count): (d+2)*2^-53 < 2^-48.
constexpr double kGam64 = 1.0 / 281474976710656.0;         // 2^-48
// Margin used to turn FP32 box bounds into bounds on any FP64 w2 of the points inside.
constexpr float kBoxRel = 1.0f / 262144.0f;                // 2^-18 > kEps32 + kGam64 + products
// Absolute slack covering FP32 subnormal rounding (each op errs by at most 2^-150).
constexpr float kAbsTiny = 7.17464814e-43f;                // 2^-140

// ---------------------------------------------------------------------------- edge record
struct __align__(16) EdgeK {
    unsigned long long lo;   // (min id << 32) | max id
    unsigned long long hi;   // bits of w2 (double, >= 0)
};

__host__ __device__ inline EdgeK make_edge(double w2, int a, int b)
{
    unsigned ua = (unsigned)(a < b ? a : b), ub = (unsigned)(a < b ? b : a);
    EdgeK e;
    e.lo = ((unsigned long long)ua << 32) | ub;
#ifdef __CUDA_ARCH__
    e.hi = (unsigned long long)__double_as_longlong(w2);
#else
    union { double d; unsigned long long u; } c; c.d = w2; e.hi = c.u;
#endif
    return e;
}
__host__ __device__ inline int edge_u(const EdgeK &e) { return (int)(e.lo >> 32); }
__host__ __device__ inline int edge_v(const EdgeK &e) { return (int)(e.lo & 0xffffffffu); }
__device__ inline double edge_w2(const EdgeK &e) { return __longlong_as_double((long long)e.hi); }
__host__ __device__ inline bool edge_less(const EdgeK &a, const EdgeK &b)
{
    return a.hi != b.hi ? a.hi < b.hi : a.lo < b.lo;
}

// ------------------------------------------------------------------------- arena allocator
struct Arena {
    char *base = nullptr;
    size_t cap = 0;
    size_t off = 0;
    size_t peak = 0;
    bool failed = false;
    void *take(size_t bytes)
    {
        // 256-byte aligned device addresses (a caller's arena may start anywhere)
        const size_t mis = (size_t)(reinterpret_cast<uintptr_t>(base) & 255);
        size_t a = ((off + mis + 255) & ~size_t(255)) - mis;
        if (a + bytes > cap) { failed = true; return nullptr; }
        off = a + bytes;
        if (off > peak) peak = off;
        return base + a;
    }
    template <class T> T *get(size_t count) { return (T *)take(sizeof(T) * (count ? count : 1)); }
};

// ---------------------------------------------------------------------------- point / tree
struct Points {
    int n = 0, d = 0;
    float *x32 = nullptr;    // [d][n]
    double *x64 = nullptr;   // [d][n]
    int *pid = nullptr;      // tree position -> input id
    int *pos = nullptr;      // input id -> tree position
    float delta = 0.f;       // max |x64 - x32| over all coordinates (0 for FP32 input)
};

struct Tree {
    int N = 0;                 // nodes
    int depth = 0;             // levels
    float *lo = nullptr, *hi = nullptr;   // [d][N]
    int *begin = nullptr, *end = nullptr, *left = nullptr, *right = nullptr, *parent = nullptr;
    float *diam2 = nullptr;    // rigorous upper bound of any FP64 w2 inside the node
    int *comp = nullptr;       // per round: component id if all points in one, else -1
    float *cdmin = nullptr, *cdmax = nullptr;   // HDBSCAN*: cd2 bounds (rounded outward)
    int *arrive = nullptr;     // scratch counters for bottom-up passes
};

// -------------------------------------------------------------------- small device helpers
__device__ inline float atomicMinF(float *addr, float v)
{
    return v >= 0.f ? __int_as_float(atomicMin((int *)addr, __float_as_int(v)))
                    : __uint_as_float(atomicMax((unsigned *)addr, __float_as_uint(v)));
}
__device__ inline float atomicMaxF(float *addr, float v)
{
    return v >= 0.f ? __int_as_float(atomicMax((int *)addr, __float_as_int(v)))
                    : __uint_as_float(atomicMin((unsigned *)addr, __float_as_uint(v)));
}
// WriteMin of a non-negative double (its bit pattern orders like the value).
__device__ inline void atomicMinPosD(double *addr, double v)
{
    atomicMin((unsigned long long *)addr, (unsigned long long)__double_as_longlong(v));
}

// Rigorous bounds on the FP64 w2 of any point pair inside boxes from FP32 box arithmetic.
__device__ inline float lower_w2(float q) { float r = __fsub_rd(__fmul_rd(q, 1.0f - kBoxRel), kAbsTiny); return r > 0.f ? r : 0.f; }
__device__ inline float upper_w2(float q) { return __fadd_ru(__fmul_ru(q, 1.0f + kBoxRel), kAbsTiny); }

// Packed node record of the traversals: l = {begin, end, left child, component label of the
// round} (the right child is always left + 1), m = {diam2 bound, cdmin, cdmax, 0}.  32 bytes,
// read in one 256-bit load.
struct __align__(32) NodeRec {
    int4 l;
    float4 m;
};

// 256-bit read-only global load (sm_100 and later): 32 bytes from a 32-byte aligned address that
// no thread writes during the kernel.  One load touches one 32-byte sector, where two 128-bit
// loads would each cost a pass of the L1 data pipe.
__device__ __forceinline__ void ldg256(const void *p, float4 &a, float4 &b)
{
    asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
        : "l"(p));
}
// Packed node boxes: a row of 2 DP floats per node (DP = d rounded up to 4, 8 or 16) in groups of
// four dimensions, lo[4c .. 4c+3] then hi[4c .. 4c+3] for group c (padded dimensions 0 on both
// sides), so that one 256-bit load brings both bounds of four dimensions.
__host__ __device__ constexpr int box_lo(int k) { return 8 * (k >> 2) + (k & 3); }
__host__ __device__ constexpr int box_hi(int k) { return 8 * (k >> 2) + 4 + (k & 3); }

__device__ __forceinline__ void load_rec(const NodeRec *r, int x, int4 &l, float4 &m)
{
    float4 f;
    ldg256(r + x, f, m);
    l = make_int4(__float_as_int(f.x), __float_as_int(f.y), __float_as_int(f.z), __float_as_int(f.w));
}

__device__ inline unsigned lanemask_lt() { unsigned m; asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m)); return m; }

// Block-wide append of cnt >= 0 items per thread: one atomic on the counter per block (a counter
// bumped once per warp by thousands of warps serialises them).  Every thread of the block must
// call it (block-uniform control flow; blockDim.x a multiple of 32); sh: 32 ints of shared
// memory.  Returns the thread's first slot.
__device__ inline int block_append(int *counter, int cnt, int *sh)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        const int t = lane < nw ? sh[lane] : 0;
        int s = t;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        const int total = __shfl_sync(0xffffffffu, s, 31);
        int base = 0;
        if (lane == 0 && total) base = atomicAdd(counter, total);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (lane < nw) sh[lane] = base + s - t;
    }
    __syncthreads();
    const int r = sh[wid] + x - cnt;
    __syncthreads();
    return r;
}

// ------------------------------------------------------------------------- host-side API
// util.cu
int scan_exclusive_i32(const int *in, int *out, int n, int *total_dev, cudaStream_t st, Arena &ar);
int scan_exclusive_i64(const long long *in, long long *out, int n, long long *total_dev, cudaStream_t st, Arena &ar);
// the same with the length read on the device: min(n_max, *n_dev)
int scan_exclusive_i32_dev(const int *in, int *out, const int *n_dev, int n_max, int *total_dev, cudaStream_t st,
                           Arena &ar);
int scan_exclusive_i64_dev(const long long *in, long long *out, const int *n_dev, int n_max, long long *total_dev,
                           cudaStream_t st, Arena &ar);
// message for the last failure on this thread (read by wm_last_error_detail)
void set_error_detail(const char *msg);
// host_scratch: at least 16 KiB of host memory (pinned preferred) for the digit histogram readback
int radix_sort_edges(EdgeK *keys, EdgeK *tmp, int m, cudaStream_t st, Arena &ar, EdgeK **result, void *host_scratch);
void fill_i32(int *p, int v, size_t n, cudaStream_t st);

// Every kernel launch of the library goes through launch(), which counts it.
extern std::atomic<long long> g_launch_count;

template <typename... KArgs, typename... Args>
inline void launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args &&...args)
{
    g_launch_count.fetch_add(1, std::memory_order_relaxed);
    kernel<<<grid, block, smem, st>>>(std::forward<Args>(args)...);
}

// Streaming multiprocessors of the current device (read once per device and cached); grids are
// sized in multiples of it.
inline int num_sms()
{
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); dev = 0; }
    std::atomic<int> &c = cache[dev & 63];
    int v = c.load(std::memory_order_relaxed);
    if (v <= 0) {
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
            cudaGetLastError();
            v = 1;
        }
        c.store(v, std::memory_order_relaxed);
    }
    return v;
}

// kernel launch helpers
inline int grid_for(long long work, int block, int max_blocks = -1)
{
    if (max_blocks < 0) max_blocks = num_sms() * 16;
    long long g = (work + block - 1) / block;
    if (g < 1) g = 1;
    if (g > max_blocks) g = max_blocks;
    return (int)g;
}

}  // namespace wm
