// util.cu -- device-wide primitives: exclusive prefix sum and a stable LSD radix sort of
// 128-bit edge keys (the "prefix sum" and sorting primitives of Sec. 2.2, written for the GPU).
#include "wm_internal.cuh"

namespace wm {

namespace {

constexpr int kScanBlock = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanBlock * kScanItems;

template <typename T>
__device__ inline T block_exclusive_scan(T v, T *smem_warp, T &total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) smem_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T w = lane < nw ? smem_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) smem_warp[lane] = w;
    }
    __syncthreads();
    total = smem_warp[nw - 1];
    T r = x - v + (warp > 0 ? smem_warp[warp - 1] : 0);
    __syncthreads();
    return r;
}

template <typename T>
__global__ void scan_reduce_kernel(const T *__restrict__ in, int n, T *__restrict__ block_sums,
                                   const int *__restrict__ n_dev)
{
    if (n_dev) n = min(n, *n_dev);
    __shared__ T sw[32];
    long long base = (long long)blockIdx.x * kScanTile;
    T s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        long long idx = base + (long long)threadIdx.x * kScanItems + i;
        if (idx < n) s += in[idx];
    }
    T total;
    block_exclusive_scan(s, sw, total);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

template <typename T>
__global__ void scan_down_kernel(const T *__restrict__ in, T *__restrict__ out, int n,
                                 const T *__restrict__ block_offs, T *total_dev, int nblocks,
                                 const int *__restrict__ n_dev)
{
    if (n_dev) n = min(n, *n_dev);
    __shared__ T sw[32];
    long long base = (long long)blockIdx.x * kScanTile;
    T v[kScanItems];
    T s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        long long idx = base + (long long)threadIdx.x * kScanItems + i;
        v[i] = idx < n ? in[idx] : 0;
        s += v[i];
    }
    T total;
    T ex = block_exclusive_scan(s, sw, total) + (block_offs ? block_offs[blockIdx.x] : 0);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        long long idx = base + (long long)threadIdx.x * kScanItems + i;
        if (idx < n) out[idx] = ex;
        ex += v[i];
    }
    if (total_dev && blockIdx.x == nblocks - 1 && threadIdx.x == blockDim.x - 1) *total_dev = ex;
}

__global__ void fill_i32_kernel(int *p, int v, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) p[i] = v;
}

}  // namespace

void fill_i32(int *p, int v, size_t n, cudaStream_t st)
{
    if (n == 0) return;
    launch(fill_i32_kernel, grid_for((long long)n, 256), 256, 0, st, p, v, n);
}

// out[i] = sum_{j<i} in[j]; *total_dev (optional, device) = sum of all.  in may equal out.
// With n_dev, the length is min(n, *n_dev), read on the device (n is then a bound).
template <typename T>
static int scan_exclusive_t(const T *in, T *out, int n, T *total_dev, cudaStream_t st, Arena &ar,
                            const int *n_dev = nullptr)
{
    if (n <= 0) {
        if (total_dev) cudaMemsetAsync(total_dev, 0, sizeof(T), st);
        return 0;
    }
    int nb = (n + kScanTile - 1) / kScanTile;
    if (nb == 1) {
        launch(scan_down_kernel<T>, 1, kScanBlock, 0, st, in, out, n, (const T *)nullptr, total_dev, 1, n_dev);
        return 0;
    }
    size_t mark = ar.off;
    T *sums = ar.get<T>(nb);
    if (!sums) return WM_ENOMEM;
    // blocks past the device length contribute 0, so the last block still writes the total
    launch(scan_reduce_kernel<T>, nb, kScanBlock, 0, st, in, n, sums, n_dev);
    int rc = scan_exclusive_t<T>(sums, sums, nb, (T *)nullptr, st, ar);
    if (rc) return rc;
    launch(scan_down_kernel<T>, nb, kScanBlock, 0, st, in, out, n, (const T *)sums, total_dev, nb, n_dev);
    ar.off = mark;
    return 0;
}

int scan_exclusive_i32(const int *in, int *out, int n, int *total_dev, cudaStream_t st, Arena &ar)
{
    return scan_exclusive_t<int>(in, out, n, total_dev, st, ar);
}

int scan_exclusive_i64(const long long *in, long long *out, int n, long long *total_dev, cudaStream_t st, Arena &ar)
{
    return scan_exclusive_t<long long>(in, out, n, total_dev, st, ar);
}

int scan_exclusive_i32_dev(const int *in, int *out, const int *n_dev, int n_max, int *total_dev, cudaStream_t st,
                           Arena &ar)
{
    return scan_exclusive_t<int>(in, out, n_max, total_dev, st, ar, n_dev);
}

int scan_exclusive_i64_dev(const long long *in, long long *out, const int *n_dev, int n_max, long long *total_dev,
                           cudaStream_t st, Arena &ar)
{
    return scan_exclusive_t<long long>(in, out, n_max, total_dev, st, ar, n_dev);
}

// ------------------------------------------------------------------------------ radix sort
namespace {

constexpr int kRsBlock = 256;

__device__ inline unsigned digit_of(const EdgeK &e, int byte)
{
    unsigned long long w = byte < 8 ? e.lo : e.hi;
    return (unsigned)(w >> ((byte & 7) * 8)) & 0xffu;
}

// Histogram of every byte position over all keys: ghist[byte*256 + digit].
__global__ void rs_hist_all(const EdgeK *__restrict__ a, int m, unsigned *__restrict__ ghist)
{
    __shared__ unsigned h[16 * 256];
    for (int i = threadIdx.x; i < 16 * 256; i += blockDim.x) h[i] = 0;
    __syncthreads();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x) {
        EdgeK e = a[i];
#pragma unroll
        for (int b = 0; b < 16; ++b) atomicAdd(&h[b * 256 + digit_of(e, b)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 16 * 256; i += blockDim.x)
        if (h[i]) atomicAdd(&ghist[i], h[i]);
}

// Per-block histogram of one byte over the block's contiguous chunk: bh[digit*G + block].
__global__ void rs_pass_hist(const EdgeK *__restrict__ a, int m, int byte, int chunk, int *__restrict__ bh)
{
    __shared__ int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    long long beg = (long long)blockIdx.x * chunk, end = beg + chunk < m ? beg + chunk : m;
    for (long long i = beg + threadIdx.x; i < end; i += blockDim.x) atomicAdd(&h[digit_of(a[i], byte)], 1);
    __syncthreads();
    bh[threadIdx.x * gridDim.x + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: block processes its chunk in order, 256 keys per step.
__global__ void __launch_bounds__(kRsBlock) rs_pass_scatter(const EdgeK *__restrict__ a, EdgeK *__restrict__ out, int m,
                                                            int byte, int chunk, const int *__restrict__ offs)
{
    __shared__ int base[256];
    __shared__ int wcnt[8][256];   // (step << 6) | count, entries of other steps read as 0
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    base[threadIdx.x] = offs[threadIdx.x * gridDim.x + blockIdx.x];
    for (int i = threadIdx.x; i < 8 * 256; i += blockDim.x) (&wcnt[0][0])[i] = -1;
    __syncthreads();
    long long beg = (long long)blockIdx.x * chunk, end = beg + chunk < m ? beg + chunk : m;
    int step = 0;
    for (long long t0 = beg; t0 < end; t0 += kRsBlock, ++step) {
        long long idx = t0 + threadIdx.x;
        bool valid = idx < end;
        EdgeK e;
        unsigned dg = 256;
        if (valid) { e = a[idx]; dg = digit_of(e, byte); }
        unsigned peers = __match_any_sync(0xffffffffu, dg);
        int rank = __popc(peers & lanemask_lt());
        int leader = __ffs(peers) - 1;
        if (valid && lane == leader) wcnt[warp][dg] = (step << 6) | __popc(peers);
        __syncthreads();
        if (valid) {
            int off = base[dg] + rank;
            for (int w = 0; w < warp; ++w) {
                int c = wcnt[w][dg];
                if (c >= 0 && (c >> 6) == step) off += c & 63;
            }
            out[off] = e;
        }
        __syncthreads();
        {
            int dgt = threadIdx.x, add = 0;
            for (int w = 0; w < 8; ++w) {
                int c = wcnt[w][dgt];
                if (c >= 0 && (c >> 6) == step) add += c & 63;
            }
            base[dgt] += add;
        }
        __syncthreads();
    }
}

}  // namespace

// Sorts m keys ascending as 128-bit unsigned integers (stable LSD, 8-bit digits, byte
// positions on which all keys agree are skipped).  The result is in *result (keys or tmp).
int radix_sort_edges(EdgeK *keys, EdgeK *tmp, int m, cudaStream_t st, Arena &ar, EdgeK **result, void *host_scratch)
{
    *result = keys;
    if (m <= 1) return 0;
    size_t mark = ar.off;
    unsigned *ghist = ar.get<unsigned>(16 * 256);
    unsigned *hhist = (unsigned *)host_scratch;
    if (!ghist) return WM_ENOMEM;
    cudaMemsetAsync(ghist, 0, sizeof(unsigned) * 16 * 256, st);
    launch(rs_hist_all, grid_for(m, 256, num_sms() * 4), 256, 0, st, keys, m, ghist);
    cudaMemcpyAsync(hhist, ghist, sizeof(unsigned) * 16 * 256, cudaMemcpyDeviceToHost, st);
    cudaError_t ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) { ar.off = mark; return WM_ECUDA; }
    bool need[16];
    for (int b = 0; b < 16; ++b) {
        need[b] = true;
        for (int g = 0; g < 256; ++g)
            if (hhist[b * 256 + g] == (unsigned)m) { need[b] = false; break; }
    }
    int G = (m + 2047) / 2048;
    if (G > 1024) G = 1024;
    int chunk = (m + G - 1) / G;
    chunk = (chunk + kRsBlock - 1) / kRsBlock * kRsBlock;
    G = (m + chunk - 1) / chunk;
    int *bh = ar.get<int>((size_t)256 * G);
    if (!bh) { ar.off = mark; return WM_ENOMEM; }
    EdgeK *src = keys, *dst = tmp;
    for (int b = 0; b < 16; ++b) {
        if (!need[b]) continue;
        launch(rs_pass_hist, G, 256, 0, st, src, m, b, chunk, bh);
        int rc = scan_exclusive_i32(bh, bh, 256 * G, nullptr, st, ar);
        if (rc) { ar.off = mark; return rc; }
        launch(rs_pass_scatter, G, kRsBlock, 0, st, src, dst, m, b, chunk, bh);
        EdgeK *t = src; src = dst; dst = t;
    }
    *result = src;
    ar.off = mark;
    return 0;
}

}  // namespace wm
