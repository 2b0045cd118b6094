// Exclusive prefix sum (Sec. 2.2, Eq. 1): counts (int32) -> offsets
// (int64) with the total appended.  Reduce-then-scan in three launches:
// tile sums, a scan of the tile sums, and a rescan of every tile with its
// prefix.  Every thread owns kItems consecutive counts; warps combine with
// shuffles.  No kernel waits on another block, so nothing can spin.
#include <mutex>

#include "problem.cuh"

namespace ci {

constexpr int kScanThreads = 512;
constexpr int kItems = 8;
constexpr int kTile = kScanThreads * kItems;

__device__ __forceinline__ int64_t warp_incl_scan(int64_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// Exclusive scan of one value per thread across the block; returns the
// thread's exclusive prefix and writes the block total to *total.
__device__ int64_t block_excl_scan(int64_t v, int64_t *total) {
    __shared__ int64_t warp_sums[kScanThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t incl = warp_incl_scan(v);
    if (lane == 31) warp_sums[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int64_t w = lane < kScanThreads / 32 ? warp_sums[lane] : 0;
        int64_t wi = warp_incl_scan(w);
        if (lane < kScanThreads / 32) warp_sums[lane] = wi - w;
        if (lane == kScanThreads / 32 - 1) *total = wi;
    }
    __syncthreads();
    int64_t r = warp_sums[wid] + incl - v;
    __syncthreads();
    return r;
}

// The kItems counts of a thread: two 16-byte loads when they are all in
// range and x is 16-byte aligned (VEC), else one load each.
template <bool VEC>
__device__ __forceinline__ void load_items(const int32_t *x, int64_t n, int64_t base, int32_t (&v)[kItems]) {
    if (VEC && base + kItems <= n) {
        const int4 a = *reinterpret_cast<const int4 *>(x + base);
        const int4 b = *reinterpret_cast<const int4 *>(x + base + 4);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
        return;
    }
#pragma unroll
    for (int i = 0; i < kItems; ++i) v[i] = base + i < n ? x[base + i] : 0;
}

template <bool VEC>
__global__ void __launch_bounds__(kScanThreads) k_tile_sums(const int32_t *x, int64_t n, int64_t *sums) {
    __shared__ int64_t tot;
    int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kItems;
    int32_t c[kItems];
    load_items<VEC>(x, n, base, c);
    int64_t v = 0;
#pragma unroll
    for (int i = 0; i < kItems; ++i) v += c[i];
    block_excl_scan(v, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// In-place exclusive scan of nb tile sums by one block (loops for nb > block).
__global__ void __launch_bounds__(kScanThreads) k_scan_sums(int64_t *sums, int64_t nb) {
    __shared__ int64_t tot;
    int64_t carry = 0;
    for (int64_t b0 = 0; b0 < nb; b0 += kScanThreads) {
        int64_t i = b0 + threadIdx.x;
        int64_t v = i < nb ? sums[i] : 0;
        int64_t e = block_excl_scan(v, &tot);
        if (i < nb) sums[i] = carry + e;
        carry += tot;
        __syncthreads();
    }
}

// VEC: y is 16-byte aligned too, and full runs are stored as pairs
template <bool VEC>
__global__ void __launch_bounds__(kScanThreads) k_tile_apply(const int32_t *x, int64_t n, const int64_t *sums,
                                                             int64_t *y) {
    __shared__ int64_t tot;
    int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kItems;
    int32_t v[kItems];
    load_items<VEC>(x, n, base, v);
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < kItems; ++i) s += v[i];
    int64_t e = block_excl_scan(s, &tot) + sums[blockIdx.x];
    if (VEC && base + kItems <= n) {
        int64_t o[kItems];
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            o[i] = e;
            e += v[i];
        }
#pragma unroll
        for (int i = 0; i < kItems; i += 2)
            *reinterpret_cast<longlong2 *>(y + base + i) = make_longlong2(o[i], o[i + 1]);
        if (base + kItems == n) y[n] = e;   // the total
        return;
    }
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        if (base + i < n) y[base + i] = e;
        e += v[i];
        if (base + i == n - 1) y[n] = e;   // the total
    }
}

__global__ void k_zero_total(int64_t *y) { y[0] = 0; }

void exclusive_scan_i32(const int32_t *counts, int64_t n, int64_t *offsets, DevBuf<int64_t> &scratch,
                        cudaStream_t s) {
    if (n < 0) fail(CI_ERR_INVALID_ARG, "scan length < 0");
    if (n == 0) {
        launch("k_zero_total", k_zero_total, 1, 1, 0, s, offsets);
        CI_CHECK_LAUNCH();
        return;
    }
    int64_t nb = (n + kTile - 1) / kTile;
    if (nb > INT32_MAX) fail(CI_ERR_CAPACITY, "scan too long");
    scratch.ensure((size_t)nb);
    const bool vec = (uintptr_t)counts % 16 == 0 && (uintptr_t)offsets % 16 == 0;
    if (vec) {
        launch("k_tile_sums", k_tile_sums<true>, (unsigned)nb, kScanThreads, 0, s, counts, n, scratch.ptr);
        launch("k_scan_sums", k_scan_sums, 1, kScanThreads, 0, s, scratch.ptr, nb);
        launch("k_tile_apply", k_tile_apply<true>, (unsigned)nb, kScanThreads, 0, s, counts, n, scratch.ptr, offsets);
    } else {
        launch("k_tile_sums", k_tile_sums<false>, (unsigned)nb, kScanThreads, 0, s, counts, n, scratch.ptr);
        launch("k_scan_sums", k_scan_sums, 1, kScanThreads, 0, s, scratch.ptr, nb);
        launch("k_tile_apply", k_tile_apply<false>, (unsigned)nb, kScanThreads, 0, s, counts, n, scratch.ptr,
               offsets);
    }
    CI_CHECK_LAUNCH();
}

__global__ void k_gather_i64(const int64_t *src, const int64_t *idx, int64_t n, int64_t *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = src[idx[i]];
}

std::vector<int64_t> gather_i64(const int64_t *src, const std::vector<int64_t> &idx, cudaStream_t s) {
    const int64_t n = (int64_t)idx.size();
    std::vector<int64_t> out((size_t)n);
    if (n == 0) return out;
    if (n <= 2) {
        for (int64_t i = 0; i < n; ++i)
            CI_CUDA(cudaMemcpyAsync(&out[i], src + idx[i], sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    } else {
        DevBuf<int64_t> di((size_t)n), dout((size_t)n);
        CI_CUDA(cudaMemcpyAsync(di.ptr, idx.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, s));
        launch("k_gather_i64", k_gather_i64, grid_for(n, 256), 256, 0, s, src, (const int64_t *)di.ptr, n, dout.ptr);
        CI_CUDA(cudaMemcpyAsync(out.data(), dout.ptr, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, s));
    }
    CI_CUDA(cudaStreamSynchronize(s));
    return out;
}

}  // namespace ci

// ---------------------------------------------------------------------------
// Allocation-free variant of the exclusive scan.
//
// For callers that must not allocate device memory: code running under a
// caching allocator that already owns the device's memory budget (a
// framework pool, a serving process with a fixed reservation), and code on
// a latency-critical thread where cudaMalloc / cudaFree would stall it by
// synchronising the device.  The tile sums live in one file-scope device
// array instead of a library-owned buffer; the caller still passes counts
// and offsets.
namespace ci {

constexpr int64_t kNoAllocMaxTiles = 65536;  // n <= 65536 * 4096 = 2^28 counts
static __device__ __align__(256) int64_t g_scan_tiles[kNoAllocMaxTiles];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
int64_t *g_noalloc_ptr[kMaxDevices];  // device address of g_scan_tiles per device ordinal
}  // namespace

// Device address of g_scan_tiles on the current device (looked up once per
// device; the host-side name is only a stand-in for the device symbol).
static int64_t *noalloc_scratch() {
    int dev = 0;
    CI_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) fail(CI_ERR_CAPACITY, "device ordinal %d above %d", dev, kMaxDevices);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        CI_CUDA(cudaGetSymbolAddress(&p, g_scan_tiles));
        g_noalloc_ptr[dev] = (int64_t *)p;
    }
    return g_noalloc_ptr[dev];
}

}  // namespace ci

extern "C" ci_status ci_exclusive_scan_noalloc(const int32_t *counts, int64_t n, int64_t *offsets,
                                               void *stream) {
    return ci::guard([&] {
        using namespace ci;
        if (n < 0) fail(CI_ERR_INVALID_ARG, "n < 0");
        if (!offsets || (n > 0 && !counts)) fail(CI_ERR_INVALID_ARG, "counts/offsets are NULL");
        const int64_t nb = (n + kTile - 1) / kTile;
        if (nb > kNoAllocMaxTiles)
            fail(CI_ERR_CAPACITY, "ci_exclusive_scan_noalloc: n = %lld exceeds the maximum %lld counts",
                 (long long)n, (long long)(kNoAllocMaxTiles * kTile));
        cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
        int64_t *tiles = noalloc_scratch();
        if (n == 0) {
            launch("k_zero_total", k_zero_total, 1, 1, 0, s, offsets);
            return;
        }
        // every tile sum is written by k_tile_sums before it is read
        const bool vec = (uintptr_t)counts % 16 == 0 && (uintptr_t)offsets % 16 == 0;
        launch("k_tile_sums", vec ? k_tile_sums<true> : k_tile_sums<false>, (unsigned)nb, kScanThreads, 0, s, counts,
               n, tiles);
        launch("k_scan_sums", k_scan_sums, 1, kScanThreads, 0, s, tiles, nb);
        launch("k_tile_apply", vec ? k_tile_apply<true> : k_tile_apply<false>, (unsigned)nb, kScanThreads, 0, s,
               counts, n, (const int64_t *)tiles, offsets);
    });
}
