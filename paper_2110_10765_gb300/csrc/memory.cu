// Device memory of the library: one stream-ordered pool per device.
// Allocation and release are ordered on a stream, so the build pipeline
// drops its temporaries without synchronising and reuses freed blocks
// without calling into the driver again.
#include <mutex>

#include "common.cuh"

namespace ci {

static thread_local cudaStream_t t_stream = nullptr;
static thread_local bool t_release_legacy = false;

cudaStream_t current_stream() { return t_stream; }
StreamScope::StreamScope(cudaStream_t s) : prev(t_stream) { t_stream = s; }
StreamScope::~StreamScope() { t_stream = prev; }

HandleRelease::HandleRelease() : prev(t_release_legacy) {
    if (cudaDeviceSynchronize() != cudaSuccess) (void)cudaGetLastError();
    t_release_legacy = true;
}
HandleRelease::~HandleRelease() { t_release_legacy = prev; }

namespace {
constexpr int kMaxDev = 64;
constexpr uint64_t kKeepBytes = 16ull << 30;  // freed memory kept for reuse
cudaMemPool_t g_pool[kMaxDev];
bool g_made[kMaxDev];
std::mutex g_mu;
}  // namespace

static cudaMemPool_t device_pool() {
    int dev = 0;
    CI_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDev) fail(CI_ERR_CAPACITY, "device %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_made[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        CI_CUDA(cudaMemPoolCreate(&g_pool[dev], &props));
        uint64_t keep = kKeepBytes;
        CI_CUDA(cudaMemPoolSetAttribute(g_pool[dev], cudaMemPoolAttrReleaseThreshold, &keep));
        g_made[dev] = true;
    }
    return g_pool[dev];
}

void *pool_alloc(size_t bytes, cudaStream_t s) {
    cudaMemPool_t pool = device_pool();
    void *p = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync(&p, bytes, pool, s);
    if (e == cudaErrorMemoryAllocation) {
        // blocks released on other streams may still be pending: wait for
        // them, hand unused memory back, and try once more
        (void)cudaGetLastError();
        CI_CUDA(cudaDeviceSynchronize());
        CI_CUDA(cudaMemPoolTrimTo(pool, 0));
        e = cudaMallocFromPoolAsync(&p, bytes, pool, s);
    }
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        fail(e == cudaErrorMemoryAllocation ? CI_ERR_OOM : CI_ERR_CUDA, "device allocation of %zu bytes failed: %s",
             bytes, cudaGetErrorString(e));
    }
    return p;
}

void pool_free(void *p, cudaStream_t s) {
    if (cudaFreeAsync(p, t_release_legacy ? nullptr : s) != cudaSuccess) (void)cudaGetLastError();
}

}  // namespace ci
