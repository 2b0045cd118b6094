// Shared internals of libmfdci: status handling, device buffers, bit helpers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/mfdci.h"

namespace ci {

// ------------------------------------------------------------------ errors

// Exception used inside the library; converted to ci_status at the ABI.
struct Error : std::runtime_error {
    ci_status status;
    Error(ci_status s, const std::string &m) : std::runtime_error(m), status(s) {}
};

[[noreturn]] void fail(ci_status s, const char *fmt, ...);
void set_last_error(const std::string &m);

#define CI_CUDA(call)                                                              \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            ::ci::fail(e_ == cudaErrorMemoryAllocation ? CI_ERR_OOM : CI_ERR_CUDA, \
                       "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),     \
                       __FILE__, __LINE__);                                        \
        }                                                                          \
    } while (0)

#define CI_CHECK_LAUNCH() CI_CUDA(cudaGetLastError())

// Run f and convert exceptions to a status (the body of every ABI call).
template <class F>
ci_status guard(F &&f) {
    try {
        f();
        return CI_OK;
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.status;
    } catch (const std::bad_alloc &) {
        set_last_error("host allocation failed");
        return CI_ERR_OOM;
    } catch (const std::exception &e) {
        set_last_error(e.what());
        return CI_ERR_INTERNAL;
    } catch (...) {
        set_last_error("unknown exception");
        return CI_ERR_INTERNAL;
    }
}

// ------------------------------------------------------------------ memory

// Device memory comes from one stream-ordered pool per device
// (cudaMallocFromPoolAsync / cudaFreeAsync).  A buffer is allocated on the
// stream current on the calling thread and released on that same stream,
// so a temporary needs no synchronisation before it is dropped and freed
// blocks are reused without a round trip to the driver.  Every ABI call
// that takes a stream makes it current (StreamScope) for its duration;
// without one the legacy default stream is current.
cudaStream_t current_stream();
struct StreamScope {
    cudaStream_t prev;
    explicit StreamScope(cudaStream_t s);
    ~StreamScope();
    StreamScope(const StreamScope &) = delete;
    StreamScope &operator=(const StreamScope &) = delete;
};
void *pool_alloc(size_t bytes, cudaStream_t s);
void pool_free(void *p, cudaStream_t s);
// Handle destruction: waits for the device, then releases every buffer on
// the legacy default stream while it is alive (the stream a buffer was
// allocated on may no longer exist).
struct HandleRelease {
    bool prev;
    HandleRelease();
    ~HandleRelease();
    HandleRelease(const HandleRelease &) = delete;
    HandleRelease &operator=(const HandleRelease &) = delete;
};

// Owning device buffer from the pool.
template <class T>
struct DevBuf {
    T *ptr = nullptr;
    size_t n = 0;
    cudaStream_t st = nullptr;   // stream of the allocation and of the release
    DevBuf() = default;
    explicit DevBuf(size_t count) { alloc(count); }
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    DevBuf(DevBuf &&o) noexcept : ptr(o.ptr), n(o.n), st(o.st) { o.ptr = nullptr; o.n = 0; }
    DevBuf &operator=(DevBuf &&o) noexcept {
        if (this != &o) { release(); ptr = o.ptr; n = o.n; st = o.st; o.ptr = nullptr; o.n = 0; }
        return *this;
    }
    ~DevBuf() { release(); }
    void alloc(size_t count) {
        release();
        if (count == 0) count = 1;  // keep a valid pointer for empty arrays
        st = current_stream();
        ptr = static_cast<T *>(pool_alloc(count * sizeof(T), st));
        n = count;
    }
    void ensure(size_t count) { if (n < count || ptr == nullptr) alloc(count); }
    void release() {
        if (ptr) pool_free(ptr, st);
        ptr = nullptr;
        n = 0;
    }
    void upload(const std::vector<T> &h, cudaStream_t s) {
        alloc(h.size());
        if (!h.empty())
            CI_CUDA(cudaMemcpyAsync(ptr, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    }
    size_t bytes() const { return n * sizeof(T); }
};

bool is_device_pointer(const void *p);

// Copy count elements to a destination that may be host or device memory.
void copy_out(void *dst, const void *src_dev, size_t bytes, cudaStream_t s);

inline int grid_for(int64_t work, int per_block, int cap = 152 * 16) {
    int64_t g = (work + per_block - 1) / per_block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

int sm_count();

// ------------------------------------------------------------------ bits

constexpr int kMaxWords = 4;   // S <= 256
constexpr int kMaxA = 16;      // particles per species

// Bit string of one species determinant (W <= 4 words).
struct Bits {
    uint64_t w[kMaxWords];
};

__host__ __device__ inline int popc64(uint64_t x) {
#ifdef __CUDA_ARCH__
    return __popcll(x);
#else
    return __builtin_popcountll(x);
#endif
}

// Mask of the states strictly below state o (o < 64*W).
__host__ __device__ inline uint64_t below_mask_word(int o, int word) {
    int lo = word * 64;
    if (o <= lo) return 0ull;
    if (o >= lo + 64) return ~0ull;
    return (1ull << (o - lo)) - 1ull;
}

}  // namespace ci

namespace ci {

// ------------------------------------------------------------------ tracing

// When tracing is on (ci_trace_enable), every kernel launch of the library
// is bracketed by two CUDA events on the launch stream; ci_trace_read sums
// their elapsed times per kernel name.
bool trace_on();
void trace_begin(const char *name, cudaStream_t s, void **token);
void trace_end(void *token, cudaStream_t s);

// Programmatic dependent launch: a kernel launched by launch_pdl may be
// set up while the kernel before it on the stream drains, so it must call
// pdl_wait() before its first access to memory that kernel wrote (every
// kernel launched this way calls it first thing; without the launch
// attribute the wait returns at once).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <class K, class... Args>
inline void launch_pdl(const char *name, K kernel, dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args... args) {
    void *tok = nullptr;
    if (trace_on()) trace_begin(name, s, &tok);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, args...);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (tok) trace_end(tok, s);
    if (e != cudaSuccess)
        fail(e == cudaErrorMemoryAllocation ? CI_ERR_OOM : CI_ERR_CUDA, "launch of %s failed: %s", name,
             cudaGetErrorString(e));
}

template <class K, class... Args>
inline void launch(const char *name, K kernel, dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                   Args... args) {
    void *tok = nullptr;
    if (trace_on()) trace_begin(name, s, &tok);
    kernel<<<grid, block, smem, s>>>(args...);
    cudaError_t e = cudaGetLastError();
    if (tok) trace_end(tok, s);
    if (e != cudaSuccess)
        fail(e == cudaErrorMemoryAllocation ? CI_ERR_OOM : CI_ERR_CUDA, "launch of %s failed: %s", name,
             cudaGetErrorString(e));
}

}  // namespace ci
