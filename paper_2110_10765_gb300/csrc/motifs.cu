// The paper's motif benchmarks in GB300 form:
//  * Sec. 2.2, Fig. 5: the serial prefix sum on the device (one thread, the
//    control the parallel scan of Eq. 1 is measured against);
//  * Sec. 2.3, Listing 7, Fig. 6: filling a shared array from per-row
//    offsets.  Row i stores every j in 1..m with j mod p == 0.  Its slot is
//    offset(i) + (rank of j among the stored ones) - 1, known without an
//    atomic counter, so rows come out ascending and the fill is
//    deterministic;
//  * Sec. 2.4, Eq. 2, Listings 8-9, Fig. 7: the small-array reduction
//    a(k) = sum_i sum_j x(k,i) y(k,j), k < m, over all n^2 pairs (x, y
//    column-major m x n, FP32 values).  Each lane keeps its share of the m
//    sums in registers (the paper's "scalar reductions" form), blocks add
//    their warps in shared memory and the grid's partials are summed in a
//    fixed order, in FP64.
#include "problem.cuh"

namespace ci {

namespace {

__global__ void k_scan_serial(const int32_t *__restrict__ x, int64_t n, int64_t *__restrict__ y) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    int64_t s = 0;
    y[0] = 0;
    int64_t i = 0;
    for (; i + 8 <= n; i += 8) {   // eight loads in flight, the adds in order
        int32_t v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = x[i + u];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            s += v[u];
            y[i + u + 1] = s;
        }
    }
    for (; i < n; ++i) {
        s += x[i];
        y[i + 1] = s;
    }
}

// one warp per row: the stored j are p, 2p, ..., (m/p) p
__global__ void k_fill_shared(const int64_t *__restrict__ offset, int64_t n, int m, int p, int32_t *__restrict__ arr) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int cnt = m / p;
    for (int64_t i = warp; i < n; i += nwarps) {
        int32_t *row = arr + offset[i];
        for (int t = lane; t < cnt; t += 32) row[t] = (t + 1) * p;
    }
}

constexpr int kRedI = 16;      // columns i per warp
constexpr int kRedWarps = 8;

// Block (bi, bj): columns i in [bi*128, bi*128+128) (16 per warp), columns j
// in its chunk.  Lane l owns k = l, l + 32, ... (M/32 of them, M >= 32) or, for
// M < 32, k = l % M with the lanes split over i.
template <int M>
__global__ void __launch_bounds__(256) k_array_reduce(const float *__restrict__ x, const float *__restrict__ y,
                                                      int64_t n, int64_t jchunk, double *__restrict__ part) {
    constexpr int KL = M >= 32 ? M / 32 : 1;      // k per lane
    constexpr int LG = M >= 32 ? 1 : 32 / M;      // lane groups splitting the i of a warp
    __shared__ float red[kRedWarps][32 * KL];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int kb = M >= 32 ? lane : lane % M;
    const int grp = M >= 32 ? 0 : lane / M;
    const int64_t i0 = ((int64_t)blockIdx.x * kRedWarps + w) * kRedI;
    const int64_t j0 = (int64_t)blockIdx.y * jchunk, j1 = min(n, j0 + jchunk);
    float xr[kRedI / LG > 0 ? kRedI / LG : 1][KL];
    constexpr int NI = kRedI / LG > 0 ? kRedI / LG : 1;
#pragma unroll
    for (int a = 0; a < NI; ++a) {
        const int64_t i = i0 + grp + (int64_t)a * LG;
#pragma unroll
        for (int c = 0; c < KL; ++c) xr[a][c] = i < n ? x[i * M + kb + 32 * c] : 0.f;
    }
    float acc[KL];
#pragma unroll
    for (int c = 0; c < KL; ++c) acc[c] = 0.f;
    for (int64_t j = j0; j < j1; ++j) {
#pragma unroll
        for (int c = 0; c < KL; ++c) {
            const float yv = y[j * M + kb + 32 * c];
#pragma unroll
            for (int a = 0; a < NI; ++a) acc[c] = fmaf(xr[a][c], yv, acc[c]);
        }
    }
#pragma unroll
    for (int c = 0; c < KL; ++c) red[w][lane + 32 * c] = acc[c];
    __syncthreads();
    // block partial: a(k) over the warps and (M < 32) the lane groups
    for (int k = threadIdx.x; k < M; k += blockDim.x) {
        double s = 0.0;
        for (int ww = 0; ww < kRedWarps; ++ww) {
            if (M >= 32) {
                s += red[ww][k];
            } else {
                for (int g = 0; g < LG; ++g) s += red[ww][g * M + k];
            }
        }
        part[((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * M + k] = s;
    }
}

__global__ void k_array_reduce_final(const double *__restrict__ part, int64_t nblk, int m, float *__restrict__ a) {
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        double s = 0.0;
        for (int64_t b = 0; b < nblk; ++b) s += part[b * m + k];
        a[k] = (float)s;
    }
}

template <int M>
void launch_reduce(const float *x, const float *y, int64_t n, float *a, cudaStream_t s) {
    const int64_t bi = (n + kRedI * kRedWarps - 1) / (kRedI * kRedWarps);
    // enough blocks for every SM several times over: split the j range
    int64_t nc = std::max<int64_t>(1, ((int64_t)sm_count() * 8 + bi - 1) / bi);
    nc = std::min<int64_t>(nc, std::min<int64_t>(n, 65535));
    const int64_t jchunk = (n + nc - 1) / nc;
    nc = (n + jchunk - 1) / jchunk;
    if (bi > INT32_MAX) fail(CI_ERR_CAPACITY, "array reduction grid too large (n = %lld)", (long long)n);
    DevBuf<double> part((size_t)(bi * nc * M));
    launch("k_array_reduce", k_array_reduce<M>, dim3((unsigned)bi, (unsigned)nc), 256, 0, s, x, y, n, jchunk,
           part.ptr);
    launch("k_array_reduce_final", k_array_reduce_final, 1, 256, 0, s, (const double *)part.ptr, bi * nc, M, a);
}

}  // namespace

}  // namespace ci

extern "C" ci_status ci_scan_serial(const int32_t *counts, int64_t n, int64_t *offsets, void *stream) {
    return ci::guard([&] {
        cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
        ci::StreamScope scope(s);
        if (n < 0) ci::fail(CI_ERR_INVALID_ARG, "n < 0");
        if (!offsets || !ci::is_device_pointer(offsets) || (n > 0 && (!counts || !ci::is_device_pointer(counts))))
            ci::fail(CI_ERR_INVALID_ARG, "counts and offsets must be device pointers");
        ci::launch("k_scan_serial", ci::k_scan_serial, 1, 32, 0, s, counts, n, offsets);
        CI_CUDA(cudaStreamSynchronize(s));
    });
}

extern "C" ci_status ci_fill_shared(const int64_t *offset, int64_t n, int32_t m, int32_t p, int32_t *arr,
                                    void *stream) {
    return ci::guard([&] {
        cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
        ci::StreamScope scope(s);
        if (n < 0 || m < 0 || p < 1) ci::fail(CI_ERR_INVALID_ARG, "need n >= 0, m >= 0, p >= 1");
        if (n == 0) return;
        if (!offset || !arr || !ci::is_device_pointer(offset) || !ci::is_device_pointer(arr))
            ci::fail(CI_ERR_INVALID_ARG, "offset and arr must be device pointers");
        ci::launch("k_fill_shared", ci::k_fill_shared, ci::grid_for(n * 32, 256, ci::sm_count() * 16), 256, 0, s,
                   offset, n, (int)m, (int)p, arr);
        CI_CUDA(cudaStreamSynchronize(s));
    });
}

extern "C" ci_status ci_array_reduction(const float *x, const float *y, int64_t n, int32_t m, float *a,
                                        void *stream) {
    return ci::guard([&] {
        cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
        ci::StreamScope scope(s);
        if (n < 0) ci::fail(CI_ERR_INVALID_ARG, "n < 0");
        if (!a || !ci::is_device_pointer(a)) ci::fail(CI_ERR_INVALID_ARG, "a must be a device pointer");
        if (n > 0 && (!x || !y || !ci::is_device_pointer(x) || !ci::is_device_pointer(y)))
            ci::fail(CI_ERR_INVALID_ARG, "x and y must be device pointers");
        if (m != 8 && m != 16 && m != 32 && m != 64 && m != 128 && m != 256)
            ci::fail(CI_ERR_INVALID_ARG, "m must be 8, 16, 32, 64, 128 or 256 (got %d)", m);
        if (n == 0) {
            CI_CUDA(cudaMemsetAsync(a, 0, sizeof(float) * m, s));
            CI_CUDA(cudaStreamSynchronize(s));
            return;
        }
        switch (m) {
            case 8: ci::launch_reduce<8>(x, y, n, a, s); break;
            case 16: ci::launch_reduce<16>(x, y, n, a, s); break;
            case 32: ci::launch_reduce<32>(x, y, n, a, s); break;
            case 64: ci::launch_reduce<64>(x, y, n, a, s); break;
            case 128: ci::launch_reduce<128>(x, y, n, a, s); break;
            case 256: ci::launch_reduce<256>(x, y, n, a, s); break;
            default: ci::fail(CI_ERR_INVALID_ARG, "m must be 8, 16, 32, 64, 128 or 256 (got %d)", m);
        }
        CI_CUDA(cudaStreamSynchronize(s));
    });
}
