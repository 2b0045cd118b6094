// SpMM Y = H X over the CSR matrix (Fig. 2, optional FMA of H_ij with the
// j-th vector element), X and Y row-major [dim][NV].  One warp per row:
// lanes stride over the row's nonzeros with coalesced col/val loads and one
// vector load of X's row per nonzero, then a butterfly reduction.
#include <cuda_bf16.h>

#include "problem.cuh"

namespace ci {

template <class TX, int NV>
struct VecLoad {
    __device__ static void load(const TX *p, TX *x) {
#pragma unroll
        for (int i = 0; i < NV; ++i) x[i] = p[i];
    }
};
template <>
struct VecLoad<float, 8> {
    __device__ static void load(const float *p, float *x) {
        float4 a = __ldg(reinterpret_cast<const float4 *>(p));
        float4 b = __ldg(reinterpret_cast<const float4 *>(p) + 1);
        x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
        x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
    }
};
template <>
struct VecLoad<float, 4> {
    __device__ static void load(const float *p, float *x) {
        float4 a = __ldg(reinterpret_cast<const float4 *>(p));
        x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
    }
};
template <>
struct VecLoad<double, 8> {
    __device__ static void load(const double *p, double *x) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            double2 a = __ldg(reinterpret_cast<const double2 *>(p) + i);
            x[2 * i] = a.x; x[2 * i + 1] = a.y;
        }
    }
};

// Value of a stored element in the arithmetic type (bf16 widened to float).
__device__ __forceinline__ float load_val(const float *p) { return __ldcs(p); }
__device__ __forceinline__ float load_val(const double *p) { return (float)__ldcs(p); }
__device__ __forceinline__ float load_val(const __nv_bfloat16 *p) {
    return __bfloat162float(__ushort_as_bfloat16(__ldcs(reinterpret_cast<const unsigned short *>(p))));
}
template <class TX, class TV>
__device__ __forceinline__ TX load_as(const TV *p) { return (TX)load_val(p); }
template <>
__device__ __forceinline__ double load_as<double, double>(const double *p) { return __ldcs(p); }

// row_scale: null, or a per-row factor of the stored values (BF16 form)
template <class TV, class TX, int NV>
__global__ void __launch_bounds__(256) k_spmm(const int64_t *__restrict__ bnd, const int64_t *__restrict__ rp,
                                              const int32_t *__restrict__ col, const TV *__restrict__ val,
                                              const TX *__restrict__ X, TX *__restrict__ Y,
                                              const float *__restrict__ row_scale) {
    pdl_wait();
    constexpr int U = 4;  // nonzeros in flight per lane
    const int lane = threadIdx.x & 31;
    const int64_t r_end = bnd[blockIdx.x + 1];   // rows as in k_spmm8_half
    for (int64_t r = bnd[blockIdx.x] + (threadIdx.x >> 5); r < r_end; r += blockDim.x >> 5) {
        TX acc[NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) acc[i] = 0;
        const int64_t e1 = rp[r + 1];
        int64_t e = rp[r] + lane;
        for (; e + 32 * (U - 1) < e1; e += 32 * U) {
            int c[U];
            TX v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {  // col/val stream once: evict-first loads
                c[u] = __ldcs(col + e + 32 * u);
                v[u] = load_as<TX>(val + e + 32 * u);
            }
            TX x[U][NV];
#pragma unroll
            for (int u = 0; u < U; ++u) VecLoad<TX, NV>::load(X + (int64_t)c[u] * NV, x[u]);
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int i = 0; i < NV; ++i) acc[i] = fma(v[u], x[u][i], acc[i]);
        }
        for (; e < e1; e += 32) {
            const int c = __ldcs(col + e);
            const TX v = load_as<TX>(val + e);
            TX x[NV];
            VecLoad<TX, NV>::load(X + (int64_t)c * NV, x);
#pragma unroll
            for (int i = 0; i < NV; ++i) acc[i] = fma(v, x[i], acc[i]);
        }
#pragma unroll
        for (int i = 0; i < NV; ++i) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], o);
        }
        if (lane < NV) {
            TX y = acc[0];
#pragma unroll
            for (int i = 1; i < NV; ++i)
                if (lane == i) y = acc[i];
            Y[r * NV + lane] = row_scale ? y * (TX)row_scale[r] : y;
        }
    }
}

// Eight-vector float SpMM with two lanes per nonzero: lane pair (2j, 2j+1)
// shares nonzero e and each lane gathers one 16-byte half of X's row, so a
// warp instruction touches 16 rows of X (one sector each) instead of
// issuing two loads per row.  Lanes accumulate their four components over
// the row's nonzeros j, j+16, ... in ascending order, then reduce over the
// 16 lanes of the same parity.  CTA b takes the consecutive rows
// [bnd[b], bnd[b+1]) (about kSpmmWork nonzeros, see k_spmm_bounds) and its
// eight warps interleave over them: the rows a CTA holds at once mostly
// belong to one proton-state block, whose rows share many X rows (reused
// from L1), and many short CTAs of even work keep every SM busy to the end.

// row_scale: null, or a per-row factor of the stored values (BF16 form)
// TY: float, or double for Y written in FP64 (the Lanczos block W).
template <class TV, class TY = float>
__global__ void __launch_bounds__(256) k_spmm8_half(const int64_t *__restrict__ bnd, const int64_t *__restrict__ rp,
                                                    const int32_t *__restrict__ col, const TV *__restrict__ val,
                                                    const float *__restrict__ X, TY *__restrict__ Y,
                                                    const float *__restrict__ row_scale) {
    pdl_wait();
    constexpr int U = 4;  // nonzeros in flight per lane pair
    const int lane = threadIdx.x & 31, half = lane & 1, pair = lane >> 1;
    const int64_t r_end = bnd[blockIdx.x + 1];
    const float4 *X4 = reinterpret_cast<const float4 *>(X);
    for (int64_t r = bnd[blockIdx.x] + (threadIdx.x >> 5); r < r_end; r += blockDim.x >> 5) {
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        const int64_t e1 = rp[r + 1];
        int64_t e = rp[r] + pair;
        for (; e + 16 * (U - 1) < e1; e += 16 * U) {
            int c[U];
            float v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                c[u] = __ldcs(col + e + 16 * u);
                v[u] = load_val(val + e + 16 * u);
            }
            float4 x[U];
#pragma unroll
            for (int u = 0; u < U; ++u) x[u] = __ldg(X4 + (int64_t)c[u] * 2 + half);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                a0 = fmaf(v[u], x[u].x, a0);
                a1 = fmaf(v[u], x[u].y, a1);
                a2 = fmaf(v[u], x[u].z, a2);
                a3 = fmaf(v[u], x[u].w, a3);
            }
        }
        for (; e < e1; e += 16) {
            const int c = __ldcs(col + e);
            const float v = load_val(val + e);
            const float4 x = __ldg(X4 + (int64_t)c * 2 + half);
            a0 = fmaf(v, x.x, a0);
            a1 = fmaf(v, x.y, a1);
            a2 = fmaf(v, x.z, a2);
            a3 = fmaf(v, x.w, a3);
        }
#pragma unroll
        for (int o = 16; o > 1; o >>= 1) {
            a0 += __shfl_xor_sync(0xffffffffu, a0, o);
            a1 += __shfl_xor_sync(0xffffffffu, a1, o);
            a2 += __shfl_xor_sync(0xffffffffu, a2, o);
            a3 += __shfl_xor_sync(0xffffffffu, a3, o);
        }
        if (lane < 2) {
            const float sc = row_scale ? row_scale[r] : 1.f;
            if constexpr (sizeof(TY) == 4) {
                reinterpret_cast<float4 *>(Y)[r * 2 + half] = make_float4(a0 * sc, a1 * sc, a2 * sc, a3 * sc);
            } else {
                double2 *y = reinterpret_cast<double2 *>(Y) + r * 4 + half * 2;
                y[0] = make_double2(a0 * sc, a1 * sc);
                y[1] = make_double2(a2 * sc, a3 * sc);
            }
        }
    }
}

// ---- half storage (Fig. 2, optional FMA: the stored H_ij also updates the
// j-th output with the i-th input).  Row i keeps the columns j >= i; the
// stored element adds H_ij X_j to Y_i and, for j > i, H_ij X_i to Y_j.  Y is
// zeroed first and every update is an atomic add, so the summation order
// (and the last bits of Y) vary from run to run.

// 8 FP32 vectors, two lanes per nonzero as k_spmm8_half, vector atomics.
template <class TV>
__global__ void __launch_bounds__(256) k_spmm8_upper(int64_t dim, const int64_t *__restrict__ rp,
                                                     const int32_t *__restrict__ col, const TV *__restrict__ val,
                                                     const float *__restrict__ X, float *__restrict__ Y,
                                                     const float *__restrict__ row_scale) {
    const int lane = threadIdx.x & 31, half = lane & 1, pair = lane >> 1;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const float4 *X4 = reinterpret_cast<const float4 *>(X);
    float4 *Y4 = reinterpret_cast<float4 *>(Y);
    for (int64_t r = warp; r < dim; r += nwarps) {
        const float sc = row_scale ? row_scale[r] : 1.f;
        const float4 xr = __ldg(X4 + r * 2 + half);
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        const int64_t e1 = rp[r + 1];
        for (int64_t e = rp[r] + pair; e < e1; e += 16) {
            const int c = __ldcs(col + e);
            const float v = load_val(val + e) * sc;
            const float4 x = __ldg(X4 + (int64_t)c * 2 + half);
            a0 = fmaf(v, x.x, a0);
            a1 = fmaf(v, x.y, a1);
            a2 = fmaf(v, x.z, a2);
            a3 = fmaf(v, x.w, a3);
            if (c != r) atomicAdd(Y4 + (int64_t)c * 2 + half, make_float4(v * xr.x, v * xr.y, v * xr.z, v * xr.w));
        }
#pragma unroll
        for (int o = 16; o > 1; o >>= 1) {
            a0 += __shfl_xor_sync(0xffffffffu, a0, o);
            a1 += __shfl_xor_sync(0xffffffffu, a1, o);
            a2 += __shfl_xor_sync(0xffffffffu, a2, o);
            a3 += __shfl_xor_sync(0xffffffffu, a3, o);
        }
        if (lane < 2) atomicAdd(Y4 + r * 2 + half, make_float4(a0, a1, a2, a3));
    }
}

// Any vector count and type: one thread per (row, vector), scalar atomics.
template <class TV, class TX, int NV>
__global__ void k_spmm_upper(int64_t dim, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                             const TV *__restrict__ val, const TX *__restrict__ X, TX *__restrict__ Y,
                             const float *__restrict__ row_scale) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < dim * NV;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / NV;
        const int q = (int)(t - r * NV);
        const TX sc = row_scale ? (TX)row_scale[r] : (TX)1;
        const TX xr = X[r * NV + q];
        TX acc = 0;
        for (int64_t e = rp[r]; e < rp[r + 1]; ++e) {
            const int c = col[e];
            const TX v = load_as<TX>(val + e) * sc;
            acc += v * X[(int64_t)c * NV + q];
            if (c != r) atomicAdd(Y + (int64_t)c * NV + q, v * xr);
        }
        atomicAdd(Y + r * NV + q, acc);
    }
}

// Work of rows [0, r): nonzeros plus kSpmmRowCost per row (a row also costs
// its pointers and its Y store), strictly increasing in r.  Range b starts
// at the first row whose work reaches b / nb of the total; the last range
// ends at dim, so trailing empty rows are covered too.
constexpr int64_t kSpmmWork = 10240, kSpmmRowCost = 16;
__global__ void k_spmm_bounds(int64_t dim, const int64_t *__restrict__ rp, int64_t nb, int64_t *__restrict__ bnd) {
    const int64_t total = rp[dim] + kSpmmRowCost * dim;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g <= nb; g += (int64_t)gridDim.x * blockDim.x) {
        if (g == nb) {
            bnd[g] = dim;
            continue;
        }
        const int64_t target = total / nb * g + total % nb * g / nb;   // floor(total * g / nb)
        int64_t lo = 0, hi = dim;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (rp[mid] + kSpmmRowCost * mid < target) lo = mid + 1; else hi = mid;
        }
        bnd[g] = lo;
    }
}

void spmm_prepare(Matrix *m, cudaStream_t s) {
    if (m->upper) return;
    const int64_t total = m->nnz + kSpmmRowCost * m->dim;
    m->spmm_nb = std::max<int64_t>(1, (total + kSpmmWork - 1) / kSpmmWork);
    if (m->spmm_nb > INT32_MAX) fail(CI_ERR_CAPACITY, "matrix too large for the SpMM's row ranges");
    m->spmm_bnd.alloc((size_t)m->spmm_nb + 1);
    launch("k_spmm_bounds", k_spmm_bounds, grid_for(m->spmm_nb + 1, 256), 256, 0, s, m->dim, m->row_ptr.ptr,
           m->spmm_nb, m->spmm_bnd.ptr);
    CI_CHECK_LAUNCH();
}

template <class TV, class TX, int NV>
static void launch_spmm_upper(const Matrix *m, const void *X, void *Y, cudaStream_t s) {
    CI_CUDA(cudaMemsetAsync(Y, 0, sizeof(TX) * (size_t)m->dim * NV, s));
    const float *scale = m->vtype == CI_BF16_ROWSCALE ? m->row_scale.ptr : nullptr;
    if (NV == 8 && sizeof(TX) == 4) {
        launch("k_spmm_upper", k_spmm8_upper<TV>, grid_for(m->dim * 32, 256, sm_count() * 8), 256, 0, s, m->dim,
               m->row_ptr.ptr, m->col.ptr, (const TV *)m->val.ptr, (const float *)X, (float *)Y, scale);
        return;
    }
    launch("k_spmm_upper", k_spmm_upper<TV, TX, NV>, grid_for(m->dim * NV, 256), 256, 0, s, m->dim, m->row_ptr.ptr,
           m->col.ptr, (const TV *)m->val.ptr, (const TX *)X, (TX *)Y, scale);
}

template <class TV, class TX, int NV>
static void launch_spmm(const Matrix *m, const void *X, void *Y, cudaStream_t s) {
    if (m->upper) {
        launch_spmm_upper<TV, TX, NV>(m, X, Y, s);
        return;
    }
    if (!m->spmm_bnd.ptr) fail(CI_ERR_INTERNAL, "matrix without SpMM row ranges");
    const int grid = (int)m->spmm_nb;
    const int64_t *bnd = m->spmm_bnd.ptr;
    const float *scale = m->vtype == CI_BF16_ROWSCALE ? m->row_scale.ptr : nullptr;
    if (NV == 8 && sizeof(TX) == 4) {
        launch_pdl("k_spmm", k_spmm8_half<TV>, grid, 256, 0, s, bnd, m->row_ptr.ptr, m->col.ptr, (const TV *)m->val.ptr,
               (const float *)X, (float *)Y, (const float *)scale);
        return;
    }
    launch_pdl("k_spmm", k_spmm<TV, TX, NV>, grid, 256, 0, s, bnd, m->row_ptr.ptr, m->col.ptr, (const TV *)m->val.ptr,
           (const TX *)X, (TX *)Y, (const float *)scale);
}

bool apply_matrix8_f64out(const Matrix *m, const float *X, double *W, cudaStream_t s) {
    if (m->upper || (m->vtype != CI_F32 && m->vtype != CI_BF16_ROWSCALE)) return false;
    if (m->dim == 0) return true;
    if (!m->spmm_bnd.ptr) fail(CI_ERR_INTERNAL, "matrix without SpMM row ranges");
    if (((uintptr_t)X % 16) != 0 || ((uintptr_t)W % 16) != 0) fail(CI_ERR_INVALID_ARG, "X and W must be 16-byte aligned");
    const int grid = (int)m->spmm_nb;
    if (m->vtype == CI_F32)
        launch_pdl("k_spmm", k_spmm8_half<float, double>, grid, 256, 0, s, (const int64_t *)m->spmm_bnd.ptr,
                   m->row_ptr.ptr, m->col.ptr, (const float *)m->val.ptr, X, W, (const float *)nullptr);
    else
        launch_pdl("k_spmm", k_spmm8_half<__nv_bfloat16, double>, grid, 256, 0, s, (const int64_t *)m->spmm_bnd.ptr,
                   m->row_ptr.ptr, m->col.ptr, (const __nv_bfloat16 *)m->val.ptr, X, W, (const float *)m->row_scale.ptr);
    CI_CHECK_LAUNCH();
    return true;
}

template <class TV, class TX>
static void dispatch(const Matrix *m, const void *X, void *Y, int nvec, cudaStream_t s) {
    switch (nvec) {
        case 1: launch_spmm<TV, TX, 1>(m, X, Y, s); break;
        case 2: launch_spmm<TV, TX, 2>(m, X, Y, s); break;
        case 3: launch_spmm<TV, TX, 3>(m, X, Y, s); break;
        case 4: launch_spmm<TV, TX, 4>(m, X, Y, s); break;
        case 5: launch_spmm<TV, TX, 5>(m, X, Y, s); break;
        case 6: launch_spmm<TV, TX, 6>(m, X, Y, s); break;
        case 7: launch_spmm<TV, TX, 7>(m, X, Y, s); break;
        case 8: launch_spmm<TV, TX, 8>(m, X, Y, s); break;
        default: fail(CI_ERR_INVALID_ARG, "nvec must be 1..8 (got %d)", nvec);
    }
}

// Upper triangle of a full CSR: per row the entries from the first column
// >= row (columns are ascending), counted, scanned, copied.
__global__ void k_upper_count(int64_t dim, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                              int32_t *__restrict__ cnt, int64_t *__restrict__ first) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < dim; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = rp[i], hi = rp[i + 1];
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (col[mid] < i) lo = mid + 1; else hi = mid;
        }
        first[i] = lo;
        cnt[i] = (int32_t)(rp[i + 1] - lo);
    }
}

template <class TV>
__global__ void k_upper_copy(int64_t dim, const int64_t *__restrict__ rp, const int64_t *__restrict__ first,
                             const int32_t *__restrict__ col, const TV *__restrict__ val,
                             const int64_t *__restrict__ urp, int32_t *__restrict__ ucol, TV *__restrict__ uval) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = warp; r < dim; r += nwarps) {
        const int64_t src = first[r], dst = urp[r], n = urp[r + 1] - urp[r];
        for (int64_t k = lane; k < n; k += 32) {
            ucol[dst + k] = col[src + k];
            uval[dst + k] = val[src + k];
        }
    }
}

void upper_matrix(const Matrix *full, Matrix *out, cudaStream_t s) {
    if (full->upper) fail(CI_ERR_INVALID_ARG, "the matrix already stores only its upper triangle");
    const int64_t dim = full->dim;
    out->dim = dim;
    out->vtype = full->vtype;
    out->upper = true;
    out->row_ptr.alloc((size_t)dim + 1);
    if (dim == 0) {
        CI_CUDA(cudaMemsetAsync(out->row_ptr.ptr, 0, sizeof(int64_t), s));
        out->nnz = 0;
        return;
    }
    DevBuf<int32_t> cnt((size_t)dim);
    DevBuf<int64_t> first((size_t)dim), scratch;
    launch("k_upper_count", k_upper_count, grid_for(dim, 256), 256, 0, s, dim, (const int64_t *)full->row_ptr.ptr,
           (const int32_t *)full->col.ptr, cnt.ptr, first.ptr);
    exclusive_scan_i32(cnt.ptr, dim, out->row_ptr.ptr, scratch, s);
    CI_CUDA(cudaMemcpyAsync(&out->nnz, out->row_ptr.ptr + dim, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CI_CUDA(cudaStreamSynchronize(s));
    const size_t esz = full->vtype == CI_F64 ? 8 : full->vtype == CI_F32 ? 4 : 2;
    out->col.alloc((size_t)std::max<int64_t>(out->nnz, 1));
    out->val.alloc(esz * (size_t)std::max<int64_t>(out->nnz, 1));
    const int grid = grid_for(dim * 32, 256, sm_count() * 8);
    if (esz == 8)
        launch("k_upper_copy", k_upper_copy<double>, grid, 256, 0, s, dim, (const int64_t *)full->row_ptr.ptr,
               (const int64_t *)first.ptr, (const int32_t *)full->col.ptr, (const double *)full->val.ptr,
               (const int64_t *)out->row_ptr.ptr, out->col.ptr, (double *)out->val.ptr);
    else if (esz == 4)
        launch("k_upper_copy", k_upper_copy<float>, grid, 256, 0, s, dim, (const int64_t *)full->row_ptr.ptr,
               (const int64_t *)first.ptr, (const int32_t *)full->col.ptr, (const float *)full->val.ptr,
               (const int64_t *)out->row_ptr.ptr, out->col.ptr, (float *)out->val.ptr);
    else
        launch("k_upper_copy", k_upper_copy<__nv_bfloat16>, grid, 256, 0, s, dim,
               (const int64_t *)full->row_ptr.ptr, (const int64_t *)first.ptr, (const int32_t *)full->col.ptr,
               (const __nv_bfloat16 *)full->val.ptr, (const int64_t *)out->row_ptr.ptr, out->col.ptr,
               (__nv_bfloat16 *)out->val.ptr);
    if (full->vtype == CI_BF16_ROWSCALE) {
        out->row_scale.alloc((size_t)dim);
        CI_CUDA(cudaMemcpyAsync(out->row_scale.ptr, full->row_scale.ptr, sizeof(float) * dim,
                                cudaMemcpyDeviceToDevice, s));
    }
    CI_CHECK_LAUNCH();
}

// 16 FP32 vectors (two 8-vector blocks side by side, 64-byte rows of X): one
// warp per row, four lanes per nonzero (a 16-byte quarter of the X row each),
// eight nonzeros per warp step.  One gather serves twice the vectors of the
// 8-wide kernel for the same L2 transactions.
template <class TV>
__global__ void __launch_bounds__(256) k_spmm16(const int64_t *__restrict__ bnd, const int64_t *__restrict__ rp,
                                                const int32_t *__restrict__ col, const TV *__restrict__ val,
                                                const float *__restrict__ X, float *__restrict__ Y,
                                                const float *__restrict__ row_scale) {
    const int lane = threadIdx.x & 31, q = lane & 3, grp = lane >> 2;
    const int64_t r_end = bnd[blockIdx.x + 1];   // rows as in k_spmm8_half
    const float4 *X4 = reinterpret_cast<const float4 *>(X);
    for (int64_t r = bnd[blockIdx.x] + (threadIdx.x >> 5); r < r_end; r += blockDim.x >> 5) {
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        const int64_t e1 = rp[r + 1];
        int64_t e = rp[r] + grp;
        for (; e + 8 < e1; e += 16) {   // two nonzeros in flight per lane quad
            const int c0 = __ldcs(col + e), c1 = __ldcs(col + e + 8);
            const float v0 = load_val(val + e), v1 = load_val(val + e + 8);
            const float4 x0 = __ldg(X4 + (int64_t)c0 * 4 + q), x1 = __ldg(X4 + (int64_t)c1 * 4 + q);
            a0 = fmaf(v0, x0.x, a0); a1 = fmaf(v0, x0.y, a1); a2 = fmaf(v0, x0.z, a2); a3 = fmaf(v0, x0.w, a3);
            a0 = fmaf(v1, x1.x, a0); a1 = fmaf(v1, x1.y, a1); a2 = fmaf(v1, x1.z, a2); a3 = fmaf(v1, x1.w, a3);
        }
        for (; e < e1; e += 8) {
            const int c = __ldcs(col + e);
            const float v = load_val(val + e);
            const float4 x = __ldg(X4 + (int64_t)c * 4 + q);
            a0 = fmaf(v, x.x, a0); a1 = fmaf(v, x.y, a1); a2 = fmaf(v, x.z, a2); a3 = fmaf(v, x.w, a3);
        }
#pragma unroll
        for (int o = 16; o > 2; o >>= 1) {
            a0 += __shfl_xor_sync(0xffffffffu, a0, o);
            a1 += __shfl_xor_sync(0xffffffffu, a1, o);
            a2 += __shfl_xor_sync(0xffffffffu, a2, o);
            a3 += __shfl_xor_sync(0xffffffffu, a3, o);
        }
        if (lane < 4) {
            const float sc = row_scale ? row_scale[r] : 1.f;
            reinterpret_cast<float4 *>(Y)[r * 4 + q] = make_float4(a0 * sc, a1 * sc, a2 * sc, a3 * sc);
        }
    }
}

void apply_matrix16(const Matrix *m, const float *X, float *Y, cudaStream_t s) {
    if (m->dim == 0) return;
    if (((uintptr_t)X % 16) != 0 || ((uintptr_t)Y % 16) != 0) fail(CI_ERR_INVALID_ARG, "X and Y must be 16-byte aligned");
    const float *scale = m->vtype == CI_BF16_ROWSCALE ? m->row_scale.ptr : nullptr;
    if (m->upper) fail(CI_ERR_INVALID_ARG, "the 16-vector product takes a full-storage matrix");
    if (!m->spmm_bnd.ptr) fail(CI_ERR_INTERNAL, "matrix without SpMM row ranges");
    const int grid = (int)m->spmm_nb;
    const int64_t *bnd = m->spmm_bnd.ptr;
    if (m->vtype == CI_F32)
        launch("k_spmm16", k_spmm16<float>, grid, 256, 0, s, bnd, m->row_ptr.ptr, m->col.ptr,
               (const float *)m->val.ptr, X, Y, scale);
    else if (m->vtype == CI_BF16_ROWSCALE)
        launch("k_spmm16", k_spmm16<__nv_bfloat16>, grid, 256, 0, s, bnd, m->row_ptr.ptr, m->col.ptr,
               (const __nv_bfloat16 *)m->val.ptr, X, Y, scale);
    else
        fail(CI_ERR_INVALID_ARG, "the 16-vector product takes FP32 or BF16 values");
    CI_CHECK_LAUNCH();
}

void apply_matrix(const Matrix *m, const void *X, void *Y, int nvec, cudaStream_t s) {
    if ((nvec < 1 || nvec > 8) && nvec != 16) fail(CI_ERR_INVALID_ARG, "nvec must be 1..8 or 16 (got %d)", nvec);
    if (m->dim == 0) return;
    if (!X || !Y) fail(CI_ERR_INVALID_ARG, "X and Y must be device pointers");
    if (nvec == 16) {   // two 8-vector blocks side by side, one gather per nonzero
        apply_matrix16(m, (const float *)X, (float *)Y, s);
        return;
    }
    size_t esz = m->vtype == CI_F64 ? 8 : 4;   // X and Y element size (float for F32 and BF16)
    size_t align = (nvec == 8 || nvec == 4) ? 16 : esz;
    if (((uintptr_t)X % align) != 0 || ((uintptr_t)Y % align) != 0)
        fail(CI_ERR_INVALID_ARG, "X and Y must be %zu-byte aligned", align);
    if (m->vtype == CI_F32) dispatch<float, float>(m, X, Y, nvec, s);
    else if (m->vtype == CI_F64) dispatch<double, double>(m, X, Y, nvec, s);
    else if (m->vtype == CI_BF16_ROWSCALE) dispatch<__nv_bfloat16, float>(m, X, Y, nvec, s);
    else fail(CI_ERR_INVALID_ARG, "value type %d not supported by ci_apply_H", m->vtype);
    CI_CHECK_LAUNCH();
}

}  // namespace ci
