// Block-diagonal preconditioner of LOBPCG over many-body basis orbitals
// (Sec. 2: basis states that give every nucleon the same single-particle
// orbital (n, l, j) and differ only in the magnetic projections m form one
// many-body basis orbital; the Hamiltonian's diagonal blocks over these
// groups make the preconditioner of the eigensolver).
//
//   T = blockdiag_b (H_bb - sigma_b I)^-1
//
// Each orbital block is cut into consecutive sub-blocks of at most kSubMax
// rows (its member rows ascending, split as evenly as possible), so one
// sub-block fits in shared memory.  sigma_b = sigma when H_bb - sigma I is
// positive definite (every Gauss-Jordan pivot positive); otherwise the
// sub-block's Gershgorin lower bound g_b minus a margin, which makes the
// shifted block strictly diagonally dominant, hence positive definite.  T is
// therefore symmetric positive definite, as LOBPCG requires.  The inverses
// are formed in FP64 and kept in FP32 (a preconditioner needs no more).
#include <algorithm>
#include <cmath>
#include <map>
#include <unordered_map>

#include <cuda_bf16.h>

#include "problem.cuh"

namespace ci {

namespace {

__device__ __forceinline__ double pc_val(float v) { return v; }
__device__ __forceinline__ double pc_val(double v) { return v; }
__device__ __forceinline__ double pc_val(__nv_bfloat16 v) { return __bfloat162float(v); }

__device__ __forceinline__ double block_min(double v, double *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double r = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = fmin(r, red[w]);
    return r;
}

__device__ __forceinline__ double block_max(double v, double *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double r = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = fmax(r, red[w]);
    return r;
}

// One CTA per sub-block (the sub-block ids of one size bin): gather H_bb
// from the CSR rows of its members into shared memory (FP64, row-major
// n x n), shift, invert in place by Gauss-Jordan elimination without
// pivoting (for a symmetric matrix every pivot is positive exactly when it
// is positive definite), store FP32.  Warps own rows, lanes columns.
template <class TV>
__global__ void __launch_bounds__(256) k_block_inv(const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                                                   const TV *__restrict__ val, const float *__restrict__ rscale,
                                                   const int32_t *__restrict__ rows,
                                                   const int64_t *__restrict__ sub_start,
                                                   const int32_t *__restrict__ sub_of,
                                                   const int32_t *__restrict__ loc_of,
                                                   const int64_t *__restrict__ inv_off,
                                                   const int32_t *__restrict__ ids, bool upper, double sigma,
                                                   float *__restrict__ inv, double *__restrict__ shift,
                                                   int32_t *__restrict__ status) {
    extern __shared__ double sm[];
    __shared__ double red[8];
    const int sb = ids[blockIdx.x];
    const int64_t r0 = sub_start[sb];
    const int n = (int)(sub_start[sb + 1] - r0);
    const int nn = n * n;
    double *A = sm;          // [n][n]
    double *ck = A + nn;     // column k before the step
    double *rk = ck + n;     // row k before the step
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;

    double gersh = 0.0, norm = 0.0, used = sigma;
    bool ok = false;
    for (int attempt = 0; attempt < 2 && !ok; ++attempt) {
        for (int t = threadIdx.x; t < nn; t += blockDim.x) A[t] = 0.0;
        __syncthreads();
        for (int li = warp; li < n; li += nwarp) {
            const int r = rows[r0 + li];
            const double sc = rscale ? (double)rscale[r] : 1.0;
            const int64_t e1 = rp[r + 1];
            // four entries per lane in flight: the column, its sub-block and
            // the value are independent loads
            for (int64_t e = rp[r] + lane; e < e1; e += 128) {
                int c[4], b[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) c[u] = e + 32 * u < e1 ? col[e + 32 * u] : -1;
#pragma unroll
                for (int u = 0; u < 4; ++u) b[u] = c[u] >= 0 ? sub_of[c[u]] : -1;
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (b[u] == sb) {
                        const int lc = loc_of[c[u]];
                        const double v = pc_val(val[e + 32 * u]) * sc;
                        A[li * n + lc] = v;
                        // half storage: the mirror element (only the upper one is stored)
                        if (upper && lc != li) A[lc * n + li] = v;
                    }
            }
        }
        __syncthreads();
        if (attempt == 0) {
            // Gershgorin lower bound and largest absolute row sum of H_bb
            double g = INFINITY, a = 0.0;
            for (int i = warp; i < n; i += nwarp) {
                double off = 0.0;
                for (int j = lane; j < n; j += 32)
                    if (j != i) off += fabs(A[i * n + j]);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) off += __shfl_xor_sync(0xffffffffu, off, o);
                g = fmin(g, A[i * n + i] - off);
                a = fmax(a, off + fabs(A[i * n + i]));
            }
            gersh = block_min(g, red);
            norm = block_max(a, red);
            used = sigma;
        } else {
            const double eta = 1e-3 * fmax(fmax(norm, fabs(sigma)), 1e-300);
            used = fmin(sigma, gersh) - eta;
        }
        for (int i = threadIdx.x; i < n; i += blockDim.x) A[i * n + i] -= used;
        __syncthreads();
        const double tol = 1e-12 * (norm + fabs(used));
        ok = true;
        for (int k = 0; k < n; ++k) {
            const double p = A[k * n + k];
            if (!(p > tol)) {   // the same value in every thread: a uniform exit
                ok = false;
                break;
            }
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                ck[i] = A[i * n + k];
                rk[i] = A[k * n + i];
            }
            __syncthreads();
            const double ip = 1.0 / p;
            for (int i = warp; i < n; i += nwarp) {
                const double f = -ck[i] * ip;
                double *Ai = A + i * n;
                if (i != k) {
                    for (int j = lane; j < n; j += 32) Ai[j] = j != k ? fma(f, rk[j], Ai[j]) : f;
                } else {
                    for (int j = lane; j < n; j += 32) Ai[j] = j != k ? rk[j] * ip : ip;
                }
            }
            __syncthreads();
        }
        __syncthreads();
    }
    float *out = inv + inv_off[sb];
    for (int t = threadIdx.x; t < nn; t += blockDim.x) out[t] = ok ? (float)A[t] : 0.0f;
    if (threadIdx.x == 0) {
        shift[sb] = ok ? used : NAN;
        if (!ok) atomicExch(status, 1);
    }
}

// W[rows] = inv_b R[rows] for every sub-block b (one CTA each), R and W
// [dim][nv] FP64, the product in FP32.
__global__ void __launch_bounds__(256) k_block_apply(const int32_t *__restrict__ rows,
                                                     const int64_t *__restrict__ sub_start,
                                                     const int64_t *__restrict__ inv_off,
                                                     const float *__restrict__ inv, int nv,
                                                     const double *__restrict__ R, double *__restrict__ W) {
    extern __shared__ float fs[];
    const int sb = blockIdx.x;
    const int64_t r0 = sub_start[sb];
    const int n = (int)(sub_start[sb + 1] - r0);
    float *Ai = fs;            // [n][n]
    float *Rs = fs + n * n;    // [n][nv]
    const float *src = inv + inv_off[sb];
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) Ai[t] = src[t];
    for (int t = threadIdx.x; t < n * nv; t += blockDim.x) {
        const int li = t / nv, v = t - li * nv;
        Rs[t] = (float)R[(int64_t)rows[r0 + li] * nv + v];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < n * nv; t += blockDim.x) {
        const int li = t / nv, v = t - li * nv;
        float acc = 0.f;
        for (int j = 0; j < n; ++j) acc = fmaf(Ai[li * n + j], Rs[j * nv + v], acc);
        W[(int64_t)rows[r0 + li] * nv + v] = acc;
    }
}

__global__ void k_row_shift(int64_t dim, const int32_t *__restrict__ sub_of, const double *__restrict__ shift,
                            double *__restrict__ out) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < dim; r += (int64_t)gridDim.x * blockDim.x)
        out[r] = shift[sub_of[r]];
}

size_t inv_smem(int smax) { return sizeof(double) * ((size_t)smax * smax + 2 * (size_t)smax); }
size_t apply_smem(int smax, int nv) { return sizeof(float) * ((size_t)smax * smax + (size_t)smax * nv); }

}  // namespace

void orbital_blocks(Problem *p, const int32_t *sp_orbital, int32_t *block, int64_t *nblocks, cudaStream_t s) {
    if (!sp_orbital) fail(CI_ERR_INVALID_ARG, "sp_orbital is NULL");
    if (!nblocks) fail(CI_ERR_INVALID_ARG, "nblocks is NULL");
    for (int a = 0; a < p->S; ++a)
        if (sp_orbital[a] < 0) fail(CI_ERR_INVALID_ARG, "sp_orbital[%d] is negative", a);
    enumerate_basis(p, s);
    if (block && p->dim > 0 && !is_device_pointer(block)) fail(CI_ERR_INVALID_ARG, "block must be a device pointer");
    // orbital occupation of every species state: the sorted orbital labels
    // of its particles, numbered in order of first appearance
    std::vector<int32_t> sid[2];
    int64_t nsid[2] = {0, 0};
    for (int q = 0; q < 2; ++q) {
        const SpeciesList &L = p->sp[q];
        std::map<std::vector<int32_t>, int32_t> ids;
        sid[q].resize(L.n);
        std::vector<int32_t> key(L.A);
        for (int64_t i = 0; i < L.n; ++i) {
            for (int t = 0; t < L.A; ++t) key[t] = sp_orbital[L.occ[(size_t)i * L.A + t]];
            std::sort(key.begin(), key.end());
            sid[q][i] = ids.emplace(key, (int32_t)ids.size()).first->second;
        }
        nsid[q] = (int64_t)ids.size();
    }
    std::vector<int32_t> h((size_t)p->dim);
    std::unordered_map<int64_t, int32_t> blk;
    const SpeciesList &P = p->sp[0];
    for (int64_t pi = 0; pi < P.n; ++pi)
        for (int64_t r = p->p_row_base[pi]; r < p->p_row_base[pi + 1]; ++r) {
            const int64_t n = p->p_nstart[pi] + (r - p->p_row_base[pi]);
            const int64_t key = (int64_t)sid[0][pi] * nsid[1] + sid[1][n];
            h[r] = blk.emplace(key, (int32_t)blk.size()).first->second;
        }
    *nblocks = (int64_t)blk.size();
    if (block && p->dim > 0) {
        CI_CUDA(cudaMemcpyAsync(block, h.data(), sizeof(int32_t) * h.size(), cudaMemcpyHostToDevice, s));
        CI_CUDA(cudaStreamSynchronize(s));
    }
}

void precond_setup(BlockPrecond &bp, const Matrix *H, const int32_t *row_block, int64_t nblocks, cudaStream_t s) {
    const int64_t dim = H->dim;
    if (!row_block || !is_device_pointer(row_block)) fail(CI_ERR_INVALID_ARG, "row_block must be a device pointer");
    if (nblocks < 1 || nblocks > dim) fail(CI_ERR_INVALID_ARG, "nblocks must be 1..dim (got %lld)", (long long)nblocks);
    std::vector<int32_t> b((size_t)dim);
    CI_CUDA(cudaMemcpyAsync(b.data(), row_block, sizeof(int32_t) * dim, cudaMemcpyDeviceToHost, s));
    CI_CUDA(cudaStreamSynchronize(s));
    std::vector<int64_t> cnt((size_t)nblocks + 1, 0);
    for (int64_t r = 0; r < dim; ++r) {
        if (b[r] < 0 || b[r] >= nblocks) fail(CI_ERR_INVALID_ARG, "row_block[%lld] = %d outside 0..nblocks-1",
                                              (long long)r, b[r]);
        ++cnt[(size_t)b[r] + 1];
    }
    for (int64_t g = 0; g < nblocks; ++g) cnt[g + 1] += cnt[g];
    std::vector<int32_t> rows((size_t)dim), sub_of((size_t)dim), loc_of((size_t)dim);
    {
        std::vector<int64_t> pos(cnt.begin(), cnt.end() - 1);
        for (int64_t r = 0; r < dim; ++r) rows[pos[b[r]]++] = (int32_t)r;   // members ascending in each block
    }
    std::vector<int64_t> sub_start{0}, inv_off{0};
    int smax = 0;
    for (int64_t g = 0; g < nblocks; ++g) {
        const int64_t c = cnt[g + 1] - cnt[g];
        if (c == 0) continue;
        const int64_t q = (c + kSubMax - 1) / kSubMax;   // sub-blocks; the first c % q get one row more
        int64_t at = cnt[g];
        for (int64_t u = 0; u < q; ++u) {
            const int64_t sz = c / q + (u < c % q ? 1 : 0);
            const int64_t sb = (int64_t)sub_start.size() - 1;
            for (int64_t l = 0; l < sz; ++l) {
                sub_of[rows[at + l]] = (int32_t)sb;
                loc_of[rows[at + l]] = (int32_t)l;
            }
            at += sz;
            sub_start.push_back(at);
            inv_off.push_back(inv_off.back() + sz * sz);
            smax = std::max(smax, (int)sz);
        }
    }
    bp.dim = dim;
    bp.nsub = (int64_t)sub_start.size() - 1;
    bp.smax = smax;
    {
        static const int kBinTop[3] = {32, 64, kSubMax};
        std::vector<int32_t> ids((size_t)bp.nsub);
        for (int64_t u = 0; u < bp.nsub; ++u) ids[u] = (int32_t)u;
        auto size_of = [&](int32_t u) { return sub_start[u + 1] - sub_start[u]; };
        auto bin_of = [&](int32_t u) { return size_of(u) <= kBinTop[0] ? 0 : size_of(u) <= kBinTop[1] ? 1 : 2; };
        std::stable_sort(ids.begin(), ids.end(), [&](int32_t x, int32_t y) {
            const int bx = bin_of(x), by = bin_of(y);
            return bx != by ? bx < by : size_of(x) > size_of(y);
        });
        for (int q = 0; q < 4; ++q) bp.bin_off[q] = 0;
        for (int q = 0; q < 3; ++q) bp.bin_max[q] = 0;
        for (int64_t u = 0; u < bp.nsub; ++u) {
            const int q = bin_of(ids[u]);
            bp.bin_off[q + 1] = u + 1;
            bp.bin_max[q] = std::max(bp.bin_max[q], (int)size_of(ids[u]));
        }
        for (int q = 1; q < 4; ++q) bp.bin_off[q] = std::max(bp.bin_off[q], bp.bin_off[q - 1]);
        bp.bin_ids.upload(ids, s);
    }
    bp.rows.upload(rows, s);
    bp.sub_of.upload(sub_of, s);
    bp.loc_of.upload(loc_of, s);
    bp.sub_start.upload(sub_start, s);
    bp.inv_off.upload(inv_off, s);
    bp.inv.alloc((size_t)inv_off.back());
    bp.shift.alloc((size_t)bp.nsub);
    bp.status.alloc(1);
}

void precond_factor(BlockPrecond &bp, const Matrix *H, double sigma, cudaStream_t s) {
    if (!std::isfinite(sigma)) fail(CI_ERR_INVALID_ARG, "sigma must be finite");
    if (bp.nsub == 0) return;
    CI_CUDA(cudaMemsetAsync(bp.status.ptr, 0, sizeof(int32_t), s));
    auto run = [&](auto kern, const auto *val, const float *rscale) {
        CI_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)inv_smem(kSubMax)));
        for (int q = 0; q < 3; ++q) {
            const int64_t nq = bp.bin_off[q + 1] - bp.bin_off[q];
            if (nq == 0) continue;
            launch("k_block_inv", kern, (unsigned)nq, 256, inv_smem(bp.bin_max[q]), s,
                   (const int64_t *)H->row_ptr.ptr, (const int32_t *)H->col.ptr, val, rscale,
                   (const int32_t *)bp.rows.ptr, (const int64_t *)bp.sub_start.ptr, (const int32_t *)bp.sub_of.ptr,
                   (const int32_t *)bp.loc_of.ptr, (const int64_t *)bp.inv_off.ptr,
                   (const int32_t *)bp.bin_ids.ptr + bp.bin_off[q], H->upper, sigma, bp.inv.ptr, bp.shift.ptr,
                   bp.status.ptr);
        }
    };
    if (H->vtype == CI_F32) run(k_block_inv<float>, (const float *)H->val.ptr, (const float *)nullptr);
    else if (H->vtype == CI_F64) run(k_block_inv<double>, (const double *)H->val.ptr, (const float *)nullptr);
    else if (H->vtype == CI_BF16_ROWSCALE)
        run(k_block_inv<__nv_bfloat16>, (const __nv_bfloat16 *)H->val.ptr, (const float *)H->row_scale.ptr);
    else fail(CI_ERR_INVALID_ARG, "value type %d not supported by the block preconditioner", H->vtype);
    int32_t st = 0;
    CI_CUDA(cudaMemcpyAsync(&st, bp.status.ptr, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CI_CUDA(cudaStreamSynchronize(s));
    if (st) fail(CI_ERR_INTERNAL, "a diagonal block stayed indefinite after the Gershgorin shift");
}

void precond_apply(const BlockPrecond &bp, const double *R, int nv, double *W, cudaStream_t s) {
    if (nv < 1 || nv > 8) fail(CI_ERR_INVALID_ARG, "nvec must be 1..8 (got %d)", nv);
    if (bp.nsub == 0) return;
    const size_t smem = apply_smem(bp.smax, nv);
    CI_CUDA(cudaFuncSetAttribute(k_block_apply, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)apply_smem(kSubMax, 8)));
    launch("k_block_apply", k_block_apply, (unsigned)bp.nsub, 256, smem, s, (const int32_t *)bp.rows.ptr,
           (const int64_t *)bp.sub_start.ptr, (const int64_t *)bp.inv_off.ptr, (const float *)bp.inv.ptr, nv, R, W);
}

void precond_row_shift(const BlockPrecond &bp, double *out, cudaStream_t s) {
    if (bp.dim == 0) return;
    launch("k_row_shift", k_row_shift, grid_for(bp.dim, 256), 256, 0, s, bp.dim, (const int32_t *)bp.sub_of.ptr,
           (const double *)bp.shift.ptr, out);
}

}  // namespace ci

extern "C" ci_status ci_orbital_blocks(ci_problem *p, const int32_t *sp_orbital, int32_t *block, int64_t *nblocks,
                                       void *stream) {
    return ci::guard([&] {
        if (!p) ci::fail(CI_ERR_INVALID_ARG, "problem is NULL");
        cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
        ci::StreamScope scope(s);
        ci::orbital_blocks(&p->impl, sp_orbital, block, nblocks, s);
    });
}

extern "C" ci_status ci_block_precond_apply(const ci_matrix *m, const int32_t *row_block, int64_t nblocks,
                                            double sigma, const double *R, double *W, int32_t nvec,
                                            double *row_shift, void *stream) {
    return ci::guard([&] {
        if (!m) ci::fail(CI_ERR_INVALID_ARG, "matrix is NULL");
        cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
        ci::StreamScope scope(s);
        const ci::Matrix *H = &m->impl;
        if (nvec < 1 || nvec > 8) ci::fail(CI_ERR_INVALID_ARG, "nvec must be 1..8 (got %d)", nvec);
        if (H->dim == 0) return;
        if (!R || !W || !ci::is_device_pointer(R) || !ci::is_device_pointer(W))
            ci::fail(CI_ERR_INVALID_ARG, "R and W must be device pointers");
        if (row_shift && !ci::is_device_pointer(row_shift)) ci::fail(CI_ERR_INVALID_ARG, "row_shift must be a device pointer");
        ci::BlockPrecond bp;
        ci::precond_setup(bp, H, row_block, nblocks, s);
        ci::precond_factor(bp, H, sigma, s);
        ci::precond_apply(bp, R, nvec, W, s);
        if (row_shift) ci::precond_row_shift(bp, row_shift, s);
        CI_CUDA(cudaStreamSynchronize(s));
    });
}
