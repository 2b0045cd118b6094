// Lowest eigenpairs of H (Fig. 1, eigensolve): block Lanczos with full FP64
// reorthogonalisation (classical Gram-Schmidt, repeated), thick restart,
// and a rank-revealing block QR that completes a deflated block with
// random directions.  H is applied by the SpMM in the matrix's precision;
// the Krylov basis, projections, Gram matrices, Ritz vectors and residuals
// are FP64.  The projected matrix T = Q^T H Q is assembled on the host
// from the Gram-Schmidt coefficients and diagonalised there (dense.h).
#include <chrono>
#include <cmath>
#include <memory>

#include <cuda_bf16.h>

#include "dense.h"
#include "problem.cuh"

namespace ci {

// ------------------------------------------------------------------ kernels

constexpr int kTnThreads = 256;   // 8 warps: warp v owns column v of B
constexpr int kMaxNa = 256;       // columns of A in one product

constexpr int kTR = 32;           // rows of A and B staged per tile
constexpr size_t kTnSmem = 96 * 1024;   // shared memory of the tiled product

// part[blk][u][v] = sum over the block's rows i of A[i][u] B[i][v]
// (u < na <= 256, v < nb <= 8).  Tiles of kTR rows of A and B are staged
// in shared memory with coalesced loads; thread t owns outputs t + 256 j.
__global__ void __launch_bounds__(kTnThreads) k_tn_partial(int64_t dim, const double *__restrict__ A, int lda, int na,
                                                           const double *__restrict__ B, int ldb, int nb,
                                                           double *__restrict__ part, int64_t rows_per_blk) {
    pdl_wait();
    extern __shared__ double sm[];
    double *As = sm;             // [kTR][na]
    double *Bs = sm + kTR * na;  // [kTR][nb]
    const int nout = na * nb;
    double acc[kMaxNa * 8 / kTnThreads];
#pragma unroll
    for (int j = 0; j < kMaxNa * 8 / kTnThreads; ++j) acc[j] = 0.0;
    const int64_t r0 = blockIdx.x * rows_per_blk;
    const int64_t r1 = min(dim, r0 + rows_per_blk);
    for (int64_t t0 = r0; t0 < r1; t0 += kTR) {
        const int rows = (int)min((int64_t)kTR, r1 - t0);
#pragma unroll 4
        for (int e = threadIdx.x; e < rows * na; e += kTnThreads) {
            const int r = e / na, u = e - r * na;
            As[e] = A[(t0 + r) * lda + u];
        }
        for (int e = threadIdx.x; e < rows * nb; e += kTnThreads) {
            const int r = e / nb, v = e - r * nb;
            Bs[e] = B[(t0 + r) * ldb + v];
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kMaxNa * 8 / kTnThreads; ++j) {
            const int o = threadIdx.x + j * kTnThreads;
            if (o < nout) {
                const int u = o / nb, v = o - u * nb;
                double s = acc[j];
                for (int r = 0; r < rows; ++r) s = fma(As[r * na + u], Bs[r * nb + v], s);
                acc[j] = s;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < kMaxNa * 8 / kTnThreads; ++j) {
        const int o = threadIdx.x + j * kTnThreads;
        if (o < nout) part[(int64_t)blockIdx.x * nout + o] = acc[j];
    }
}

// Register-tiled form of the same product for the FP64 pipe (2 FMA per
// clock per SM on this part, so the kernel is FMA-bound once every thread
// carries enough independent accumulators and the loads are hidden).
// Thread (g, s) owns the 4 x 8 outputs C[4g..4g+3][0..8) and the rows s,
// s + S, ... of every staged tile (G = nap/4 groups, S = 256 / G row
// slices); each row costs it two 32-byte A loads and four 16-byte B loads
// from shared memory for 32 FMAs.  Tiles of tr rows (the first nap columns
// of A, nap = na rounded up to 4, and the 8 columns of B) are copied into
// two shared buffers with cp.async, the next while the current one is
// used.  The slices are summed through shared memory at the end.
// Requires 16-byte aligned rows (lda, ldb even, A and B 16-byte aligned)
// and nap <= lda.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__global__ void __launch_bounds__(kTnThreads) k_tn_tiled(int64_t dim, const double *__restrict__ A, int lda, int na,
                                                         const double *__restrict__ B, int ldb,
                                                         double *__restrict__ part, int64_t rows_per_blk, int tr) {
    pdl_wait();
    extern __shared__ double sm[];
    const int nap = (na + 3) & ~3;
    const int rowlen = nap + 8;                  // one staged row: A part, then B part
    double *buf[2] = {sm, sm + (size_t)tr * rowlen};
    const int G = nap / 4;
    const int S = kTnThreads / G;
    const int g = threadIdx.x % G, sl = threadIdx.x / G;
    const bool active = sl < S;
    double acc[4][8];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int v = 0; v < 8; ++v) acc[a][v] = 0.0;
    const int64_t r0 = blockIdx.x * rows_per_blk;
    const int64_t r1 = min(dim, r0 + rows_per_blk);
    const int ntiles = (int)((r1 - r0 + tr - 1) / tr);
    const int chunks = rowlen / 2;               // 16-byte pieces per staged row
    auto stage = [&](int tile, double *dst) {
        const int64_t t0 = r0 + (int64_t)tile * tr;
        const int rows = (int)min((int64_t)tr, r1 - t0);
        for (int e = threadIdx.x; e < rows * chunks; e += kTnThreads) {
            const int r = e / chunks, c = e - r * chunks;
            const double *src = 2 * c < nap ? A + (t0 + r) * lda + 2 * c : B + (t0 + r) * ldb + (2 * c - nap);
            cp_async16(dst + (size_t)r * rowlen + 2 * c, src);
        }
        cp_async_commit();
    };
    if (ntiles > 0) stage(0, buf[0]);
    for (int tile = 0; tile < ntiles; ++tile) {
        if (tile + 1 < ntiles) {
            stage(tile + 1, buf[(tile + 1) & 1]);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const double *T = buf[tile & 1];
        const int rows = (int)min((int64_t)tr, r1 - (r0 + (int64_t)tile * tr));
        if (active) {
            for (int r = sl; r < rows; r += S) {
                const double *ar = T + (size_t)r * rowlen;
                const double2 a01 = *reinterpret_cast<const double2 *>(ar + 4 * g);
                const double2 a23 = *reinterpret_cast<const double2 *>(ar + 4 * g + 2);
                const double2 *br = reinterpret_cast<const double2 *>(ar + nap);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const double2 bv = br[q];
                    acc[0][2 * q] = fma(a01.x, bv.x, acc[0][2 * q]);
                    acc[1][2 * q] = fma(a01.y, bv.x, acc[1][2 * q]);
                    acc[2][2 * q] = fma(a23.x, bv.x, acc[2][2 * q]);
                    acc[3][2 * q] = fma(a23.y, bv.x, acc[3][2 * q]);
                    acc[0][2 * q + 1] = fma(a01.x, bv.y, acc[0][2 * q + 1]);
                    acc[1][2 * q + 1] = fma(a01.y, bv.y, acc[1][2 * q + 1]);
                    acc[2][2 * q + 1] = fma(a23.x, bv.y, acc[2][2 * q + 1]);
                    acc[3][2 * q + 1] = fma(a23.y, bv.y, acc[3][2 * q + 1]);
                }
            }
        }
        __syncthreads();   // the buffer is refilled two tiles later
    }
    // sum the S row slices: red[sl][4g + a][v]
    double *red = sm;
    const int nout = nap * 8;
    if (active) {
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int v = 0; v < 8; ++v) red[(size_t)sl * nout + (4 * g + a) * 8 + v] = acc[a][v];
    }
    __syncthreads();
    for (int o = threadIdx.x; o < na * 8; o += kTnThreads) {
        double t = 0.0;
        for (int q = 0; q < S; ++q) t += red[(size_t)q * nout + o];
        part[(int64_t)blockIdx.x * na * 8 + o] = t;
    }
}

// W[i][v] = beta W[i][v] + alpha sum_u A[i][u] C[u][v] with one row per
// thread and NB accumulators: each A element is loaded once for NB FMAs,
// C is a shared-memory broadcast.
template <int NB>
__global__ void __launch_bounds__(256) k_nn_rows(int64_t dim, const double *__restrict__ A, int lda, int na,
                                                 const double *__restrict__ C, double *__restrict__ W, int ldw,
                                                 double alpha, double beta) {
    pdl_wait();
    __shared__ double Cs[kMaxNa * NB];
    for (int e = threadIdx.x; e < na * NB; e += blockDim.x) Cs[e] = C[e];
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < dim; i += (int64_t)gridDim.x * blockDim.x) {
        const double *Ai = A + i * lda;
        double acc[NB];
#pragma unroll
        for (int v = 0; v < NB; ++v) acc[v] = 0.0;
        for (int u = 0; u < na; ++u) {
            const double a = Ai[u];
            const double *cu = Cs + u * NB;
#pragma unroll
            for (int v = 0; v < NB; ++v) acc[v] = fma(a, cu[v], acc[v]);
        }
        double *w = W + i * ldw;
#pragma unroll
        for (int v = 0; v < NB; ++v) w[v] = beta == 0.0 ? alpha * acc[v] : fma(beta, w[v], alpha * acc[v]);
    }
}

// out[o] = sum_blk part[blk][o]: one warp per output, lane l sums blocks
// l, l + 32, ... in order, then a fixed butterfly adds the 32 lane sums
// (deterministic).
__global__ void __launch_bounds__(256) k_reduce_partial(const double *__restrict__ part, int nblk, int n,
                                                        double *__restrict__ out) {
    pdl_wait();
    const int lane = threadIdx.x & 31;
    const int o = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (o >= n) return;
    double s = 0.0;
#pragma unroll 4
    for (int b = lane; b < nblk; b += 32) s += part[(int64_t)b * n + o];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
    if (lane == 0) out[o] = s;
}

// W[i][v] = beta W[i][v] + alpha sum_u A[i][u] C[u][v]   (beta == 0: W not read)
__global__ void __launch_bounds__(256) k_nn_update(int64_t dim, const double *__restrict__ A, int lda, int na,
                                                   const double *__restrict__ C, int nb, double *__restrict__ W,
                                                   int ldw, double alpha, double beta) {
    pdl_wait();
    __shared__ double Cs[kMaxNa * 8];
    for (int e = threadIdx.x; e < na * nb; e += blockDim.x) Cs[e] = C[e];
    __syncthreads();
    const int64_t total = dim * nb;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / nb;
        const int v = (int)(t % nb);
        const double *Ai = A + i * lda;
        double s = 0.0;
        for (int u = 0; u < na; ++u) s = fma(Ai[u], Cs[u * nb + v], s);
        double *w = W + i * ldw + v;
        *w = beta == 0.0 ? alpha * s : fma(beta, *w, alpha * s);
    }
}

__global__ void k_cvt_to_f32(int64_t dim, int nb, const double *__restrict__ src, int lds, float *__restrict__ dst) {
    pdl_wait();
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < dim * nb; t += (int64_t)gridDim.x * blockDim.x)
        dst[t] = (float)src[(t / nb) * lds + t % nb];
}

__global__ void k_cvt_to_f64(int64_t dim, int nb, const float *__restrict__ src, double *__restrict__ dst, int ldd) {
    pdl_wait();
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < dim * nb; t += (int64_t)gridDim.x * blockDim.x)
        dst[(t / nb) * ldd + t % nb] = (double)src[t];
}

// X16[i][0..8) = V1[i][0..8), X16[i][8..16) = V2[i][0..8) in FP32
__global__ void k_pack16(int64_t dim, const double *__restrict__ V1, int ld1, const double *__restrict__ V2, int ld2,
                         float *__restrict__ X16) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < dim * 16; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t >> 4;
        const int c = (int)(t & 15);
        X16[t] = (float)(c < 8 ? V1[i * ld1 + c] : V2[i * ld2 + c - 8]);
    }
}

// W1[i][0..8) = Y16[i][0..8), W2[i][0..8) = Y16[i][8..16) in FP64 (ld 8)
__global__ void k_unpack16(int64_t dim, const float *__restrict__ Y16, double *__restrict__ W1, double *__restrict__ W2) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < dim * 16; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t >> 4;
        const int c = (int)(t & 15);
        if (c < 8) W1[i * 8 + c] = Y16[t];
        else W2[i * 8 + c - 8] = Y16[t];
    }
}

__global__ void k_copy_cols(int64_t dim, int nb, const double *__restrict__ src, int lds, double *__restrict__ dst,
                            int ldd) {
    pdl_wait();
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < dim * nb; t += (int64_t)gridDim.x * blockDim.x)
        dst[(t / nb) * ldd + t % nb] = src[(t / nb) * lds + t % nb];
}

// y += x over n doubles
__global__ void k_axpy(int64_t n, const double *__restrict__ x, double *__restrict__ y) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        y[t] += x[t];
}

__global__ void k_zero_cols(int64_t dim, int nb, double *dst, int ldd) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < dim * nb; t += (int64_t)gridDim.x * blockDim.x)
        dst[(t / nb) * ldd + t % nb] = 0.0;
}

// First block-QR pass on the device (Cholesky QR): the Gram matrix G = W^T W
// (b x b, b <= 8) of a block that is already orthogonal to the basis is
// factored as G = L L^T; then W M with M = L^{-T} has orthonormal columns up
// to the conditioning of G, and W = (W M) R with R = L^T.  One thread per
// entry: column c of the right-looking factorisation, then thread c solves
// L x = e_c for column c of L^{-1}.  *stat = 1 (else 0) when a pivot is not
// above 1e-12 of the largest diagonal entry, nor above 1e-20 max(hnorm^2,
// that entry) (the host path's deflation level), or is not finite: the
// block is then left to the rank-revealing host path.
__global__ void k_qr1(const double *__restrict__ G, int b, double hnorm, double *__restrict__ M,
                      double *__restrict__ R, int *stat) {
    pdl_wait();
    __shared__ double A[64], Li[64], rd[8];
    __shared__ int bad;
    const int t = threadIdx.x, i = t / b, j = t % b;
    const bool on = t < b * b;
    if (on) A[t] = 0.5 * (G[i * b + j] + G[j * b + i]);
    if (t == 0) bad = 0;
    __syncthreads();
    double gmax = 0.0;
    for (int q = 0; q < b; ++q) gmax = fmax(gmax, A[q * b + q]);
    const double thr = fmax(1e-12 * gmax, 1e-20 * fmax(hnorm * hnorm, gmax)) + 1e-300;
    for (int c = 0; c < b; ++c) {
        double d = A[c * b + c];   // Schur complement pivot
        const bool ok = d > thr && d < 1e300;
        if (!ok) d = 1.0;          // any finite pivot: the result is not used
        const double l = sqrt(d), il = 1.0 / l;
        double lic = 0.0, ljc = 0.0;
        if (on && i > c && j > c) {
            lic = A[i * b + c] * il;
            ljc = A[j * b + c] * il;
        }
        __syncthreads();           // column c read by everyone
        if (t == 0) {
            rd[c] = il;
            if (!ok) bad = 1;
        }
        if (on && i > c && j > c) A[t] -= lic * ljc;
        if (on && j == c && i >= c) A[t] = i == c ? l : A[t] * il;
        __syncthreads();
    }
    if (t < b) {   // column t of L^{-1}
        for (int r = 0; r < b; ++r) {
            double x = r == t ? 1.0 : 0.0;
            for (int k = t; k < r; ++k) x -= A[r * b + k] * Li[k * b + t];
            Li[r * b + t] = r < t ? 0.0 : x * rd[r];
        }
    }
    __syncthreads();
    if (on) {
        M[i * b + j] = Li[j * b + i];                  // M = L^{-T}
        R[i * b + j] = j >= i ? A[j * b + i] : 0.0;    // R = L^T
    }
    if (t == 0) *stat = bad;
}

// Second block-QR pass on the device.  G (b x b) is the Gram matrix of a
// block whose columns are orthogonal up to rounding (completion columns may
// have any length); with D = diag(G)^{-1/2} and G' = D G D (unit diagonal),
// the coupled Newton-Schulz iteration Y <- Y T, Z <- T Z, T = (3I - Z Y)/2
// from Y = G', Z = I converges quadratically to Y = G'^{1/2}, Z = G'^{-1/2}
// (the eigenvalues of G' lie in (0, 3) here).  Then V Mi with Mi = D Z is
// orthonormal, and the block's coupling becomes R2 = Y D^{-1} R.  One thread
// per entry (b*b <= 64); the iteration stops after the update made with
// |I - Z Y| <= 1e-12, whose error is of second order; *flag |= fail when 40
// iterations leave T off the identity or a column has no length.  skip
// (nullable): set to 1 when every entry of G is within kOrthSkip of the
// identity's (V orthonormal already: Mi = I, R2 = R, and the caller skips
// the product V Mi and the copy, leaving the block, its shadow and its FP32
// copy as the first pass made them), else to 0.
constexpr double kOrthSkip = 1e-13;
__global__ void k_qr2(const double *__restrict__ G, int b, double *__restrict__ Mi, const double *__restrict__ R,
                      double *__restrict__ R2, int *flag, int fail, int *skip) {
    pdl_wait();
    __shared__ double Y[64], Z[64], Tm[64], d[8];
    const int t = threadIdx.x, i = t / b, j = t % b;
    const bool on = t < b * b;
    if (skip) {
        const double e = on ? fabs(0.5 * (G[i * b + j] + G[j * b + i]) - (i == j ? 1.0 : 0.0)) : 0.0;
        const bool far = __syncthreads_or(on && !(e <= kOrthSkip));
        if (!far) {
            if (on) {
                Mi[t] = i == j ? 1.0 : 0.0;
                R2[t] = R[t];
            }
            if (t == 0) *skip = 1;
            return;
        }
        if (t == 0) *skip = 0;
    }
    if (t < b) {
        const double g = G[t * b + t];
        d[t] = g > 0.0 ? 1.0 / sqrt(g) : 1.0;
        if (!(g > 0.0)) atomicOr(flag, fail);
    }
    __syncthreads();
    if (on) {
        Y[t] = d[i] * (0.5 * (G[i * b + j] + G[j * b + i])) * d[j];
        Z[t] = i == j ? 1.0 : 0.0;
    }
    bool conv = false;
    for (int it = 0; it < 40 && !conv; ++it) {
        __syncthreads();
        double dev = 0.0;
        if (on) {
            double zy = 0.0;
            for (int k = 0; k < b; ++k) zy = fma(Z[i * b + k], Y[k * b + j], zy);
            const double e = (i == j ? 1.0 : 0.0) - zy;   // T = I + E/2, E = I - Z Y
            Tm[t] = (i == j ? 1.0 : 0.0) + 0.5 * e;
            dev = fabs(e);
        }
        __syncthreads();
        double yn = 0.0, zn = 0.0;
        if (on) {
            for (int k = 0; k < b; ++k) {
                yn = fma(Y[i * b + k], Tm[k * b + j], yn);
                zn = fma(Tm[i * b + k], Z[k * b + j], zn);
            }
        }
        conv = !__syncthreads_or(dev > 1e-12);   // this last update leaves O(dev^2): rounding level
        if (on) {
            Y[t] = yn;
            Z[t] = zn;
        }
    }
    __syncthreads();
    if (!conv && t == 0) atomicOr(flag, fail);
    if (on) {
        Mi[t] = d[i] * Z[t];
        double x = 0.0;
        for (int k = 0; k < b; ++k) x = fma(Y[i * b + k], R[k * b + j] / d[k], x);
        R2[t] = x;
    }
}

// Uniform(-1, 1) entries from SplitMix64 at position (i*nb + v) of stream seed.
__global__ void k_random_cols(int64_t dim, int nb, uint64_t seed, double *dst, int ldd) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < dim * nb; t += (int64_t)gridDim.x * blockDim.x) {
        uint64_t z = seed + (uint64_t)(t + 1) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        dst[(t / nb) * ldd + t % nb] = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
    }
}

// R = HX - X diag(theta): R[i][v] = HX[i][v] - theta[v] X[i][v]
template <class TX>
__global__ void k_residual(int64_t dim, int nb, const TX *__restrict__ HX, const double *__restrict__ X, int ldx,
                           const double *__restrict__ theta, double *__restrict__ R) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < dim * nb; t += (int64_t)gridDim.x * blockDim.x) {
        const int v = (int)(t % nb);
        R[t] = (double)HX[t] - theta[v] * X[(t / nb) * ldx + v];
    }
}

__device__ __forceinline__ double as_double(float v) { return v; }
__device__ __forceinline__ double as_double(double v) { return v; }
__device__ __forceinline__ double as_double(__nv_bfloat16 v) { return __bfloat162float(v); }

// d[i] = H[i][i] (0 if the row has no diagonal entry): binary search of
// the ascending columns of row i; BF16 values times the row's scale.
template <class TV>
__global__ void k_diag(int64_t dim, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                       const TV *__restrict__ val, const float *__restrict__ row_scale, double *__restrict__ d) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < dim; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = rp[i], hi = rp[i + 1];
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (col[mid] < i) lo = mid + 1; else hi = mid;
        }
        const double v = (lo < rp[i + 1] && col[lo] == i) ? as_double(val[lo]) : 0.0;
        d[i] = row_scale ? v * row_scale[i] : v;
    }
}

// Diagonal (Jacobi) preconditioner of LOBPCG: W[i][v] = R[i][v] / (d_i - theta_v),
// with the shift kept at least floor * |theta_v| (sign preserved) away from 0.
__global__ void k_precond(int64_t dim, int nb, const double *__restrict__ R, const double *__restrict__ d,
                          const double *__restrict__ theta, double floor, double *__restrict__ W) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < dim * nb; t += (int64_t)gridDim.x * blockDim.x) {
        const int v = (int)(t % nb);
        double den = d[t / nb] - theta[v];
        const double lim = floor * fmax(fabs(theta[v]), 1.0);
        if (fabs(den) < lim) den = den < 0 ? -lim : lim;
        W[t] = R[t] / den;
    }
}

// ------------------------------------------------------------------ FP64 products

static void set_tn_attributes() {
    static bool attr = false;
    if (!attr) {
        CI_CUDA(cudaFuncSetAttribute(k_tn_partial, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(sizeof(double) * kTR * (kMaxNa + 8))));
        CI_CUDA(cudaFuncSetAttribute(k_tn_tiled, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)std::max(kTnSmem, sizeof(double) * kTnThreads * 8 * 4)));
        attr = true;
    }
}

// part[blk][na][nb] = A^T B over row blocks of rows_per_blk rows, on the
// FP64 CUDA cores.
static void fp64_tn(int64_t dim, const double *A, int lda, int na, const double *B, int ldb, int nb, double *part,
                    int nblk, int64_t rows_per_blk, cudaStream_t s) {
    set_tn_attributes();
    const int nap = (na + 3) & ~3;
    const bool aligned = ((uintptr_t)A % 16 == 0) && ((uintptr_t)B % 16 == 0) && lda % 2 == 0 && ldb % 2 == 0 &&
                         nap <= lda;
    if (nb == 8 && aligned) {
        // two staged tiles, later reused for the slice sums, in at most
        // kTnSmem bytes
        const int S = kTnThreads / (nap / 4);
        int tr = (int)(kTnSmem / sizeof(double)) / (2 * (nap + 8));
        if (tr > 128) tr = 128;
        const size_t smem = sizeof(double) * std::max((size_t)2 * tr * (nap + 8), (size_t)S * nap * 8);
        launch_pdl("k_tn_partial", k_tn_tiled, nblk, kTnThreads, smem, s, dim, A, lda, na, B, ldb, part,
               rows_per_blk, tr);
    } else {
        const size_t smem = sizeof(double) * kTR * (na + nb);
        launch_pdl("k_tn_partial", k_tn_partial, nblk, kTnThreads, smem, s, dim, A, lda, na, B, ldb, nb, part,
               rows_per_blk);
    }
}

// W = beta W + alpha A C on the FP64 CUDA cores.
static void fp64_nn(int64_t dim, const double *A, int lda, int na, const double *C, int nb, double *Wout, int ldw,
                    double alpha, double beta, cudaStream_t s) {
    const int grid = nb == 8 ? grid_for(dim, 256, sm_count() * 8) : grid_for(dim * nb, 256, sm_count() * 8);
    if (nb == 8)
        launch_pdl("k_nn_update", k_nn_rows<8>, grid, 256, 0, s, dim, A, lda, na, C, Wout, ldw, alpha, beta);
    else
        launch_pdl("k_nn_update", k_nn_update, grid, 256, 0, s, dim, A, lda, na, C, nb, Wout, ldw, alpha, beta);
    CI_CHECK_LAUNCH();
}

// ------------------------------------------------------------------ driver

namespace {

struct Solver {
    const Matrix *H;
    cudaStream_t s;
    int64_t dim;
    int b, k, mmax;
    bool f64;
    int nblk;
    // basis products on the tensor cores (FP64-exact digit planes) unless
    // the caller asked for the FP64 CUDA-core kernels
    bool tc = true;
    int oz_nblk = 1;
    DevBuf<int> ozflag;
    DevBuf<unsigned long long> Qfix;   // fixed-point shadow of Q for the tensor-core products
    int64_t rows_per_blk;
    DevBuf<double> Q, W, W2, tmp, part, Cdev, Mdev, theta_dev, Cacc;
    DevBuf<float> X32, Y32;
    int x32_col = -1;   // X32 holds Q[:, x32_col : x32_col + b] in FP32 (else -1)
    DevBuf<double> X64;
    double hnorm = 0.0;
    // pinned copy of the projection coefficients of the latest step, read
    // after the next host sync instead of a sync of its own
    double *pin_coef = nullptr;
    size_t pin_len = 0;
    cudaEvent_t ev_coef = nullptr;   // after their copy
    // the block QR's coupling R of the last two block steps: computed on the
    // device by the second pass, copied to pinned memory with the device
    // pass's status, read by take_R
    DevBuf<double> Rdev, R2dev;
    DevBuf<int> qstat, qskip;
    double *pin_R = nullptr;   // [2][64]
    int *pin_stat = nullptr;   // [2][2]: status, second-pass product skipped
    int last_skip = 0;
    cudaEvent_t ev_R[2] = {nullptr, nullptr};
    int pend_m = 0, pend_lo = 0, pend_nb = 0, pend_passes = 0;
    bool pend = false;

    Solver(const Matrix *H_, cudaStream_t s_, int b_, int k_, int mmax_)
        : H(H_), s(s_), dim(H_->dim), b(b_), k(k_), mmax(mmax_), f64(H_->vtype == CI_F64) {
        int sms = sm_count();
        nblk = (int)std::min<int64_t>((int64_t)sms * 2, (dim + 63) / 64);
        if (nblk < 1) nblk = 1;
        rows_per_blk = (dim + nblk - 1) / nblk;
        oz_nblk = oz_tn_blocks(dim);
        Q.alloc((size_t)dim * mmax);
        W.alloc((size_t)dim * b);
        tmp.alloc((size_t)dim * std::max(mmax, b));
        part.alloc((size_t)std::max(nblk, oz_nblk) * kMaxNa * 8);
        ozflag.alloc(1);
        CI_CUDA(cudaMemsetAsync(ozflag.ptr, 0, sizeof(int), s));
        if (b == 8) Qfix.alloc((size_t)dim * mmax);
        Cdev.alloc((size_t)kMaxNa * 8);
        Mdev.alloc((size_t)kMaxNa * 8);
        theta_dev.alloc(64);
        if (f64) X64.alloc((size_t)dim * b);
        else { X32.alloc((size_t)dim * b); Y32.alloc((size_t)dim * b); }
    }

    ~Solver() {
        if (pin_R) {
            cudaStreamSynchronize(s);
            cudaFreeHost(pin_R);
            cudaFreeHost(pin_stat);
        }
        for (cudaEvent_t &e : ev_R)
            if (e) cudaEventDestroy(e);
        if (ev_coef) cudaEventDestroy(ev_coef);
        if (pin_coef) {
            cudaStreamSynchronize(s);
            cudaFreeHost(pin_coef);
        }
    }
    Solver(const Solver &) = delete;
    Solver &operator=(const Solver &) = delete;

    int grid(int64_t work) const { return grid_for(work, 256, sm_count() * 8); }

    // C (na x nb) = A^T B over all rows; result in Cout (device) and, if
    // host != null, copied to host.  basis: A holds orthonormal basis
    // columns (|A| <= 1), which the tensor-core product takes.
    bool use_tc(bool basis, int na, int nb) const { return basis && tc && nb == 8 && Qfix.ptr && oz_supported(na); }
    // the shadow of the basis column that A points at
    const unsigned long long *shadow(const double *A) const { return Qfix.ptr + (A - Q.ptr); }
    // Q[:, c0:c0+nc] = src (leading dimension lds), with the shadow
    // (an entry out of the shadow's range sets bit 0 of *flag, ozflag by
    // default).  x32: nullable, also receives the columns in FP32 (the next
    // SpMM's input; x32_col records which block it holds).  skip: nullable
    // device flag, when set nothing is copied (the columns, shadow and FP32
    // copy are already in place).
    void copy_into_basis(const double *src, int lds, int c0, int nc, int *flag = nullptr, float *x32 = nullptr,
                         const int *skip = nullptr) {
        x32_col = -1;
        if (tc && Qfix.ptr) {
            oz_copy_fix(dim, nc, src, lds, Q.ptr + c0, mmax, Qfix.ptr + c0, mmax, x32, flag ? flag : ozflag.ptr, s,
                        skip);
            if (x32) x32_col = c0;
        } else {
            launch_pdl("k_copy_cols", k_copy_cols, grid(dim * nc), 256, 0, s, dim, nc, src, lds, Q.ptr + c0, mmax);
        }
        CI_CHECK_LAUNCH();
    }

    void tn(const double *A, int lda, int na, const double *B, int ldb, int nb, double *Cout,
            std::vector<double> *host, bool basis = false) {
        if (use_tc(basis, na, nb)) {
            oz_tn(dim, shadow(A), lda, na, B, ldb, part.ptr, oz_nblk, ozflag.ptr, s);
            launch_pdl("k_reduce_partial", k_reduce_partial, (na * nb + 7) / 8, 256, 0, s, part.ptr, oz_nblk, na * nb,
                   Cout);
            CI_CHECK_LAUNCH();
            if (host) {
                host->resize((size_t)na * nb);
                CI_CUDA(cudaMemcpyAsync(host->data(), Cout, sizeof(double) * na * nb, cudaMemcpyDeviceToHost, s));
                CI_CUDA(cudaStreamSynchronize(s));
            }
            return;
        }
        fp64_tn(dim, A, lda, na, B, ldb, nb, part.ptr, nblk, rows_per_blk, s);
        launch_pdl("k_reduce_partial", k_reduce_partial, (na * nb + 7) / 8, 256, 0, s, part.ptr, nblk, na * nb, Cout);
        CI_CHECK_LAUNCH();
        if (host) {
            host->resize((size_t)na * nb);
            CI_CUDA(cudaMemcpyAsync(host->data(), Cout, sizeof(double) * na * nb, cudaMemcpyDeviceToHost, s));
            CI_CUDA(cudaStreamSynchronize(s));
        }
    }

    // skip: nullable device flag that cancels the (tensor-core) product
    void nn(const double *A, int lda, int na, const double *C, int nb, double *Wout, int ldw, double alpha,
            double beta, bool basis = false, const int *skip = nullptr) {
        if (use_tc(basis, na, nb)) {
            oz_nn(dim, shadow(A), lda, na, C, Wout, ldw, alpha, beta, ozflag.ptr, s, skip);
            CI_CHECK_LAUNCH();
            return;
        }
        fp64_nn(dim, A, lda, na, C, nb, Wout, ldw, alpha, beta, s);
    }

    void upload(const std::vector<double> &h, double *d) {
        CI_CUDA(cudaMemcpyAsync(d, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice, s));
    }

    // Wout [dim][nb] (contiguous) = H V, V with leading dimension ldv.
    void apply(const double *V, int ldv, int nb, double *Wout) {
        if (f64) {
            launch_pdl("k_copy_cols", k_copy_cols, grid(dim * nb), 256, 0, s, dim, nb, V, ldv, X64.ptr, nb);
            apply_matrix(H, X64.ptr, Wout, nb, s);
        } else {
            // a block just written by the second pass comes with its FP32 copy
            if (!(nb == b && ldv == mmax && x32_col >= 0 && V == Q.ptr + x32_col))
                launch_pdl("k_cvt_to_f32", k_cvt_to_f32, grid(dim * nb), 256, 0, s, dim, nb, V, ldv, X32.ptr);
            x32_col = -1;
            if (!(nb == 8 && apply_matrix8_f64out(H, X32.ptr, Wout, s))) {
                apply_matrix(H, X32.ptr, Y32.ptr, nb, s);
                launch_pdl("k_cvt_to_f64", k_cvt_to_f64, grid(dim * nb), 256, 0, s, dim, nb, Y32.ptr, Wout, nb);
            }
        }
        CI_CHECK_LAUNCH();
    }

    // W1 = H V1 and W2 = H V2 (8 vectors each, outputs ld 8): one 16-vector
    // product for an FP32 or BF16 H, else two 8-vector ones
    DevBuf<float> X16, Y16;
    void apply2(const double *V1, int ld1, const double *V2, int ld2, double *W1, double *W2) {
        if (f64 || b != 8 || H->upper) {
            apply(V1, ld1, 8, W1);
            apply(V2, ld2, 8, W2);
            return;
        }
        X16.ensure((size_t)dim * 16);
        Y16.ensure((size_t)dim * 16);
        launch("k_pack16", k_pack16, grid(dim * 16), 256, 0, s, dim, V1, ld1, V2, ld2, X16.ptr);
        apply_matrix16(H, X16.ptr, Y16.ptr, s);
        launch("k_unpack16", k_unpack16, grid(dim * 16), 256, 0, s, dim, (const float *)Y16.ptr, W1, W2);
        CI_CHECK_LAUNCH();
    }

    // Project the block Wb [dim][nb] (ld nb) against Q[:, 0:m], `passes`
    // times; returns the summed coefficients (m x nb, host).
    // Orthogonalise Wb [dim][nb] (ld nb) against Q[:, 0:m]: first against
    // the columns [lo, m) (the newest blocks, which carry the large
    // three-term components), then `passes` full classical Gram-Schmidt
    // passes against all m columns.  coef (m x nb, host) receives the sum
    // of all projection coefficients, i.e. Q^T (H V_j).  One host sync.
    void project(double *Wb, int nb, int m, int lo, int passes, std::vector<double> *coef) {
        if (coef) coef->assign((size_t)m * nb, 0.0);
        if (m == 0) return;
        const int nl = m - lo;
        Cacc.ensure((size_t)(passes + 1) * kMaxNa * 8);
        double *cl = Cacc.ptr;
        if (nl > 0) {
            tn(Q.ptr + lo, mmax, nl, Wb, nb, nb, cl, nullptr, true);
            nn(Q.ptr + lo, mmax, nl, cl, nb, Wb, nb, -1.0, 1.0, true);
        }
        for (int p = 0; p < passes; ++p) {
            double *cp = Cacc.ptr + (size_t)(p + 1) * kMaxNa * 8;
            tn(Q.ptr, mmax, m, Wb, nb, nb, cp, nullptr, true);
            nn(Q.ptr, mmax, m, cp, nb, Wb, nb, -1.0, 1.0, true);
        }
        if (!coef) return;
        std::vector<double> h((size_t)(passes + 1) * kMaxNa * 8);
        CI_CUDA(cudaMemcpyAsync(h.data(), Cacc.ptr, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s));
        CI_CUDA(cudaStreamSynchronize(s));
        fold_coef(h.data(), nb, m, lo, passes, coef);
    }

    // coef (m x nb) = the summed coefficients held in h (layout of Cacc)
    static void fold_coef(const double *h, int nb, int m, int lo, int passes, std::vector<double> *coef) {
        coef->assign((size_t)m * nb, 0.0);
        for (int i = 0; i < m - lo; ++i)
            for (int v = 0; v < nb; ++v) (*coef)[(size_t)(lo + i) * nb + v] += h[(size_t)i * nb + v];
        for (int p = 0; p < passes; ++p)
            for (size_t e = 0; e < (size_t)m * nb; ++e) (*coef)[e] += h[(size_t)(p + 1) * kMaxNa * 8 + e];
    }

    // project() whose coefficients are copied to pinned memory without a
    // sync; take_coef() reads them once the copy's event has passed.
    void project_deferred(double *Wb, int nb, int m, int lo, int passes) {
        project(Wb, nb, m, lo, passes, nullptr);
        if (m == 0) return;
        const size_t len = (size_t)(passes + 1) * kMaxNa * 8;
        if (pin_len < len) {
            if (pin_coef) {
                CI_CUDA(cudaStreamSynchronize(s));
                cudaFreeHost(pin_coef);
                pin_coef = nullptr;
            }
            CI_CUDA(cudaMallocHost(&pin_coef, sizeof(double) * len));
            pin_len = len;
        }
        CI_CUDA(cudaMemcpyAsync(pin_coef, Cacc.ptr, sizeof(double) * len, cudaMemcpyDeviceToHost, s));
        if (!ev_coef) CI_CUDA(cudaEventCreateWithFlags(&ev_coef, cudaEventDisableTiming));
        CI_CUDA(cudaEventRecord(ev_coef, s));
        pend = true;
        pend_m = m; pend_lo = lo; pend_nb = nb; pend_passes = passes;
    }
    void take_coef(std::vector<double> *coef) {
        if (!pend) { coef->assign((size_t)pend_m * pend_nb, 0.0); return; }
        CI_CUDA(cudaEventSynchronize(ev_coef));
        fold_coef(pin_coef, pend_nb, pend_m, pend_lo, pend_passes, coef);
        pend = false;
    }

    void ensure_qr_buffers() {
        if (pin_R) return;
        CI_CUDA(cudaMallocHost(&pin_R, sizeof(double) * 2 * 64));
        CI_CUDA(cudaMallocHost(&pin_stat, sizeof(int) * 4));
        for (cudaEvent_t &e : ev_R) CI_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        Rdev.alloc(64);
        R2dev.alloc(64);
        qstat.alloc(1);
        qskip.alloc(1);
        CI_CUDA(cudaMemsetAsync(qskip.ptr, 0, sizeof(int), s));
    }

    // Orthonormalise Wb [dim][b] (already orthogonal to Q[:, 0:m]) into
    // Q[:, m:m+b] on the host path.  R (b x b, row-major) receives the
    // coupling Wb = V R.  Directions below the deflation threshold are
    // replaced by random vectors orthogonal to Q and V (their coupling is
    // zero).  The first pass synchronises on the Gram matrix of Wb (its
    // eigenvalues decide the deflation); the second pass runs on the device
    // (k_qr2) and leaves its R in pinned slot `par`, read by take_R(par)
    // after event ev_R[par].
    void block_qr(double *Wb, int m, uint64_t seed, int par) {
        std::vector<double> G, w, U, R;
        tn(Wb, b, b, Wb, b, b, Cdev.ptr, &G);
        sym_eig(b, G, w, U);
        const double lmax = std::max(w[b - 1], 0.0);
        const double scale = std::max(hnorm, std::sqrt(lmax));
        const double thr = 1e-20 * scale * scale + 1e-300;
        std::vector<double> M((size_t)b * b, 0.0);
        R.assign((size_t)b * b, 0.0);
        int r = 0;
        for (int i = b - 1; i >= 0; --i) {  // largest first
            if (w[i] <= thr) break;
            double sq = std::sqrt(w[i]);
            for (int a = 0; a < b; ++a) {
                M[(size_t)a * b + r] = U[(size_t)a * b + i] / sq;
                R[(size_t)r * b + a] = U[(size_t)a * b + i] * sq;
            }
            ++r;
        }
        double *V = Q.ptr + m;
        ensure_qr_buffers();
        upload(M, Mdev.ptr);
        upload(R, Rdev.ptr);
        nn(Wb, b, b, Mdev.ptr, b, V, mmax, 1.0, 0.0);
        if (r < b) {
            // random completion of columns r..b-1
            double *Vr = tmp.ptr;
            int nr = b - r;
            launch("k_random_cols", k_random_cols, grid(dim * nr), 256, 0, s, dim, nr, seed, Vr, nr);
            CI_CHECK_LAUNCH();
            for (int pass = 0; pass < 2; ++pass) {
                if (m > 0) {
                    tn(Q.ptr, mmax, m, Vr, nr, nr, Cdev.ptr, nullptr);
                    nn(Q.ptr, mmax, m, Cdev.ptr, nr, Vr, nr, -1.0, 1.0);
                }
                if (r > 0) {
                    tn(V, mmax, r, Vr, nr, nr, Cdev.ptr, nullptr);
                    nn(V, mmax, r, Cdev.ptr, nr, Vr, nr, -1.0, 1.0);
                }
            }
            launch_pdl("k_copy_cols", k_copy_cols, grid(dim * nr), 256, 0, s, dim, nr, Vr, nr, V + r, mmax);
            CI_CHECK_LAUNCH();
        }
        CI_CUDA(cudaMemsetAsync(qstat.ptr, 0, sizeof(int), s));
        second_pass(m, par, ozflag.ptr, 4);
    }

    // Second pass of either path: V = Q[:, m:m+b] <- V G2^{-1/2} and
    // R2 = G2^{1/2} R (Rdev), with G2 the Gram matrix of V (k_qr2; a failure
    // sets `fail` in *flag, and so does bit 0 for an entry of V out of the
    // shadow's range).  V is orthonormal up to rounding or the conditioning
    // of the first pass, so its products go through the basis path.  R2 and
    // the status word go to pinned slot par, then ev_R[par].
    // On the tensor-core path a block that the first pass left orthonormal to
    // kOrthSkip skips the product V G2^{-1/2} (k_qr2 decides on the device).
    void second_pass(int m, int par, int *flag, int fail) {
        double *V = Q.ptr + m;
        const bool vtc = tc && Qfix.ptr;
        int *sk = vtc ? qskip.ptr : nullptr;
        float *x32 = f64 ? nullptr : X32.ptr;
        // the shadow (and FP32 copy) of the first pass's block: final when
        // the product below is skipped, else rewritten by the copy
        if (vtc) oz_fix(dim, b, V, mmax, Qfix.ptr + m, mmax, flag, s, x32);
        tn(V, mmax, b, V, mmax, b, Cdev.ptr, nullptr, vtc);
        launch_pdl("k_qr2", k_qr2, 1, 64, 0, s, Cdev.ptr, b, Mdev.ptr, Rdev.ptr, R2dev.ptr, flag, fail, sk);
        nn(V, mmax, b, Mdev.ptr, b, tmp.ptr, b, 1.0, 0.0, vtc, sk);
        copy_into_basis(tmp.ptr, b, m, b, flag, x32, sk);
        CI_CUDA(cudaMemcpyAsync(pin_R + 64 * par, R2dev.ptr, sizeof(double) * b * b, cudaMemcpyDeviceToHost, s));
        CI_CUDA(cudaMemcpyAsync(pin_stat + 2 * par, qstat.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
        CI_CUDA(cudaMemcpyAsync(pin_stat + 2 * par + 1, qskip.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
        CI_CUDA(cudaEventRecord(ev_R[par], s));
    }

    // The same on the device without a host sync: G = Wb^T Wb, Cholesky
    // first pass (k_qr1), V = Wb M, then the second pass.  A block that is
    // numerically rank deficient, or whose second pass does not settle, is
    // reported in its status word (take_R): the caller then redoes it with
    // block_qr from the same Wb.
    void block_qr_dev(const double *Wb, int m, int par) {
        ensure_qr_buffers();
        tn(Wb, b, b, Wb, b, b, Cdev.ptr, nullptr);
        launch_pdl("k_qr1", k_qr1, 1, 64, 0, s, Cdev.ptr, b, hnorm, Mdev.ptr, Rdev.ptr, qstat.ptr);
        CI_CHECK_LAUNCH();
        nn(Wb, b, b, Mdev.ptr, b, Q.ptr + m, mmax, 1.0, 0.0);
        second_pass(m, par, qstat.ptr, 2);
    }

    // R of the block QR that wrote pinned slot par (waits for its copy) and
    // that pass's status: 0, else the device path left the block undone
    int take_R(int par, std::vector<double> &R) {
        CI_CUDA(cudaEventSynchronize(ev_R[par]));
        R.assign(pin_R + 64 * par, pin_R + 64 * par + (size_t)b * b);
        last_skip = pin_stat[2 * par + 1];
        return pin_stat[2 * par];
    }
};

// Ritz analysis of T[0:m, 0:m] with last-block coupling R (b x b).
struct Ritz {
    std::vector<double> theta, S, res;
};

Ritz ritz(const std::vector<double> &T, int ldt, int m, int b, const std::vector<double> &R, int k) {
    Ritz o;
    std::vector<double> A((size_t)m * m);
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) A[(size_t)i * m + j] = 0.5 * (T[(size_t)i * ldt + j] + T[(size_t)j * ldt + i]);
    sym_eig(m, A, o.theta, o.S);
    o.res.assign(std::min(k, m), 0.0);
    for (int i = 0; i < (int)o.res.size(); ++i) {
        double ss = 0.0;
        for (int r = 0; r < b; ++r) {
            double x = 0.0;
            for (int c = 0; c < b; ++c) x += R[(size_t)r * b + c] * o.S[(size_t)(m - b + c) * m + i];
            ss += x * x;
        }
        o.res[i] = std::sqrt(ss);
    }
    return o;
}

}  // namespace

void lowest_eigs(const Matrix *H, const ci_eig_opts *opts_in, double *evals, double *evecs, ci_eig_info *info,
                 cudaStream_t s) {
    auto t_start = std::chrono::steady_clock::now();
    if (!H) fail(CI_ERR_INVALID_ARG, "matrix is NULL");
    if (!evals) fail(CI_ERR_INVALID_ARG, "evals is NULL");
    ci_eig_opts o = opts_in ? *opts_in : ci_eig_opts{};
    if (o.k == 0) o.k = 5;
    if (o.block == 0) o.block = 8;
    if (o.max_basis == 0) o.max_basis = 64;
    if (o.max_iter == 0) o.max_iter = 2000;
    if (o.tol == 0.0) o.tol = H->vtype == CI_F64 ? 1e-10 : 1e-6;
    if (o.seed == 0) o.seed = 1;
    if (o.reorth_passes == 0) o.reorth_passes = 1;
    if (o.check_every == 0) o.check_every = 1;   // the host check overlaps the next product
    if (o.k < 1 || o.k > 32) fail(CI_ERR_INVALID_ARG, "k must be 1..32");
    if (o.block < 1 || o.block > 8) fail(CI_ERR_INVALID_ARG, "block must be 1..8");
    if (o.reorth_passes < 1 || o.reorth_passes > 2) fail(CI_ERR_INVALID_ARG, "reorth_passes must be 1..2");
    if (o.max_basis > kMaxNa) fail(CI_ERR_CAPACITY, "max_basis above %d", kMaxNa);
    const int64_t dim = H->dim;
    if (dim < o.k) fail(CI_ERR_INVALID_ARG, "k = %d exceeds the dimension %lld", o.k, (long long)dim);
    int b = o.block;
    int mmax = (o.max_basis / b) * b;
    if (mmax < o.k + 2 * b) fail(CI_ERR_INVALID_ARG, "max_basis must be >= k + 2*block");
    const int k = o.k;
    ci_eig_info inf{};

    // small spaces: Rayleigh-Ritz on the whole space (Q = I, so the
    // projection Q^T H Q is H itself, applied to identity blocks)
    if (dim <= (int64_t)mmax + 2 * b) {
        const int n = (int)dim;
        const int bb = std::min<int>(b, n);
        DevBuf<double> E((size_t)n * bb), Wd((size_t)n * bb);
        DevBuf<float> E32((size_t)n * bb), W32((size_t)n * bb);
        std::vector<double> T((size_t)n * n, 0.0), Eh((size_t)n * bb), Wh((size_t)n * bb);
        for (int j0 = 0; j0 < n; j0 += bb) {
            int nb = std::min(bb, n - j0);
            std::fill(Eh.begin(), Eh.end(), 0.0);
            for (int v = 0; v < nb; ++v) Eh[(size_t)(j0 + v) * nb + v] = 1.0;
            if (H->vtype == CI_F64) {
                CI_CUDA(cudaMemcpyAsync(E.ptr, Eh.data(), sizeof(double) * n * nb, cudaMemcpyHostToDevice, s));
                apply_matrix(H, E.ptr, Wd.ptr, nb, s);
                CI_CUDA(cudaMemcpyAsync(Wh.data(), Wd.ptr, sizeof(double) * n * nb, cudaMemcpyDeviceToHost, s));
                CI_CUDA(cudaStreamSynchronize(s));
            } else {
                std::vector<float> Ef(Eh.begin(), Eh.begin() + (size_t)n * nb), Wf((size_t)n * nb);
                CI_CUDA(cudaMemcpyAsync(E32.ptr, Ef.data(), sizeof(float) * n * nb, cudaMemcpyHostToDevice, s));
                apply_matrix(H, E32.ptr, W32.ptr, nb, s);
                CI_CUDA(cudaMemcpyAsync(Wf.data(), W32.ptr, sizeof(float) * n * nb, cudaMemcpyDeviceToHost, s));
                CI_CUDA(cudaStreamSynchronize(s));
                for (size_t e = 0; e < Wf.size(); ++e) Wh[e] = Wf[e];
            }
            for (int i = 0; i < n; ++i)
                for (int v = 0; v < nb; ++v) T[(size_t)i * n + j0 + v] = Wh[(size_t)i * nb + v];
        }
        std::vector<double> A((size_t)n * n), w, Z;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) A[(size_t)i * n + j] = 0.5 * (T[(size_t)i * n + j] + T[(size_t)j * n + i]);
        sym_eig(n, A, w, Z);
        for (int i = 0; i < k; ++i) evals[i] = w[i];
        if (evecs) {
            std::vector<double> X((size_t)n * k);
            for (int r = 0; r < n; ++r)
                for (int i = 0; i < k; ++i) X[(size_t)r * k + i] = Z[(size_t)r * n + i];
            CI_CUDA(cudaMemcpyAsync(evecs, X.data(), sizeof(double) * n * k, cudaMemcpyHostToDevice, s));
        }
        // residuals of the Ritz pairs against the dense projection (exact space)
        for (int i = 0; i < k; ++i) {
            double ss = 0.0;
            for (int r = 0; r < n; ++r) {
                double x = 0.0;
                for (int c = 0; c < n; ++c) x += T[(size_t)r * n + c] * Z[(size_t)c * n + i];
                x -= w[i] * Z[(size_t)r * n + i];
                ss += x * x;
            }
            inf.residual[i] = std::sqrt(ss);
        }
        inf.iterations = (n + bb - 1) / bb;
        inf.converged = k;
        inf.basis_size = n;
        inf.hnorm_est = std::max(std::fabs(w.front()), std::fabs(w.back()));
        CI_CUDA(cudaStreamSynchronize(s));
        inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
        if (info) *info = inf;
        return;
    }

    Solver sv(H, s, b, k, mmax);
    sv.tc = o.fp64_products == 0;
    std::vector<double> T((size_t)mmax * mmax, 0.0);
    std::vector<double> coef;
    // start block (its R is not needed: pinned slot 1, never read)
    launch("k_random_cols", k_random_cols, sv.grid(dim * b), 256, 0, s, dim, b, o.seed, sv.W.ptr, b);
    CI_CHECK_LAUNCH();
    sv.block_qr(sv.W.ptr, 0, o.seed ^ 0x5bd1e995ull, 1);
    int m_cur = b, j0 = 0;
    int it = 0, since_check = 0;
    bool converged = false;
    Ritz last;
    int m_act = 0;
    std::vector<double> Rlast;
    bool applied = false;   // H V_j already enqueued (before the last host Ritz check)
    // W = H V_j alternates between two buffers, so that a step's W is still
    // there when its block QR has to be redone on the host path
    sv.W2.alloc((size_t)dim * b);
    double *Wcur = sv.W.ptr, *Wnext = sv.W2.ptr;
    int par = 0, host_qr = 0, one_pass = 0;
    while (true) {
        // W = H V_j, orthogonalised against the whole basis
        if (!applied) sv.apply(sv.Q.ptr + j0, mmax, b, Wcur);
        applied = false;
        sv.project_deferred(Wcur, b, m_cur, std::max(0, j0 - b), o.reorth_passes);
        ++it;
        // next block, on the device: no host sync before the next product
        // is enqueued
        sv.block_qr_dev(Wcur, m_cur, par);
        sv.take_coef(&coef);
        for (int i = 0; i < j0; ++i)
            for (int v = 0; v < b; ++v) {
                T[(size_t)i * mmax + j0 + v] = coef[(size_t)i * b + v];
                T[(size_t)(j0 + v) * mmax + i] = coef[(size_t)i * b + v];
            }
        for (int u = 0; u < b; ++u)  // diagonal block, symmetrised
            for (int v = 0; v < b; ++v)
                T[(size_t)(j0 + u) * mmax + j0 + v] =
                    0.5 * (coef[(size_t)(j0 + u) * b + v] + coef[(size_t)(j0 + v) * b + u]);
        const int row0 = m_cur, col0 = j0, qpar = par;
        par ^= 1;
        m_act = m_cur;
        j0 = m_cur;
        m_cur += b;
        const bool full = m_cur + b > mmax;
        // the next product only needs the new block: the GPU computes it
        // while the host reads the coupling and solves the projected problem
        // (wasted once, at convergence)
        if (!full && it < o.max_iter) {
            sv.apply(sv.Q.ptr + j0, mmax, b, Wnext);
            applied = true;
        }
        if (sv.take_R(qpar, Rlast) == 0) {
            one_pass += sv.last_skip;
        } else {
            // rank deficient (or the second pass did not settle): the
            // rank-revealing host path redoes the block from the same W, and
            // the product just enqueued is redone with the new block
            sv.block_qr(Wcur, row0, o.seed + 0x9E37ull * (uint64_t)(it + 1), qpar);
            sv.take_R(qpar, Rlast);
            applied = false;
            ++host_qr;
        }
        for (int r = 0; r < b; ++r)
            for (int c = 0; c < b; ++c) {
                T[(size_t)(row0 + r) * mmax + col0 + c] = Rlast[(size_t)r * b + c];
                T[(size_t)(col0 + c) * mmax + row0 + r] = Rlast[(size_t)r * b + c];
            }
        std::swap(Wcur, Wnext);
        ++since_check;
        if (since_check >= o.check_every || full || it >= o.max_iter) {
            since_check = 0;
            last = ritz(T, mmax, m_act, b, Rlast, k);
            sv.hnorm = std::max(sv.hnorm, std::max(std::fabs(last.theta.front()), std::fabs(last.theta.back())));
            converged = (int)last.res.size() >= k;
            for (int i = 0; i < k && converged; ++i)
                if (last.res[i] > o.tol * sv.hnorm) converged = false;
            if (converged || it >= o.max_iter) break;
        }
        if (full) {
            // thick restart: keep the lowest Ritz vectors and the new block
            int keep = std::max(k + b, m_act / 2);
            keep = std::min(keep, m_act - b);
            std::vector<double> Sk((size_t)m_act * keep);
            for (int r = 0; r < m_act; ++r)
                for (int i = 0; i < keep; ++i) Sk[(size_t)r * keep + i] = last.S[(size_t)r * m_act + i];
            for (int c0 = 0; c0 < keep; c0 += 8) {
                int nc = std::min(8, keep - c0);
                std::vector<double> Sc((size_t)m_act * nc);
                for (int r = 0; r < m_act; ++r)
                    for (int i = 0; i < nc; ++i) Sc[(size_t)r * nc + i] = Sk[(size_t)r * keep + c0 + i];
                sv.upload(Sc, sv.Mdev.ptr);
                sv.nn(sv.Q.ptr, mmax, m_act, sv.Mdev.ptr, nc, sv.tmp.ptr + c0, keep, 1.0, 0.0, true);
            }
            // new block Q[:, m_act:m_act+b] -> Q[:, keep:keep+b]; Ritz vectors -> Q[:, 0:keep]
            sv.copy_into_basis(sv.Q.ptr + m_act, mmax, keep, b);
            sv.copy_into_basis(sv.tmp.ptr, keep, 0, keep);
            std::fill(T.begin(), T.end(), 0.0);
            for (int i = 0; i < keep; ++i) T[(size_t)i * mmax + i] = last.theta[i];
            for (int r = 0; r < b; ++r)
                for (int i = 0; i < keep; ++i) {
                    double x = 0.0;
                    for (int c = 0; c < b; ++c) x += Rlast[(size_t)r * b + c] * last.S[(size_t)(m_act - b + c) * m_act + i];
                    T[(size_t)(keep + r) * mmax + i] = x;
                    T[(size_t)i * mmax + keep + r] = x;
                }
            m_cur = keep + b;
            j0 = keep;
            ++inf.restarts;
        }
    }
    // Ritz pairs, eigenvectors and FP64 residuals with the stored H
    for (int i = 0; i < k; ++i) evals[i] = last.theta[i];
    std::vector<double> Sk((size_t)m_act * k);
    for (int r = 0; r < m_act; ++r)
        for (int i = 0; i < k; ++i) Sk[(size_t)r * k + i] = last.S[(size_t)r * m_act + i];
    double *X = sv.tmp.ptr;  // [dim][k]
    for (int c0 = 0; c0 < k; c0 += 8) {
        int nc = std::min(8, k - c0);
        std::vector<double> Sc((size_t)m_act * nc);
        for (int r = 0; r < m_act; ++r)
            for (int i = 0; i < nc; ++i) Sc[(size_t)r * nc + i] = Sk[(size_t)r * k + c0 + i];
        sv.upload(Sc, sv.Mdev.ptr);
        sv.nn(sv.Q.ptr, mmax, m_act, sv.Mdev.ptr, nc, X + c0, k, 1.0, 0.0);
    }
    for (int c0 = 0; c0 < k; c0 += b) {
        int nc = std::min(b, k - c0);
        sv.apply(X + c0, k, nc, sv.W.ptr);  // W [dim][nc] = H x
        std::vector<double> th(last.theta.begin() + c0, last.theta.begin() + c0 + nc);
        sv.upload(th, sv.theta_dev.ptr);
        double *Rr = sv.Q.ptr;  // basis no longer needed: scratch [dim][nc]
        launch("k_residual", k_residual<double>, sv.grid(dim * nc), 256, 0, s, dim, nc, sv.W.ptr, X + c0, k, sv.theta_dev.ptr, Rr);
        CI_CHECK_LAUNCH();
        std::vector<double> G;
        sv.tn(Rr, nc, nc, Rr, nc, nc, sv.Cdev.ptr, &G);
        for (int i = 0; i < nc; ++i) inf.residual[c0 + i] = std::sqrt(std::max(G[(size_t)i * nc + i], 0.0));
    }
    if (evecs) CI_CUDA(cudaMemcpyAsync(evecs, X, sizeof(double) * dim * k, cudaMemcpyDeviceToDevice, s));
    int ozf = 0;
    CI_CUDA(cudaMemcpyAsync(&ozf, sv.ozflag.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
    CI_CUDA(cudaStreamSynchronize(s));
    if (ozf) fail(CI_ERR_INTERNAL, "a tensor-core basis product or the device block QR failed (flag %d)", ozf);
    inf.iterations = it;
    inf.basis_size = m_act;
    inf.hnorm_est = sv.hnorm;
    inf.host_qr = host_qr;
    inf.qr_one_pass = one_pass;
    inf.converged = 0;
    for (int i = 0; i < k; ++i)
        if (last.res[i] <= o.tol * sv.hnorm) ++inf.converged;
    inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    if (info) *info = inf;
    if (!converged) fail(CI_ERR_NOT_CONVERGED, "block Lanczos stopped after %d steps (%d of %d converged)", it,
                         inf.converged, k);
}

// ------------------------------------------------------------------ LOBPCG

// Lower Cholesky factor of the symmetric positive definite n x n matrix A
// (row-major); false if a pivot is not above rel * max diagonal.
static bool cholesky_lower(int n, const std::vector<double> &A, std::vector<double> &L, double rel) {
    L.assign((size_t)n * n, 0.0);
    double dmax = 0.0;
    for (int i = 0; i < n; ++i) dmax = std::max(dmax, A[(size_t)i * n + i]);
    for (int j = 0; j < n; ++j) {
        double d = A[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) d -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
        if (!(d > rel * dmax)) return false;
        const double ljj = std::sqrt(d);
        L[(size_t)j * n + j] = ljj;
        for (int i = j + 1; i < n; ++i) {
            double x = A[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) x -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
            L[(size_t)i * n + j] = x / ljj;
        }
    }
    return true;
}

// Lowest nb pairs of the pencil (GA, GB), n x n: GB = L L^T, eigenpairs of
// L^-1 GA L^-T, C = L^-T Z (n x nb, row-major).  False if GB is not
// positive definite enough.
static bool pencil_lowest(int n, int nb, const std::vector<double> &GA, const std::vector<double> &GB,
                          std::vector<double> &theta, std::vector<double> &C) {
    std::vector<double> L;
    if (!cholesky_lower(n, GB, L, 1e-8)) return false;   // the blocks are orthonormalised: GB ~ I
    // M = L^-1 GA L^-T: solve L Y = GA, then L M^T = Y^T
    std::vector<double> Y((size_t)n * n), M((size_t)n * n);
    for (int c = 0; c < n; ++c)
        for (int i = 0; i < n; ++i) {
            double x = GA[(size_t)i * n + c];
            for (int k = 0; k < i; ++k) x -= L[(size_t)i * n + k] * Y[(size_t)k * n + c];
            Y[(size_t)i * n + c] = x / L[(size_t)i * n + i];
        }
    for (int r = 0; r < n; ++r)
        for (int i = 0; i < n; ++i) {
            double x = Y[(size_t)r * n + i];
            for (int k = 0; k < i; ++k) x -= L[(size_t)i * n + k] * M[(size_t)r * n + k];
            M[(size_t)r * n + i] = x / L[(size_t)i * n + i];
        }
    for (int r = 0; r < n; ++r)
        for (int c = r + 1; c < n; ++c) {
            const double a = 0.5 * (M[(size_t)r * n + c] + M[(size_t)c * n + r]);
            M[(size_t)r * n + c] = a;
            M[(size_t)c * n + r] = a;
        }
    std::vector<double> w, Z;
    if (!sym_eig(n, M, w, Z)) return false;
    theta.assign(w.begin(), w.begin() + nb);
    // C = L^-T Z[:, :nb]: back substitution with L^T
    C.assign((size_t)n * nb, 0.0);
    for (int v = 0; v < nb; ++v)
        for (int i = n - 1; i >= 0; --i) {
            double x = Z[(size_t)i * n + v];
            for (int k = i + 1; k < n; ++k) x -= L[(size_t)k * n + i] * C[(size_t)k * nb + v];
            C[(size_t)i * nb + v] = x / L[(size_t)i * n + i];
        }
    return true;
}

void lowest_eigs_lobpcg(const Matrix *H, const ci_eig_opts *opts_in, const int32_t *row_block, int64_t nblocks,
                        double *evals, double *evecs, ci_eig_info *info, cudaStream_t s) {
    auto t_start = std::chrono::steady_clock::now();
    if (!H) fail(CI_ERR_INVALID_ARG, "matrix is NULL");
    if (!evals) fail(CI_ERR_INVALID_ARG, "evals is NULL");
    ci_eig_opts o = opts_in ? *opts_in : ci_eig_opts{};
    if (o.k == 0) o.k = 5;
    if (o.block == 0) o.block = 8;
    if (o.max_iter == 0) o.max_iter = 1000;
    // BF16 values with per-row scales are not exactly symmetric (H_ij and H_ji
    // round differently): the true residual stops near that rounding
    if (o.tol == 0.0) o.tol = H->vtype == CI_F64 ? 1e-10 : H->vtype == CI_BF16_ROWSCALE ? 4e-3 : 1e-6;
    if (o.seed == 0) o.seed = 1;
    if (o.block < 1 || o.block > 8) fail(CI_ERR_INVALID_ARG, "block must be 1..8");
    if (o.k < 1 || o.k > o.block) fail(CI_ERR_INVALID_ARG, "LOBPCG needs 1 <= k <= block (k = %d, block = %d)", o.k,
                                       o.block);
    const int64_t dim = H->dim;
    const int nb = o.block, k = o.k;
    if (dim <= 4 * (int64_t)nb) {  // too small for three blocks: the dense path of the Lanczos solver
        ci_eig_opts d = o;
        d.max_basis = 0;
        lowest_eigs(H, &d, evals, evecs, info, s);
        return;
    }
    Solver sv(H, s, nb, k, nb);
    const size_t blk = (size_t)dim * nb;
    DevBuf<double> X(blk), AX(blk), Wd(blk), AW(blk), P(blk), AP(blk), R(blk), Xn(blk), AXn(blk), Pn(blk), APn(blk);
    DevBuf<double> dg((size_t)dim), G((size_t)12 * 64), Cd((size_t)3 * 64);
    if (H->vtype == CI_F64)
        launch("k_diag", k_diag<double>, sv.grid(dim), 256, 0, s, dim, H->row_ptr.ptr, H->col.ptr,
               (const double *)H->val.ptr, (const float *)nullptr, dg.ptr);
    else if (H->vtype == CI_F32)
        launch("k_diag", k_diag<float>, sv.grid(dim), 256, 0, s, dim, H->row_ptr.ptr, H->col.ptr,
               (const float *)H->val.ptr, (const float *)nullptr, dg.ptr);
    else if (H->vtype == CI_BF16_ROWSCALE)
        launch("k_diag", k_diag<__nv_bfloat16>, sv.grid(dim), 256, 0, s, dim, H->row_ptr.ptr, H->col.ptr,
               (const __nv_bfloat16 *)H->val.ptr, (const float *)H->row_scale.ptr, dg.ptr);
    else
        fail(CI_ERR_INVALID_ARG, "value type %d not supported by LOBPCG", H->vtype);
    // many-body-orbital block preconditioner (else the diagonal of H): the
    // shifted blocks are inverted at iterations 0, 2, 6, 14, ... with the
    // shift sigma = theta_1 - |r_1| of the latest Rayleigh-Ritz
    std::unique_ptr<BlockPrecond> bp;
    if (row_block) {
        bp.reset(new BlockPrecond);
        precond_setup(*bp, H, row_block, nblocks, s);
    }
    int next_factor = 0;
    const int bb = nb * nb;
    // Gram blocks into G (device), one copy to the host
    auto gram = [&](const std::vector<std::pair<const double *, const double *>> &pairs, std::vector<double> &h) {
        for (size_t q = 0; q < pairs.size(); ++q)
            sv.tn(pairs[q].first, nb, nb, pairs[q].second, nb, nb, G.ptr + q * 64, nullptr);
        h.resize(pairs.size() * 64);
        CI_CUDA(cudaMemcpyAsync(h.data(), G.ptr, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s));
        CI_CUDA(cudaStreamSynchronize(s));
    };
    // out = sum_q A_q C_q (C_q nb x nb row-major blocks of the host matrix C)
    auto combine = [&](const std::vector<const double *> &As, const std::vector<double> &C, int row0, double *out) {
        std::vector<double> cq((size_t)As.size() * bb);
        for (size_t q = 0; q < As.size(); ++q)
            for (int u = 0; u < nb; ++u)
                for (int v = 0; v < nb; ++v) cq[q * bb + u * nb + v] = C[(size_t)(row0 + (int)q * nb + u) * nb + v];
        CI_CUDA(cudaMemcpyAsync(Cd.ptr, cq.data(), sizeof(double) * cq.size(), cudaMemcpyHostToDevice, s));
        for (size_t q = 0; q < As.size(); ++q) sv.nn(As[q], nb, nb, Cd.ptr + q * bb, nb, out, nb, 1.0, q ? 1.0 : 0.0);
    };
    std::vector<double> theta(nb, 0.0), rn(nb, 0.0), h, C;
    auto upload_theta = [&]() { sv.upload(theta, sv.theta_dev.ptr); };
    // start: random block, Rayleigh-Ritz on it
    launch("k_random_cols", k_random_cols, sv.grid(dim * nb), 256, 0, s, dim, nb, o.seed, X.ptr, nb);
    sv.apply(X.ptr, nb, nb, AX.ptr);
    gram({{X.ptr, X.ptr}, {X.ptr, AX.ptr}}, h);
    {
        std::vector<double> GB(h.begin(), h.begin() + bb), GA(h.begin() + 64, h.begin() + 64 + bb);
        if (!pencil_lowest(nb, nb, GA, GB, theta, C)) fail(CI_ERR_INTERNAL, "LOBPCG start block is degenerate");
        combine({X.ptr}, C, 0, Xn.ptr);
        combine({AX.ptr}, C, 0, AXn.ptr);
        std::swap(X, Xn);
        std::swap(AX, AXn);
    }
    bool haveP = false, converged = false;
    int it = 0;
    double hnorm = 0.0;
    ci_eig_info inf{};
    DevBuf<double> Cp((size_t)64), Tmp(blk), ATmp(blk);
    // B -= A (A^T B) (and AB -= AA (A^T B)), on the device
    auto project_out = [&](const double *A, const double *AA, double *B, double *AB) {
        sv.tn(A, nb, nb, B, nb, nb, Cp.ptr, nullptr);
        sv.nn(A, nb, nb, Cp.ptr, nb, B, nb, -1.0, 1.0);
        if (AB) sv.nn(AA, nb, nb, Cp.ptr, nb, AB, nb, -1.0, 1.0);
    };
    // B = B L^-T with B^T B = L L^T (and AB likewise); false if B lost rank
    // before (optional): the squared column norms before a projection; a
    // column that lost more than all but 1e-8 of it is mostly rounding
    // (and for P, drift of its tracked H product): the block is not used
    auto chol_qr = [&](DevBuf<double> &B, DevBuf<double> *AB, const std::vector<double> *before) -> bool {
        std::vector<double> g;
        gram({{B.ptr, B.ptr}}, g);
        // columns scaled to unit norm first (D G D, D = diag(G)^-1/2), so the
        // rank test is relative to each column's own length
        std::vector<double> Gm(g.begin(), g.begin() + bb), L, dsc(nb);
        for (int i = 0; i < nb; ++i) {
            const double d = Gm[(size_t)i * nb + i];
            if (!(d > 1e-300)) return false;
            if (before && !(d > 1e-8 * (*before)[i])) return false;
            dsc[i] = 1.0 / std::sqrt(d);
        }
        for (int i = 0; i < nb; ++i)
            for (int j = 0; j < nb; ++j) Gm[(size_t)i * nb + j] *= dsc[i] * dsc[j];
        if (!cholesky_lower(nb, Gm, L, 1e-14)) return false;
        std::vector<double> Mi((size_t)bb, 0.0);   // D L^-T, upper triangular
        for (int c = 0; c < nb; ++c)
            for (int i = c; i >= 0; --i) {
                double x = i == c ? 1.0 : 0.0;
                for (int k2 = i + 1; k2 <= c; ++k2) x -= L[(size_t)k2 * nb + i] * Mi[(size_t)k2 * nb + c];
                Mi[(size_t)i * nb + c] = x / L[(size_t)i * nb + i];
            }
        for (int i = 0; i < nb; ++i)
            for (int c = 0; c < nb; ++c) Mi[(size_t)i * nb + c] *= dsc[i];
        sv.upload(Mi, Cp.ptr);
        sv.nn(B.ptr, nb, nb, Cp.ptr, nb, Tmp.ptr, nb, 1.0, 0.0);
        std::swap(B, Tmp);
        if (AB) {
            sv.nn(AB->ptr, nb, nb, Cp.ptr, nb, ATmp.ptr, nb, 1.0, 0.0);
            std::swap(*AB, ATmp);
        }
        return true;
    };
    for (; it < o.max_iter; ++it) {
        // the H products are applied afresh every iteration: products carried
        // through the updates drift by the SpMM's rounding, which the
        // orthonormalisation of nearly converged blocks would amplify
        if (it > 0) {
            if (haveP && nb == 8) sv.apply2(X.ptr, nb, P.ptr, nb, AX.ptr, AP.ptr);
            else {
                sv.apply(X.ptr, nb, nb, AX.ptr);
                if (haveP) sv.apply(P.ptr, nb, nb, AP.ptr);
            }
        }
        upload_theta();
        launch("k_residual", k_residual<double>, sv.grid(dim * nb), 256, 0, s, dim, nb, AX.ptr, X.ptr, nb,
               sv.theta_dev.ptr, R.ptr);
        for (int v = 0; v < nb; ++v) hnorm = std::max(hnorm, std::fabs(theta[v]));
        gram({{R.ptr, R.ptr}}, h);
        for (int v = 0; v < nb; ++v) rn[v] = std::sqrt(std::max(h[(size_t)v * nb + v], 0.0));
        converged = true;
        for (int v = 0; v < k; ++v)
            if (rn[v] > o.tol * hnorm) converged = false;
        if (converged) break;
        // W: preconditioned residuals, orthonormal and orthogonal to X (two
        // Gram-Schmidt passes, then Cholesky QR); AW = H W
        if (bp) {
            if (it == next_factor) {
                precond_factor(*bp, H, theta[0] - rn[0], s);
                next_factor = 2 * it + 2;
            }
            precond_apply(*bp, R.ptr, nb, Wd.ptr, s);
        } else {
            launch("k_precond", k_precond, sv.grid(dim * nb), 256, 0, s, dim, nb, R.ptr, dg.ptr, sv.theta_dev.ptr,
                   1e-8, Wd.ptr);
        }
        auto col_norms = [&](const double *B) {
            std::vector<double> g;
            gram({{B, B}}, g);
            std::vector<double> d(nb);
            for (int i = 0; i < nb; ++i) d[i] = g[(size_t)i * nb + i];
            return d;
        };
        std::vector<double> wn = col_norms(Wd.ptr);
        project_out(X.ptr, nullptr, Wd.ptr, nullptr);
        project_out(X.ptr, nullptr, Wd.ptr, nullptr);
        bool useW = chol_qr(Wd, nullptr, &wn);
        if (!useW) {   // the preconditioned residuals lie in span(X) (e.g. diagonal H): take R itself
            launch_pdl("k_copy_cols", k_copy_cols, sv.grid(dim * nb), 256, 0, s, dim, nb, R.ptr, nb, Wd.ptr, nb);
            project_out(X.ptr, nullptr, Wd.ptr, nullptr);
            project_out(X.ptr, nullptr, Wd.ptr, nullptr);
            useW = chol_qr(Wd, nullptr, nullptr);
        }
        if (useW) sv.apply(Wd.ptr, nb, nb, AW.ptr);
        // P: orthogonal to X and W, orthonormal (its H product follows)
        bool useP = haveP;
        if (useP) {
            std::vector<double> g0;
            gram({{P.ptr, P.ptr}}, g0);
            std::vector<double> before(nb);
            for (int i = 0; i < nb; ++i) before[i] = g0[(size_t)i * nb + i];
            for (int pass = 0; pass < 2; ++pass) {
                project_out(X.ptr, AX.ptr, P.ptr, AP.ptr);
                if (useW) project_out(Wd.ptr, AW.ptr, P.ptr, AP.ptr);
            }
            useP = chol_qr(P, &AP, &before);
        }
        if (!useW && !useP) break;        // the search space is X alone
        // Rayleigh-Ritz on S = [X W P] (orthonormal blocks): the pencil's
        // overlap is I up to rounding; its Cholesky keeps the new X exactly
        // orthonormal in it
        std::vector<const double *> S{X.ptr}, AS{AX.ptr};
        if (useW) { S.push_back(Wd.ptr); AS.push_back(AW.ptr); }
        if (useP) { S.push_back(P.ptr); AS.push_back(AP.ptr); }
        const int nblk = (int)S.size(), n = nblk * nb;
        std::vector<std::pair<const double *, const double *>> pairs;
        for (int a = 0; a < nblk; ++a)
            for (int b = a; b < nblk; ++b) {
                pairs.push_back({S[a], S[b]});
                pairs.push_back({S[a], AS[b]});
            }
        gram(pairs, h);
        std::vector<double> GA((size_t)n * n), GB((size_t)n * n);
        int q = 0;
        for (int a = 0; a < nblk; ++a)
            for (int b = a; b < nblk; ++b, q += 2)
                for (int u = 0; u < nb; ++u)
                    for (int v = 0; v < nb; ++v) {
                        const double gb = h[(size_t)q * 64 + u * nb + v], ga = h[(size_t)(q + 1) * 64 + u * nb + v];
                        GB[(size_t)(a * nb + u) * n + b * nb + v] = gb;
                        GB[(size_t)(b * nb + v) * n + a * nb + u] = gb;
                        GA[(size_t)(a * nb + u) * n + b * nb + v] = ga;
                        if (a != b) GA[(size_t)(b * nb + v) * n + a * nb + u] = ga;
                    }
        for (int r = 0; r < n; ++r)   // S^T H S is symmetric: average the diagonal blocks
            for (int c = r + 1; c < n; ++c)
                if (r / nb == c / nb) {
                    const double x = 0.5 * (GA[(size_t)r * n + c] + GA[(size_t)c * n + r]);
                    GA[(size_t)r * n + c] = x;
                    GA[(size_t)c * n + r] = x;
                }
        if (!pencil_lowest(n, nb, GA, GB, theta, C)) break;
        // P = W Cw (+ P Cp), X = X Cx + P; the same for the H products
        std::vector<const double *> ws(S.begin() + 1, S.end()), aws(AS.begin() + 1, AS.end());
        combine(ws, C, nb, Pn.ptr);
        combine({X.ptr}, C, 0, Xn.ptr);
        launch("k_axpy", k_axpy, sv.grid(dim * nb), 256, 0, s, (int64_t)blk, Pn.ptr, Xn.ptr);
        (void)aws;
        std::swap(X, Xn);
        std::swap(P, Pn);
        haveP = true;
    }
    // FP64 residuals of the final pairs with the stored H
    upload_theta();
    sv.apply(X.ptr, nb, nb, AXn.ptr);
    launch("k_residual", k_residual<double>, sv.grid(dim * nb), 256, 0, s, dim, nb, AXn.ptr, X.ptr, nb,
           sv.theta_dev.ptr, R.ptr);
    gram({{R.ptr, R.ptr}, {X.ptr, X.ptr}}, h);
    for (int i = 0; i < k; ++i) {
        evals[i] = theta[i];
        inf.residual[i] = std::sqrt(std::max(h[(size_t)i * nb + i], 0.0));
    }
    if (evecs) {
        launch_pdl("k_copy_cols", k_copy_cols, sv.grid(dim * k), 256, 0, s, dim, k, X.ptr, nb, evecs, k);
        CI_CHECK_LAUNCH();
    }
    CI_CUDA(cudaStreamSynchronize(s));
    inf.iterations = it;
    inf.basis_size = 3 * nb;
    inf.hnorm_est = hnorm;
    inf.converged = 0;
    for (int i = 0; i < k; ++i)
        if (inf.residual[i] <= std::max(o.tol, 1e-12) * hnorm * 1.5) ++inf.converged;
    inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    if (info) *info = inf;
    if (!converged) fail(CI_ERR_NOT_CONVERGED, "LOBPCG stopped after %d iterations", it);
}

// Refinement of k Ritz pairs with the FP64 Hamiltonian applied on the fly:
// Rayleigh-Ritz on span(X) with H in FP64, then `iters` Rayleigh-Ritz steps
// on span[X, R] (R = H X - X Theta, the FP64 residuals).  X [dim][k] is
// overwritten with the refined vectors (orthonormal), evals / resid (host)
// receive the Ritz values and the FP64 residual norms.
void refine_eigs(Problem *P, int k, int iters, double *X, double *evals, double *resid, cudaStream_t s) {
    if (k < 1 || k > 16) fail(CI_ERR_INVALID_ARG, "k must be 1..16 (got %d)", k);
    if (iters < 0 || iters > 16) fail(CI_ERR_INVALID_ARG, "iters must be 0..16 (got %d)", iters);
    if (!evals) fail(CI_ERR_INVALID_ARG, "evals is NULL");
    enumerate_basis(P, s);
    const int64_t dim = P->dim;
    if (dim < 2 * (int64_t)k) fail(CI_ERR_INVALID_ARG, "dimension %lld too small for k = %d", (long long)dim, k);
    if (!X || !is_device_pointer(X)) fail(CI_ERR_INVALID_ARG, "evecs must be a device pointer");
    Matrix shape;   // only the dimension: the products below are dense
    shape.dim = dim;
    shape.vtype = CI_F64;
    const int n2 = 2 * k;
    Solver sv(&shape, s, 8, k, 8);
    DevBuf<double> S((size_t)dim * n2), HS((size_t)dim * n2), T8((size_t)dim * 8), Y8((size_t)dim * 8),
        Tmp((size_t)dim * n2), Rb((size_t)dim * k), G((size_t)n2 * n2);
    // HS[:, c0:c0+nc] = H S[:, c0:c0+nc], eight columns per on-the-fly pass
    auto apply_cols = [&](int c0, int nc) {
        for (int g = 0; g < nc; g += 8) {
            const int m = std::min(8, nc - g);
            CI_CUDA(cudaMemsetAsync(T8.ptr, 0, sizeof(double) * dim * 8, s));
            launch_pdl("k_copy_cols", k_copy_cols, sv.grid(dim * m), 256, 0, s, dim, m, S.ptr + c0 + g, n2, T8.ptr, 8);
            h64_apply(P, T8.ptr, Y8.ptr, s);
            launch_pdl("k_copy_cols", k_copy_cols, sv.grid(dim * m), 256, 0, s, dim, m, Y8.ptr, 8, HS.ptr + c0 + g, n2);
        }
    };
    auto gram = [&](const double *A, const double *B, int n, std::vector<double> &h) {
        sv.tn(A, n2, n, B, n2, n, G.ptr, &h);
    };
    // [S HS][:, 0:k] = [S HS][:, 0:n] C (n x k, host)
    auto rotate = [&](int n, const std::vector<double> &C) {
        sv.upload(C, sv.Cdev.ptr);
        sv.nn(S.ptr, n2, n, sv.Cdev.ptr, k, Tmp.ptr, k, 1.0, 0.0);
        launch_pdl("k_copy_cols", k_copy_cols, sv.grid(dim * k), 256, 0, s, dim, k, Tmp.ptr, k, S.ptr, n2);
        sv.nn(HS.ptr, n2, n, sv.Cdev.ptr, k, Tmp.ptr, k, 1.0, 0.0);
        launch_pdl("k_copy_cols", k_copy_cols, sv.grid(dim * k), 256, 0, s, dim, k, Tmp.ptr, k, HS.ptr, n2);
    };
    std::vector<double> theta(k), C, ga, gb;
    // Rayleigh-Ritz on n columns of S (pencil S^T H S, S^T S)
    auto rayleigh_ritz = [&](int n) -> bool {
        gram(S.ptr, HS.ptr, n, ga);
        gram(S.ptr, S.ptr, n, gb);
        for (int r = 0; r < n; ++r)   // S^T H S is symmetric: average the rounding
            for (int c = r + 1; c < n; ++c) {
                const double a = 0.5 * (ga[(size_t)r * n + c] + ga[(size_t)c * n + r]);
                ga[(size_t)r * n + c] = ga[(size_t)c * n + r] = a;
            }
        if (!pencil_lowest(n, k, ga, gb, theta, C)) return false;
        rotate(n, C);
        return true;
    };
    launch_pdl("k_copy_cols", k_copy_cols, sv.grid(dim * k), 256, 0, s, dim, k, X, k, S.ptr, n2);
    apply_cols(0, k);
    if (!rayleigh_ritz(k)) fail(CI_ERR_INVALID_ARG, "the k vectors are linearly dependent");
    std::vector<double> rn(k, 0.0);
    auto residuals = [&]() {
        sv.upload(theta, sv.theta_dev.ptr);
        // R = HX - X Theta into the second half of S (HX made contiguous first)
        launch_pdl("k_copy_cols", k_copy_cols, sv.grid(dim * k), 256, 0, s, dim, k, HS.ptr, n2, Tmp.ptr, k);
        launch("k_residual", k_residual<double>, sv.grid(dim * k), 256, 0, s, dim, k, Tmp.ptr, S.ptr, n2,
               sv.theta_dev.ptr, Rb.ptr);
        launch_pdl("k_copy_cols", k_copy_cols, sv.grid(dim * k), 256, 0, s, dim, k, Rb.ptr, k, S.ptr + k, n2);
        std::vector<double> h;
        gram(S.ptr + k, S.ptr + k, k, h);
        for (int v = 0; v < k; ++v) rn[v] = std::sqrt(std::max(h[(size_t)v * k + v], 0.0));
        return h;
    };
    for (int it = 0; it < iters; ++it) {
        std::vector<double> h = residuals();
        // unit residual columns, orthonormal (Cholesky QR), then Rayleigh-Ritz
        // on [X, R]; stop when R has no usable direction left
        std::vector<double> L, dsc(k);
        bool ok = true;
        for (int v = 0; v < k; ++v) {
            const double d = h[(size_t)v * k + v];
            if (!(d > 1e-300)) { ok = false; break; }
            dsc[v] = 1.0 / std::sqrt(d);
        }
        if (!ok) break;
        std::vector<double> Gm(h);
        for (int i = 0; i < k; ++i)
            for (int j = 0; j < k; ++j) Gm[(size_t)i * k + j] *= dsc[i] * dsc[j];
        if (!cholesky_lower(k, Gm, L, 1e-10)) break;
        std::vector<double> Mi((size_t)k * k, 0.0);   // D L^-T
        for (int c = 0; c < k; ++c)
            for (int i = c; i >= 0; --i) {
                double x = i == c ? 1.0 : 0.0;
                for (int q = i + 1; q <= c; ++q) x -= L[(size_t)q * k + i] * Mi[(size_t)q * k + c];
                Mi[(size_t)i * k + c] = x / L[(size_t)i * k + i];
            }
        for (int i = 0; i < k; ++i)
            for (int c = 0; c < k; ++c) Mi[(size_t)i * k + c] *= dsc[i];
        sv.upload(Mi, sv.Cdev.ptr);
        sv.nn(S.ptr + k, n2, k, sv.Cdev.ptr, k, Tmp.ptr, k, 1.0, 0.0);
        launch_pdl("k_copy_cols", k_copy_cols, sv.grid(dim * k), 256, 0, s, dim, k, Tmp.ptr, k, S.ptr + k, n2);
        apply_cols(k, k);
        if (!rayleigh_ritz(n2)) break;
    }
    residuals();
    launch_pdl("k_copy_cols", k_copy_cols, sv.grid(dim * k), 256, 0, s, dim, k, S.ptr, n2, X, k);
    CI_CUDA(cudaStreamSynchronize(s));
    for (int v = 0; v < k; ++v) {
        evals[v] = theta[v];
        if (resid) resid[v] = rn[v];
    }
}

}  // namespace ci

extern "C" ci_status ci_lowest_eigs(const ci_matrix *m, const ci_eig_opts *opts, double *evals, double *evecs,
                                    ci_eig_info *info, void *stream) {
    return ci::guard([&] {
        if (!m) ci::fail(CI_ERR_INVALID_ARG, "matrix is NULL");
        ci::StreamScope scope(reinterpret_cast<cudaStream_t>(stream));
        ci::lowest_eigs(&m->impl, opts, evals, evecs, info, reinterpret_cast<cudaStream_t>(stream));
    });
}

extern "C" ci_status ci_lowest_eigs_lobpcg(const ci_matrix *m, const ci_eig_opts *opts, const int32_t *row_block,
                                           int64_t nblocks, double *evals, double *evecs, ci_eig_info *info,
                                           void *stream) {
    return ci::guard([&] {
        if (!m) ci::fail(CI_ERR_INVALID_ARG, "matrix is NULL");
        ci::StreamScope scope(reinterpret_cast<cudaStream_t>(stream));
        ci::lowest_eigs_lobpcg(&m->impl, opts, row_block, nblocks, evals, evecs, info, reinterpret_cast<cudaStream_t>(stream));
    });
}

extern "C" ci_status ci_refine_eigs(ci_problem *p, int32_t k, int32_t iters, double *evecs, double *evals,
                                    double *residuals, void *stream) {
    return ci::guard([&] {
        if (!p) ci::fail(CI_ERR_INVALID_ARG, "problem is NULL");
        cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
        ci::StreamScope scope(s);
        ci::refine_eigs(&p->impl, k, iters, evecs, evals, residuals, s);
    });
}

// Sec. 2, Fig. 1 eigensolve: the reorthogonalisation products of the block
// Lanczos solver, exposed for testing and for callers with their own basis.
extern "C" ci_status ci_basis_product(int32_t op, int32_t method, int64_t n, const double *A, int32_t lda,
                                      int32_t na, double *B, int32_t ldb, int32_t nb, double *C, double alpha,
                                      double beta, void *stream) {
    return ci::guard([&] {
        using namespace ci;
        cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
        StreamScope scope(s);
        if (op != CI_PRODUCT_TN && op != CI_PRODUCT_NN) fail(CI_ERR_INVALID_ARG, "op must be CI_PRODUCT_TN or _NN");
        if (method != CI_PRODUCT_FP64 && method != CI_PRODUCT_TC) fail(CI_ERR_INVALID_ARG, "unknown method %d", method);
        if (n < 0 || !A || !B || !C) fail(CI_ERR_INVALID_ARG, "n >= 0 and A, B, C are required");
        if (na < 1 || na > kMaxNa || nb < 1 || nb > 8 || lda < na || ldb < nb)
            fail(CI_ERR_INVALID_ARG, "need 1 <= na <= %d, 1 <= nb <= 8, lda >= na, ldb >= nb", kMaxNa);
        if (method == CI_PRODUCT_TC && (nb != 8 || !oz_supported(na)))
            fail(CI_ERR_INVALID_ARG, "the tensor-core product needs nb = 8 and na <= 64");
        DevBuf<int> flag(1);
        CI_CUDA(cudaMemsetAsync(flag.ptr, 0, sizeof(int), s));
        DevBuf<unsigned long long> Y;
        const int ldy = (na + 1) & ~1;
        if (method == CI_PRODUCT_TC && n > 0) {   // the fixed-point shadow of A
            Y.alloc((size_t)n * ldy);
            oz_fix(n, na, A, lda, Y.ptr, ldy, flag.ptr, s);
        }
        if (op == CI_PRODUCT_TN) {
            if (n == 0) {
                CI_CUDA(cudaMemsetAsync(C, 0, sizeof(double) * na * nb, s));
            } else {
                const int nblk = method == CI_PRODUCT_TC ? oz_tn_blocks(n)
                                                         : (int)std::min<int64_t>(2 * sm_count(), (n + 63) / 64);
                DevBuf<double> part((size_t)nblk * na * nb), Bc;
                const double *Bt = B;
                int ldbt = ldb;
                if (method == CI_PRODUCT_TC && (ldb & 1)) {   // the tensor copies want an even row stride
                    Bc.alloc((size_t)n * 8);
                    launch_pdl("k_copy_cols", k_copy_cols, grid_for((int64_t)n * 8, 256, sm_count() * 8), 256, 0, s,
                           (int64_t)n, 8, B, ldb, Bc.ptr, 8);
                    Bt = Bc.ptr;
                    ldbt = 8;
                }
                if (method == CI_PRODUCT_TC) oz_tn(n, Y.ptr, ldy, na, Bt, ldbt, part.ptr, nblk, flag.ptr, s);
                else fp64_tn(n, A, lda, na, B, ldb, nb, part.ptr, nblk, (n + nblk - 1) / nblk, s);
                launch_pdl("k_reduce_partial", k_reduce_partial, (na * nb + 7) / 8, 256, 0, s, part.ptr, nblk, na * nb, C);
            }
        } else if (n > 0) {
            if (method == CI_PRODUCT_TC) oz_nn(n, Y.ptr, ldy, na, C, B, ldb, alpha, beta, flag.ptr, s);
            else fp64_nn(n, A, lda, na, C, nb, B, ldb, alpha, beta, s);
        }
        int f = 0;
        CI_CUDA(cudaMemcpyAsync(&f, flag.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
        CI_CUDA(cudaStreamSynchronize(s));
        if (f & 1) fail(CI_ERR_INVALID_ARG, "an entry of A (or a non-finite value) is outside the digits' range");
        if (f & 2) fail(CI_ERR_TIMEOUT, "a tensor-core wait ran out");
    });
}
