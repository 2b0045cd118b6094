// Batched block Lanczos with device-side control (see engine.cuh).
//
// One step of every running slot, in launch order:
//   X = float(Q[:, j0:j0+8]);  W = H X                       (prepx, spmm)
//   W -= Q[:, lo:m] (Q[:, lo:m]^T W)   lo = the two newest blocks  (tn, reduce, nn)
//   W -= Q[:, 0:m] (Q[:, 0:m]^T W)     one full FP64 pass           (tn, reduce, nn)
//   T[:, j0 block] = the projection coefficients                     (tupdate)
//   block QR of W into Q[:, m:m+8]: Gram matrix, 8x8 eigensolve with
//   rank test, random completion of deflated directions, second pass
//   (tn, reduce, qr1, nn, rand, tn, reduce, nn, tn, reduce, qr2, nn)
//   advance the basis; Ritz check with an FP64 Jacobi eigensolver of T
//   where due; thick restart of full bases (advance, ritz, restart)
// Every kernel reads the slot's state and skips slots it does not concern.
#include <algorithm>
#include <cmath>

#include <map>
#include <mutex>

#include "engine.cuh"

namespace ci {

enum Phase { PH_STEP = 0, PH_INIT = 1, PH_FINAL = 2 };
enum Mode { M_LOC = 0, M_FULL = 1, M_GRAM = 2, M_GRAMV = 3, M_RAND = 4, M_RESID = 5, M_QR1 = 6, M_QR2 = 7,
            M_RITZ = 8 };

__device__ __forceinline__ bool eligible(const SlotDev &s, int phase) {
    if (phase == PH_STEP) return s.state == S_RUN;
    if (phase == PH_INIT) return s.state == S_INIT;
    return (s.state == S_CONV || s.state == S_FAIL) && !(s.flags & F_FINAL);
}

// Operand description of an A^T B product for a slot and mode.
struct TnOps {
    const double *A;
    int lda, na;
    const double *B;
    int ldb, nb;
};

__device__ __forceinline__ bool tn_ops(const SlotDev &s, int mode, int MB, TnOps &o) {
    switch (mode) {
        case M_LOC: {
            const int lo = max(0, s.j0 - EB);
            o = {s.Q + lo, MB, s.m_cur - lo, s.W, EB, EB};
            return o.na > 0;
        }
        case M_FULL: o = {s.Q, MB, s.m_cur, s.W, EB, EB}; return s.m_cur > 0;
        case M_GRAM: o = {s.W, EB, EB, s.W, EB, EB}; return true;
        case M_GRAMV: o = {s.Q + s.m_cur, MB, EB, s.Q + s.m_cur, MB, EB}; return true;
        case M_RAND:
            o = {s.Q, MB, s.m_cur + s.rank, s.Q + s.m_cur + s.rank, MB, EB - s.rank};
            return s.rank < EB && o.na > 0;
        case M_RESID: o = {s.W, EB, EB, s.W, EB, EB}; return true;
    }
    return false;
}

struct DensePtrs {
    double *T, *S, *theta, *Cl, *Cf, *Cr, *G, *M, *R, *res, *evals, *tres;
};

// ---------------------------------------------------------------- row kernels

// X[r][v] = float(Q[r][j0 + v])   (step)   or   float(W[r][v])   (final)
__global__ void __launch_bounds__(256) k_e_prepx(SlotDev *slots, const Tile *tiles, const int32_t *ntiles, int MB,
                                                 int phase) {
    for (int t = blockIdx.x; t < *ntiles; t += gridDim.x) {
        const Tile tl = tiles[t];
        const SlotDev &s = slots[tl.slot];
        if (!eligible(s, phase)) continue;
        for (int e = threadIdx.x; e < tl.nr * EB; e += blockDim.x) {
            const int64_t r = tl.r0 + e / EB;
            const int v = e % EB;
            s.X[r * EB + v] = phase == PH_FINAL ? (float)s.W[r * EB + v] : (float)s.Q[r * MB + s.j0 + v];
        }
    }
}

// W = H X (step) or Y = H X (final), two lanes per nonzero (half rows of X)
__global__ void __launch_bounds__(256) k_e_spmm(SlotDev *slots, const Tile *tiles, const int32_t *ntiles, int phase) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, half = lane & 1, pair = lane >> 1;
    for (int t = blockIdx.x; t < *ntiles; t += gridDim.x) {
        const Tile tl = tiles[t];
        const SlotDev &s = slots[tl.slot];
        if (!eligible(s, phase)) continue;
        const float4 *X4 = reinterpret_cast<const float4 *>(s.X);
        for (int rr = wid; rr < tl.nr; rr += 8) {
            const int64_t r = tl.r0 + rr;
            float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
            const int64_t e1 = s.rp[r + 1];
            int64_t e = s.rp[r] + pair;
            constexpr int U = 4;   // nonzeros in flight per lane pair
            for (; e + 16 * (U - 1) < e1; e += 16 * U) {
                int c[U];
                float v[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    c[u] = __ldcs(s.col + e + 16 * u);
                    v[u] = __ldcs(s.val + e + 16 * u);
                }
                float4 x[U];
#pragma unroll
                for (int u = 0; u < U; ++u) x[u] = __ldg(X4 + (int64_t)c[u] * 2 + half);
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    a0 = fmaf(v[u], x[u].x, a0); a1 = fmaf(v[u], x[u].y, a1);
                    a2 = fmaf(v[u], x[u].z, a2); a3 = fmaf(v[u], x[u].w, a3);
                }
            }
            for (; e < e1; e += 16) {
                const int c = __ldcs(s.col + e);
                const float v = __ldcs(s.val + e);
                const float4 x = __ldg(X4 + (int64_t)c * 2 + half);
                a0 = fmaf(v, x.x, a0); a1 = fmaf(v, x.y, a1); a2 = fmaf(v, x.z, a2); a3 = fmaf(v, x.w, a3);
            }
#pragma unroll
            for (int o = 16; o > 1; o >>= 1) {
                a0 += __shfl_xor_sync(0xffffffffu, a0, o);
                a1 += __shfl_xor_sync(0xffffffffu, a1, o);
                a2 += __shfl_xor_sync(0xffffffffu, a2, o);
                a3 += __shfl_xor_sync(0xffffffffu, a3, o);
            }
            if (lane < 2) {
                if (phase == PH_FINAL) {
                    reinterpret_cast<float4 *>(s.Y)[r * 2 + half] = make_float4(a0, a1, a2, a3);
                } else {
                    double *w = s.W + r * EB + 4 * half;
                    w[0] = a0; w[1] = a1; w[2] = a2; w[3] = a3;
                }
            }
        }
    }
}

// part[t][u*nb + v] = sum over the tile's rows of A[r][u] B[r][v]
constexpr int kER = 32;  // rows staged per pass
__global__ void __launch_bounds__(256) k_e_tn(SlotDev *slots, const Tile *tiles, const int32_t *ntiles, int MB,
                                              int phase, int mode, double *part) {
    extern __shared__ double sm[];
    for (int t = blockIdx.x; t < *ntiles; t += gridDim.x) {
        const Tile tl = tiles[t];
        const SlotDev &s = slots[tl.slot];
        if (!eligible(s, phase)) continue;
        TnOps o;
        if (!tn_ops(s, mode, MB, o)) continue;
        const int nout = o.na * o.nb;
        double *As = sm, *Bs = sm + kER * o.na;
        double acc[EMBMAX * EB / 256 + 1];
#pragma unroll
        for (int j = 0; j < EMBMAX * EB / 256 + 1; ++j) acc[j] = 0.0;
        for (int r0 = 0; r0 < tl.nr; r0 += kER) {
            const int rows = min(kER, tl.nr - r0);
            __syncthreads();
            for (int e = threadIdx.x; e < rows * o.na; e += blockDim.x) {
                const int r = e / o.na, u = e - r * o.na;
                As[e] = o.A[(tl.r0 + r0 + r) * o.lda + u];
            }
            for (int e = threadIdx.x; e < rows * o.nb; e += blockDim.x) {
                const int r = e / o.nb, v = e - r * o.nb;
                Bs[e] = o.B[(tl.r0 + r0 + r) * o.ldb + v];
            }
            __syncthreads();
#pragma unroll
            for (int j = 0; j < EMBMAX * EB / 256 + 1; ++j) {
                const int idx = threadIdx.x + j * 256;
                if (idx < nout) {
                    const int u = idx / o.nb, v = idx - u * o.nb;
                    double a = acc[j];
                    for (int r = 0; r < rows; ++r) a = fma(As[r * o.na + u], Bs[r * o.nb + v], a);
                    acc[j] = a;
                }
            }
        }
#pragma unroll
        for (int j = 0; j < EMBMAX * EB / 256 + 1; ++j) {
            const int idx = threadIdx.x + j * 256;
            if (idx < nout) part[(int64_t)t * MB * EB + idx] = acc[j];
        }
        __syncthreads();
    }
}

// Per-slot sum of the tile partials (deterministic order): grid (slots, chunks of 32 outputs)
__global__ void __launch_bounds__(256) k_e_reduce(SlotDev *slots, int nslots, int MB, int phase, int mode,
                                                  const double *part, DensePtrs d) {
    __shared__ double red[8][33];
    const int si = blockIdx.x;
    if (si >= nslots) return;
    const SlotDev &s = slots[si];
    if (!eligible(s, phase)) return;
    TnOps o;
    if (!tn_ops(s, mode, MB, o)) return;
    const int nout = o.na * o.nb;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int idx = blockIdx.y * 32 + lane;
    if (blockIdx.y * 32 >= nout) return;
    double acc = 0.0;
    if (idx < nout)
        for (int t = s.tile0 + w; t < s.tile1; t += 8) acc += part[(int64_t)t * MB * EB + idx];
    red[w][lane] = acc;
    __syncthreads();
    if (w == 0 && idx < nout) {
        double tot = 0.0;
#pragma unroll
        for (int i = 0; i < 8; ++i) tot += red[i][lane];
        double *dst;
        switch (mode) {
            case M_LOC: dst = d.Cl + (int64_t)si * 2 * EB * EB; break;
            case M_FULL: dst = d.Cf + (int64_t)si * MB * EB; break;
            case M_RAND: dst = d.Cr + (int64_t)si * MB * EB; break;
            default: dst = d.G + (int64_t)si * EB * EB; break;
        }
        dst[idx] = tot;
    }
}

// Row updates: LOC / FULL: W -= Q_cols C; QR1: Q[:, m:m+8] = W M; RAND:
// Q[:, m+rank:m+8] -= Q[:, 0:m+rank] Cr; QR2: V = V M (in place per row);
// RITZ: W = Q[:, 0:m_act] S[:, c0:c0+nc] (final phase).
// QR2 (the in-place 8 x 8 update) is its own instantiation: its loop-invariant
// 8 x 8 matrix lives in registers, which the other modes must not pay for.
template <bool QR2>
__global__ void __launch_bounds__(256) k_e_nn(SlotDev *slots, const Tile *tiles, const int32_t *ntiles, int MB,
                                              int phase, int mode, DensePtrs d, int c0) {
    __shared__ double Cs[EMBMAX * EB];
    for (int t = blockIdx.x; t < *ntiles; t += gridDim.x) {
        const Tile tl = tiles[t];
        const SlotDev &s = slots[tl.slot];
        __syncthreads();
        if (!eligible(s, phase)) continue;
        const int si = tl.slot;
        const double *C;
        int na, nb, a0 = 0;
        const double *A;
        int lda;
        switch (mode) {
            case M_LOC: a0 = max(0, s.j0 - EB); na = s.m_cur - a0; nb = EB; C = d.Cl + (int64_t)si * 2 * EB * EB;
                A = s.Q + a0; lda = MB; break;
            case M_FULL: na = s.m_cur; nb = EB; C = d.Cf + (int64_t)si * MB * EB; A = s.Q; lda = MB; break;
            case M_QR1: na = EB; nb = EB; C = d.M + (int64_t)si * EB * EB; A = s.W; lda = EB; break;
            case M_RAND:
                if (s.rank >= EB) continue;
                na = s.m_cur + s.rank; nb = EB - s.rank; C = d.Cr + (int64_t)si * MB * EB; A = s.Q; lda = MB; break;
            case M_QR2: na = EB; nb = EB; C = d.M + (int64_t)si * EB * EB; A = s.Q + s.m_cur; lda = MB; break;
            default: {  // M_RITZ
                na = s.m_act; nb = min(EB, s.k - c0);
                if (nb <= 0) continue;
                C = nullptr; A = s.Q; lda = MB;
            }
        }
        if (na <= 0) continue;
        if (mode == M_RITZ) {
            const double *Sm = d.S + (int64_t)si * MB * MB;
            for (int e = threadIdx.x; e < na * nb; e += blockDim.x) Cs[e] = Sm[(e / nb) * MB + c0 + e % nb];
        } else {
            for (int e = threadIdx.x; e < na * nb; e += blockDim.x) Cs[e] = C[e];
        }
        __syncthreads();
        if (QR2) {  // in place: each thread owns a whole row
            for (int rr = threadIdx.x; rr < tl.nr; rr += blockDim.x) {
                double *row = s.Q + (tl.r0 + rr) * MB + s.m_cur;
                double x[EB], y[EB];
#pragma unroll
                for (int u = 0; u < EB; ++u) x[u] = row[u];
#pragma unroll
                for (int v = 0; v < EB; ++v) {
                    double a = 0.0;
#pragma unroll
                    for (int u = 0; u < EB; ++u) a = fma(x[u], Cs[u * EB + v], a);
                    y[v] = a;
                }
#pragma unroll
                for (int v = 0; v < EB; ++v) row[v] = y[v];
            }
            continue;
        }
        if (nb == EB) {  // one row per thread, 8 accumulators, C broadcast from shared memory
            double *dst;     // row r of the output starts at dst + r * ldd
            int ldd;
            bool sub;        // subtract from it (projections) or overwrite
            switch (mode) {
                case M_LOC:
                case M_FULL: dst = s.W; ldd = EB; sub = true; break;
                case M_QR1: dst = s.Q + s.m_cur; ldd = MB; sub = false; break;
                case M_RAND: dst = s.Q + s.m_cur + s.rank; ldd = MB; sub = true; break;
                default: dst = s.W; ldd = EB; sub = false; break;  // M_RITZ
            }
            for (int rr = threadIdx.x; rr < tl.nr; rr += blockDim.x) {
                const int64_t r = tl.r0 + rr;
                const double *Ar = A + r * lda;
                double acc[EB];
#pragma unroll
                for (int v = 0; v < EB; ++v) acc[v] = 0.0;
#pragma unroll 2
                for (int u = 0; u < na; ++u) {
                    const double av = Ar[u];
#pragma unroll
                    for (int v = 0; v < EB; ++v) acc[v] = fma(av, Cs[u * EB + v], acc[v]);
                }
                double *w = dst + r * ldd;
#pragma unroll
                for (int v = 0; v < EB; ++v) w[v] = sub ? w[v] - acc[v] : acc[v];
            }
            continue;
        }
        for (int e = threadIdx.x; e < tl.nr * nb; e += blockDim.x) {
            const int64_t r = tl.r0 + e / nb;
            const int v = e % nb;
            const double *Ar = A + r * lda;
            double a = 0.0;
            for (int u = 0; u < na; ++u) a = fma(Ar[u], Cs[u * nb + v], a);
            switch (mode) {
                case M_LOC:
                case M_FULL: s.W[r * EB + v] -= a; break;
                case M_QR1: s.Q[r * MB + s.m_cur + v] = a; break;
                case M_RAND: s.Q[r * MB + s.m_cur + s.rank + v] -= a; break;
                default: s.W[r * EB + v] = a; break;  // M_RITZ
            }
        }
    }
}

__device__ __forceinline__ double rand_pm1(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

// Random start block into W (init) or random completion columns
// Q[:, m+rank:m+8] of rank-deficient slots (step / init).
__global__ void __launch_bounds__(256) k_e_rand(SlotDev *slots, const Tile *tiles, const int32_t *ntiles, int MB,
                                                int phase, int into_w) {
    for (int t = blockIdx.x; t < *ntiles; t += gridDim.x) {
        const Tile tl = tiles[t];
        const SlotDev &s = slots[tl.slot];
        if (!eligible(s, phase)) continue;
        if (into_w) {
            for (int e = threadIdx.x; e < tl.nr * EB; e += blockDim.x) {
                const int64_t r = tl.r0 + e / EB;
                const int v = e % EB;
                s.W[r * EB + v] = rand_pm1(s.seed, (uint64_t)r * EB + v);
            }
        } else {
            if (s.rank >= EB) continue;
            const int nb = EB - s.rank;
            const uint64_t sd = s.seed ^ (0x5851F42D4C957F2Dull * (uint64_t)(s.it + 1));
            for (int e = threadIdx.x; e < tl.nr * nb; e += blockDim.x) {
                const int64_t r = tl.r0 + e / nb;
                const int v = e % nb;
                s.Q[r * MB + s.m_cur + s.rank + v] = rand_pm1(sd, (uint64_t)r * EB + v);
            }
        }
    }
}

// Residual block of finished slots: W = Y - W diag(theta[c0:c0+nc])
__global__ void __launch_bounds__(256) k_e_resid(SlotDev *slots, const Tile *tiles, const int32_t *ntiles, DensePtrs d,
                                                 int MB, int c0) {
    for (int t = blockIdx.x; t < *ntiles; t += gridDim.x) {
        const Tile tl = tiles[t];
        const SlotDev &s = slots[tl.slot];
        if (!eligible(s, PH_FINAL)) continue;
        const int nb = min(EB, s.k - c0);
        for (int e = threadIdx.x; e < tl.nr * EB; e += blockDim.x) {
            const int64_t r = tl.r0 + e / EB;
            const int v = e % EB;
            const double th = v < nb ? d.theta[(int64_t)tl.slot * MB + c0 + v] : 0.0;
            s.W[r * EB + v] = v < nb ? (double)s.Y[r * EB + v] - th * s.W[r * EB + v] : 0.0;
        }
    }
}

// ---------------------------------------------------------------- small dense (per slot)

// Cyclic Jacobi eigen-decomposition of a symmetric n x n matrix (n <= 8)
// by one thread: A is destroyed, w ascending, U columns.
__device__ void jacobi_small(double *A, int n, double *w, double *U) {
    for (int i = 0; i < n * n; ++i) U[i] = (i / n == i % n) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 30; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                tot += A[i * n + j] * A[i * n + j];
                if (i != j) off += A[i * n + j] * A[i * n + j];
            }
        if (off <= 1e-32 * tot || off == 0.0) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = A[p * n + q];
                if (apq == 0.0) continue;
                const double tau = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
                const double tt = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                const double c = 1.0 / sqrt(1.0 + tt * tt), sn = tt * c;
                for (int j = 0; j < n; ++j) {  // rows p, q
                    const double ap = A[p * n + j], aq = A[q * n + j];
                    A[p * n + j] = c * ap - sn * aq;
                    A[q * n + j] = sn * ap + c * aq;
                }
                for (int i = 0; i < n; ++i) {  // columns p, q
                    const double ap = A[i * n + p], aq = A[i * n + q];
                    A[i * n + p] = c * ap - sn * aq;
                    A[i * n + q] = sn * ap + c * aq;
                    const double up = U[i * n + p], uq = U[i * n + q];
                    U[i * n + p] = c * up - sn * uq;
                    U[i * n + q] = sn * up + c * uq;
                }
            }
    }
    for (int i = 0; i < n; ++i) w[i] = A[i * n + i];
    for (int i = 0; i < n; ++i)  // selection sort ascending, columns with it
        for (int j = i + 1; j < n; ++j)
            if (w[j] < w[i]) {
                double x = w[i]; w[i] = w[j]; w[j] = x;
                for (int r = 0; r < n; ++r) {
                    double y = U[r * n + i]; U[r * n + i] = U[r * n + j]; U[r * n + j] = y;
                }
            }
}

// Cholesky factor of a symmetric 8 x 8 matrix (lower, row-major).  Returns
// false when a pivot falls below rel * the matching diagonal entry (the
// block is too ill-conditioned for a Cholesky QR).
__device__ bool chol8(const double *G, double *L, double rel) {
    for (int i = 0; i < EB * EB; ++i) L[i] = 0.0;
    for (int j = 0; j < EB; ++j) {
        double d = G[j * EB + j];
        for (int k = 0; k < j; ++k) d -= L[j * EB + k] * L[j * EB + k];
        if (!(d > rel * G[j * EB + j]) || !(d > 0.0)) return false;
        const double ljj = sqrt(d);
        L[j * EB + j] = ljj;
        for (int i = j + 1; i < EB; ++i) {
            double x = G[i * EB + j];
            for (int k = 0; k < j; ++k) x -= L[i * EB + k] * L[j * EB + k];
            L[i * EB + j] = x / ljj;
        }
    }
    return true;
}

// Inverse of the upper triangular R = L^T: M = R^-1 (upper), row-major.
__device__ void inv_upper_from_lower(const double *L, double *M) {
    for (int i = 0; i < EB * EB; ++i) M[i] = 0.0;
    for (int j = EB - 1; j >= 0; --j) {  // column j of R^-1 by back substitution
        M[j * EB + j] = 1.0 / L[j * EB + j];
        for (int i = j - 1; i >= 0; --i) {
            double x = 0.0;
            for (int k = i + 1; k <= j; ++k) x += L[k * EB + i] * M[k * EB + j];  // R[i][k] = L[k][i]
            M[i * EB + j] = -x / L[i * EB + i];
        }
    }
}

// qr1: W = V R.  Cholesky QR (G = W^T W = R^T R, M = R^-1, rank 8) when the
// Gram matrix is well conditioned; otherwise the eigen-decomposition of G
// decides the rank: M = U_k L_k^-1/2 on the kept directions (largest first),
// R = L_k^1/2 U_k^T, and the remaining columns are completed at random.
// qr2: G2 = V^T V ~ I, Cholesky G2 = R2^T R2, M = R2^-1, R <- R2 R.
__global__ void k_e_small(SlotDev *slots, int nslots, int phase, int which, DensePtrs d) {
    const int si = blockIdx.x * blockDim.x + threadIdx.x;
    if (si >= nslots) return;
    SlotDev &s = slots[si];
    if (!eligible(s, phase)) return;
    double A[EB * EB], L[EB * EB];
    const double *G = d.G + (int64_t)si * EB * EB;
    for (int i = 0; i < EB * EB; ++i) A[i] = 0.5 * (G[i] + G[(i % EB) * EB + i / EB]);
    double *M = d.M + (int64_t)si * EB * EB, *R = d.R + (int64_t)si * EB * EB;
    if (which == 1) {
        if (chol8(A, L, 1e-12)) {
            inv_upper_from_lower(L, M);
            for (int r = 0; r < EB; ++r)
                for (int c = 0; c < EB; ++c) R[r * EB + c] = c >= r ? L[c * EB + r] : 0.0;
            s.rank = EB;
            return;
        }
        double U[EB * EB], w[EB];
        jacobi_small(A, EB, w, U);
        const double lmax = fmax(w[EB - 1], 0.0);
        const double scale = fmax(s.hnorm, sqrt(lmax));
        const double thr = 1e-20 * scale * scale + 1e-300;
        for (int i = 0; i < EB * EB; ++i) { M[i] = 0.0; R[i] = 0.0; }
        int r = 0;
        for (int i = EB - 1; i >= 0; --i) {
            if (w[i] <= thr) break;
            const double sq = sqrt(w[i]);
            for (int a = 0; a < EB; ++a) {
                M[a * EB + r] = U[a * EB + i] / sq;
                R[r * EB + a] = U[a * EB + i] * sq;
            }
            ++r;
        }
        s.rank = r;
    } else {
        // V^T V is the identity up to rounding (and to the completed columns
        // scale), so its Cholesky factor exists
        if (!chol8(A, L, 1e-30)) {
            for (int i = 0; i < EB * EB; ++i) L[i] = (i / EB == i % EB) ? sqrt(fmax(A[i], 1e-300)) : 0.0;
        }
        inv_upper_from_lower(L, M);
        double R2[EB * EB];
        for (int r = 0; r < EB; ++r)
            for (int c = 0; c < EB; ++c) {
                double x = 0.0;
                for (int k = r; k < EB; ++k) x += L[k * EB + r] * R[k * EB + c];  // R2 = L^T R
                R2[r * EB + c] = x;
            }
        for (int i = 0; i < EB * EB; ++i) R[i] = R2[i];
    }
}

// T[:, j0 block] (and its transpose) from the projection coefficients
__global__ void k_e_tupdate(SlotDev *slots, int nslots, int MB, DensePtrs d) {
    const int si = blockIdx.x;
    if (si >= nslots) return;
    const SlotDev &s = slots[si];
    if (!eligible(s, PH_STEP)) return;
    double *T = d.T + (int64_t)si * MB * MB;
    const double *Cl = d.Cl + (int64_t)si * 2 * EB * EB, *Cf = d.Cf + (int64_t)si * MB * EB;
    const int lo = max(0, s.j0 - EB), j0 = s.j0;
    for (int e = threadIdx.x; e < s.m_cur * EB; e += blockDim.x) {
        const int i = e / EB, v = e % EB;
        double c = Cf[i * EB + v] + ((i >= lo) ? Cl[(i - lo) * EB + v] : 0.0);
        if (i >= j0) {  // diagonal block, symmetrised
            const int u = i - j0;
            const double ct = Cf[(j0 + v) * EB + u] + ((j0 + v >= lo) ? Cl[(j0 + v - lo) * EB + u] : 0.0);
            c = 0.5 * (c + ct);
            T[i * MB + j0 + v] = c;
        } else {
            T[i * MB + j0 + v] = c;
            T[(j0 + v) * MB + i] = c;
        }
    }
}

// Advance the basis after a step (or finish the start block of new slots).
__global__ void k_e_advance(SlotDev *slots, int nslots, int MB, int phase, DensePtrs d) {
    const int si = blockIdx.x * blockDim.x + threadIdx.x;
    if (si >= nslots) return;
    SlotDev &s = slots[si];
    if (!eligible(s, phase)) return;
    if (phase == PH_INIT) {
        s.m_cur = EB;
        s.j0 = 0;
        s.m_act = 0;
        s.it = 0;
        s.flags = 0;
        s.state = S_RUN;
        return;
    }
    double *T = d.T + (int64_t)si * MB * MB;
    const double *R = d.R + (int64_t)si * EB * EB;
    for (int r = 0; r < EB; ++r)
        for (int c = 0; c < EB; ++c) {
            T[(s.m_cur + r) * MB + s.j0 + c] = R[r * EB + c];
            T[(s.j0 + c) * MB + s.m_cur + r] = R[r * EB + c];
        }
    s.m_act = s.m_cur;
    s.j0 = s.m_cur;
    s.m_cur += EB;
    s.it += 1;
    s.flags = 0;
    if (s.it % s.check_every == 0 || s.m_cur + EB > MB || s.it >= s.max_iter) s.flags |= F_CHECK;
}

// Ritz analysis of T[0:m_act, 0:m_act] by parallel (round-robin) Jacobi in
// FP64, one block per slot: theta ascending, S columns, residual estimates
// ||R S[m-8:m, i]||, convergence and restart decisions.
__global__ void __launch_bounds__(256) k_e_ritz(SlotDev *slots, int nslots, int MB, DensePtrs d) {
    extern __shared__ double sm[];
    const int si = blockIdx.x;
    if (si >= nslots) return;
    SlotDev &s = slots[si];
    if (!eligible(s, PH_STEP) || !(s.flags & F_CHECK)) return;
    const int m = s.m_act;  // even (restarts keep an even number of vectors)
    double *A = sm, *V = sm + m * m;
    double *cs = V + m * m, *sn = cs + m / 2, *red = sn + m / 2;
    int *pp = (int *)(red + 64), *qq = pp + m / 2, *rank = qq + m / 2;
    const double *T = d.T + (int64_t)si * MB * MB;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        const int i = e / m, j = e % m;
        A[e] = 0.5 * (T[i * MB + j] + T[j * MB + i]);
        V[e] = i == j ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int sweep = 0; sweep < 40; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
            const double x = A[e] * A[e];
            tot += x;
            if (e / m != e % m) off += x;
        }
        for (int o = 16; o > 0; o >>= 1) {
            off += __shfl_xor_sync(0xffffffffu, off, o);
            tot += __shfl_xor_sync(0xffffffffu, tot, o);
        }
        if ((threadIdx.x & 31) == 0) { red[threadIdx.x >> 5] = off; red[32 + (threadIdx.x >> 5)] = tot; }
        __syncthreads();
        double offs = 0.0, tots = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { offs += red[i]; tots += red[32 + i]; }
        __syncthreads();
        if (offs <= 1e-30 * tots || offs == 0.0) break;
        for (int round = 0; round < m - 1; ++round) {
            for (int k = threadIdx.x; k < m / 2; k += blockDim.x) {
                const int pk = k == 0 ? 0 : ((k - 1 + round) % (m - 1)) + 1;
                const int qk = ((m - 1 - k - 1 + round) % (m - 1)) + 1;
                const int p = min(pk, qk), q = max(pk, qk);
                const double apq = A[p * m + q];
                double c = 1.0, sv = 0.0;
                if (apq != 0.0) {
                    const double tau = (A[q * m + q] - A[p * m + p]) / (2.0 * apq);
                    const double tt = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                    c = 1.0 / sqrt(1.0 + tt * tt);
                    sv = tt * c;
                }
                pp[k] = p; qq[k] = q; cs[k] = c; sn[k] = sv;
            }
            __syncthreads();
            for (int e = threadIdx.x; e < (m / 2) * m; e += blockDim.x) {  // rows
                const int k = e / m, j = e % m;
                const int p = pp[k], q = qq[k];
                const double ap = A[p * m + j], aq = A[q * m + j];
                A[p * m + j] = cs[k] * ap - sn[k] * aq;
                A[q * m + j] = sn[k] * ap + cs[k] * aq;
            }
            __syncthreads();
            for (int e = threadIdx.x; e < (m / 2) * m; e += blockDim.x) {  // columns of A and V
                const int k = e / m, i = e % m;
                const int p = pp[k], q = qq[k];
                const double ap = A[i * m + p], aq = A[i * m + q];
                A[i * m + p] = cs[k] * ap - sn[k] * aq;
                A[i * m + q] = sn[k] * ap + cs[k] * aq;
                const double vp = V[i * m + p], vq = V[i * m + q];
                V[i * m + p] = cs[k] * vp - sn[k] * vq;
                V[i * m + q] = sn[k] * vp + cs[k] * vq;
            }
            __syncthreads();
        }
    }
    // ascending order: rank of each diagonal entry (ties by index)
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const double wi = A[i * m + i];
        int r = 0;
        for (int j = 0; j < m; ++j) {
            const double wj = A[j * m + j];
            if (wj < wi || (wj == wi && j < i)) ++r;
        }
        rank[i] = r;
    }
    __syncthreads();
    double *theta = d.theta + (int64_t)si * MB, *S = d.S + (int64_t)si * MB * MB;
    for (int i = threadIdx.x; i < m; i += blockDim.x) theta[rank[i]] = A[i * m + i];
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        const int r = e / m, c = e % m;
        S[r * MB + rank[c]] = V[e];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double *R = d.R + (int64_t)si * EB * EB;
        double h = s.hnorm;
        h = fmax(h, fabs(theta[0]));
        h = fmax(h, fabs(theta[m - 1]));
        s.hnorm = h;
        bool conv = true;
        for (int i = 0; i < s.k; ++i) {
            double ss = 0.0;
            for (int r = 0; r < EB; ++r) {
                double x = 0.0;
                for (int c = 0; c < EB; ++c) x += R[r * EB + c] * S[(m - EB + c) * MB + i];
                ss += x * x;
            }
            const double ri = sqrt(ss);
            d.res[(int64_t)si * EKMAX + i] = ri;
            d.evals[(int64_t)si * EKMAX + i] = theta[i];
            if (ri > s.tol * h) conv = false;
        }
        if (conv) s.state = S_CONV;
        else if (s.it >= s.max_iter) s.state = S_FAIL;
        else if (s.m_cur + EB > MB) s.flags |= F_RESTART;
    }
}

// Thick restart, rows: Q[r][0:keep] = Q[r][0:m_act] S[:, 0:keep] and the
// newest block moved to Q[r][keep:keep+8]; one warp per row, in place.
__global__ void __launch_bounds__(256) k_e_restart_rows(SlotDev *slots, const Tile *tiles, const int32_t *ntiles,
                                                        int MB, DensePtrs d) {
    extern __shared__ double sm[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int t = blockIdx.x; t < *ntiles; t += gridDim.x) {
        const Tile tl = tiles[t];
        const SlotDev &s = slots[tl.slot];
        __syncthreads();
        if (!eligible(s, PH_STEP) || !(s.flags & F_RESTART)) continue;
        const int m = s.m_act, keep = (m / 2) & ~1;  // even: the Jacobi pairs indices
        double *Ss = sm;                 // [m][keep]
        double *rowbuf = sm + m * keep;  // [8 warps][MB]
        const double *S = d.S + (int64_t)tl.slot * MB * MB;
        for (int e = threadIdx.x; e < m * keep; e += blockDim.x) Ss[e] = S[(e / keep) * MB + e % keep];
        __syncthreads();
        double *rb = rowbuf + wid * MB;
        for (int rr = wid; rr < tl.nr; rr += 8) {
            double *row = s.Q + (tl.r0 + rr) * MB;
            for (int u = lane; u < m + EB; u += 32) rb[u] = row[u];
            __syncwarp();
            for (int j = lane; j < keep; j += 32) {
                double a = 0.0;
                for (int u = 0; u < m; ++u) a = fma(rb[u], Ss[u * keep + j], a);
                row[j] = a;
            }
            for (int v = lane; v < EB; v += 32) row[keep + v] = rb[m + v];
            __syncwarp();
        }
    }
}

// Thick restart, projected matrix: diag(theta[0:keep]) and the coupling of
// the newest block to the kept Ritz vectors, R S[m-8:m, 0:keep].
__global__ void k_e_restart_slot(SlotDev *slots, int nslots, int MB, DensePtrs d) {
    const int si = blockIdx.x;
    if (si >= nslots) return;
    SlotDev &s = slots[si];
    if (!eligible(s, PH_STEP) || !(s.flags & F_RESTART)) return;
    const int m = s.m_act, keep = (m / 2) & ~1;  // even: the Jacobi pairs indices
    double *T = d.T + (int64_t)si * MB * MB;
    const double *S = d.S + (int64_t)si * MB * MB, *R = d.R + (int64_t)si * EB * EB;
    const double *theta = d.theta + (int64_t)si * MB;
    for (int e = threadIdx.x; e < MB * MB; e += blockDim.x) T[e] = 0.0;
    __syncthreads();
    for (int i = threadIdx.x; i < keep; i += blockDim.x) T[i * MB + i] = theta[i];
    for (int e = threadIdx.x; e < EB * keep; e += blockDim.x) {
        const int r = e / keep, i = e % keep;
        double x = 0.0;
        for (int c = 0; c < EB; ++c) x += R[r * EB + c] * S[(m - EB + c) * MB + i];
        T[(keep + r) * MB + i] = x;
        T[i * MB + keep + r] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        s.m_cur = keep + EB;
        s.j0 = keep;
        s.restarts += 1;
        s.flags = 0;
    }
}

__global__ void k_e_count(SlotDev *slots, int nslots, int32_t *counters) {
    int c = 0;
    for (int i = threadIdx.x; i < nslots; i += blockDim.x) c += (slots[i].state == S_RUN || slots[i].state == S_INIT);
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    __shared__ int red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
        counters[0] = t;
    }
}

__global__ void k_e_mark_final(SlotDev *slots, int nslots, DensePtrs d, int MB) {
    const int si = blockIdx.x * blockDim.x + threadIdx.x;
    if (si >= nslots) return;
    SlotDev &s = slots[si];
    if (!eligible(s, PH_FINAL)) return;
    s.flags |= F_FINAL;
}

// tres[c0 + v] = sqrt(G[v][v]) of the residual Gram matrix
__global__ void k_e_store_resid(SlotDev *slots, int nslots, DensePtrs d, int c0) {
    const int si = blockIdx.x * blockDim.x + threadIdx.x;
    if (si >= nslots) return;
    const SlotDev &s = slots[si];
    if (!eligible(s, PH_FINAL)) return;
    const double *G = d.G + (int64_t)si * EB * EB;
    for (int v = 0; v < EB && c0 + v < s.k; ++v) d.tres[(int64_t)si * EKMAX + c0 + v] = sqrt(fmax(G[v * EB + v], 0.0));
}

// ---------------------------------------------------------------- host side

static DensePtrs dense_ptrs(Engine *e) {
    EngineDense &n = e->dn;
    return DensePtrs{n.T.ptr, n.S.ptr, n.theta.ptr, n.Cl.ptr, n.Cf.ptr, n.Cr.ptr, n.G.ptr,
                     n.M.ptr, n.R.ptr, n.res.ptr, n.evals.ptr, n.tres.ptr};
}

Engine::~Engine() {
    HandleRelease hr;
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (pinned_counter) cudaFreeHost(pinned_counter);
    slots.release(); tiles.release(); ntiles.release(); counters.release(); part.release();
    for (DevBuf<double> *b : {&dn.T, &dn.S, &dn.theta, &dn.Cl, &dn.Cf, &dn.Cr, &dn.G, &dn.M, &dn.R, &dn.res,
                              &dn.evals, &dn.tres})
        b->release();
    if (stream) cudaStreamDestroy(stream);
}

static int tile_grid(const Engine *e) { return sm_count() * e->tile_mult; }

static size_t tn_smem(int MB) { return sizeof(double) * kER * (MB + EB); }
static size_t ritz_smem(int MB) {
    const int m = MB - EB;
    return sizeof(double) * (2 * m * m + m + 64) + sizeof(int) * (2 * m);
}
static size_t restart_smem(int MB) {
    const int m = MB - EB;
    return sizeof(double) * ((size_t)m * (m / 2) + 8 * MB);
}

void engine_create(Engine *e, int max_slots, int max_tiles, int MB, cudaStream_t s) {
    if (MB % EB != 0 || MB < 4 * EB || MB > EMBMAX) fail(CI_ERR_INVALID_ARG, "basis size must be a multiple of 8 in 32..96");
    e->MB = MB;
    e->max_slots = max_slots;
    e->max_tiles = max_tiles;
    CI_CUDA(cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking));
    // the engine stream starts after the caller's work (its buffers, built
    // matrices) and owns the engine's own buffers
    {
        cudaEvent_t ev;
        CI_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        CI_CUDA(cudaEventRecord(ev, s));
        CI_CUDA(cudaStreamWaitEvent(e->stream, ev, 0));
        CI_CUDA(cudaEventDestroy(ev));
    }
    StreamScope scope(e->stream);
    e->slots.alloc(max_slots);
    e->tiles.alloc(max_tiles);
    e->ntiles.alloc(1);
    e->counters.alloc(4);
    e->part.alloc((size_t)max_tiles * MB * EB);
    EngineDense &n = e->dn;
    n.T.alloc((size_t)max_slots * MB * MB);
    n.S.alloc((size_t)max_slots * MB * MB);
    n.theta.alloc((size_t)max_slots * MB);
    n.Cl.alloc((size_t)max_slots * 2 * EB * EB);
    n.Cf.alloc((size_t)max_slots * MB * EB);
    n.Cr.alloc((size_t)max_slots * MB * EB);
    n.G.alloc((size_t)max_slots * EB * EB);
    n.M.alloc((size_t)max_slots * EB * EB);
    n.R.alloc((size_t)max_slots * EB * EB);
    n.res.alloc((size_t)max_slots * EKMAX);
    n.evals.alloc((size_t)max_slots * EKMAX);
    n.tres.alloc((size_t)max_slots * EKMAX);
    e->host_slots.assign(max_slots, SlotDev{});
    e->fresh.assign(max_slots, 0);
    CI_CUDA(cudaMemsetAsync(e->slots.ptr, 0, sizeof(SlotDev) * max_slots, e->stream));
    CI_CUDA(cudaMemsetAsync(e->ntiles.ptr, 0, sizeof(int32_t), e->stream));
    CI_CUDA(cudaMallocHost(&e->pinned_counter, sizeof(int32_t) * 4));
    CI_CUDA(cudaFuncSetAttribute(k_e_tn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tn_smem(EMBMAX)));
    CI_CUDA(cudaFuncSetAttribute(k_e_ritz, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ritz_smem(EMBMAX)));
    CI_CUDA(cudaFuncSetAttribute(k_e_restart_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)restart_smem(EMBMAX)));
    CI_CUDA(cudaStreamSynchronize(e->stream));
}

void engine_set_slot(Engine *e, int i, const SlotDev &d) {
    if (i < 0 || i >= e->max_slots) fail(CI_ERR_INVALID_ARG, "slot %d out of range", i);
    SlotDev x = d;
    x.state = S_INIT;
    x.flags = 0;
    x.m_cur = 0; x.j0 = 0; x.m_act = 0; x.it = 0; x.restarts = 0; x.rank = EB; x.hnorm = 0.0;
    e->host_slots[i] = x;
    e->fresh[i] = 1;
}

void engine_free_slot(Engine *e, int i) {
    e->host_slots[i] = SlotDev{};
    e->fresh[i] = 0;
}

void engine_retile(Engine *e) {
    // tile ranges come from the host copy; states from the device
    std::vector<SlotDev> cur(e->max_slots);
    CI_CUDA(cudaMemcpyAsync(cur.data(), e->slots.ptr, sizeof(SlotDev) * e->max_slots, cudaMemcpyDeviceToHost,
                            e->stream));
    CI_CUDA(cudaStreamSynchronize(e->stream));
    std::vector<Tile> tl;
    for (int i = 0; i < e->max_slots; ++i) {
        SlotDev &h = e->host_slots[i];
        if (h.dim == 0 || h.Q == nullptr) { h = SlotDev{}; continue; }
        // slots admitted earlier keep the control state the kernels evolved
        if (!e->fresh[i] && cur[i].Q == h.Q) h = cur[i];
        e->fresh[i] = 0;
        h.tile0 = (int32_t)tl.size();
        for (int64_t r = 0; r < h.dim; r += ETILE) tl.push_back(Tile{i, (int32_t)std::min<int64_t>(ETILE, h.dim - r), r});
        h.tile1 = (int32_t)tl.size();
    }
    if ((int)tl.size() > e->max_tiles) fail(CI_ERR_CAPACITY, "tile list of %zu tiles above %d", tl.size(), e->max_tiles);
    e->host_tiles = tl;
    int32_t nt = (int32_t)tl.size();
    if (nt) CI_CUDA(cudaMemcpyAsync(e->tiles.ptr, tl.data(), sizeof(Tile) * nt, cudaMemcpyHostToDevice, e->stream));
    CI_CUDA(cudaMemcpyAsync(e->ntiles.ptr, &nt, sizeof(int32_t), cudaMemcpyHostToDevice, e->stream));
    CI_CUDA(cudaMemcpyAsync(e->slots.ptr, e->host_slots.data(), sizeof(SlotDev) * e->max_slots, cudaMemcpyHostToDevice,
                            e->stream));
    CI_CUDA(cudaStreamSynchronize(e->stream));
}

// tn + reduce for one mode
static void tn_reduce(Engine *e, int phase, int mode) {
    const DensePtrs d = dense_ptrs(e);
    launch("k_e_tn", k_e_tn, tile_grid(e), 256, tn_smem(e->MB), e->stream, e->slots.ptr, (const Tile *)e->tiles.ptr,
           (const int32_t *)e->ntiles.ptr, e->MB, phase, mode, e->part.ptr);
    launch("k_e_reduce", k_e_reduce, dim3(e->max_slots, (e->MB * EB + 31) / 32), 256, 0, e->stream, e->slots.ptr,
           e->max_slots, e->MB, phase, mode, (const double *)e->part.ptr, d);
}

static void nn(Engine *e, int phase, int mode, int c0 = 0) {
    if (mode == M_QR2)
        launch("k_e_nn", k_e_nn<true>, tile_grid(e), 256, 0, e->stream, e->slots.ptr, (const Tile *)e->tiles.ptr,
               (const int32_t *)e->ntiles.ptr, e->MB, phase, mode, dense_ptrs(e), c0);
    else
        launch("k_e_nn", k_e_nn<false>, sm_count() * 5, 256, 0, e->stream, e->slots.ptr, (const Tile *)e->tiles.ptr,
               (const int32_t *)e->ntiles.ptr, e->MB, phase, mode, dense_ptrs(e), c0);
}

// Block QR of W into Q[:, m:m+8] with rank test and random completion.
static void block_qr(Engine *e, int phase) {
    const DensePtrs d = dense_ptrs(e);
    const int sb = (e->max_slots + 63) / 64;
    tn_reduce(e, phase, M_GRAM);
    launch("k_e_small", k_e_small, sb, 64, 0, e->stream, e->slots.ptr, e->max_slots, phase, 1, d);
    nn(e, phase, M_QR1);
    launch("k_e_rand", k_e_rand, tile_grid(e), 256, 0, e->stream, e->slots.ptr, (const Tile *)e->tiles.ptr,
           (const int32_t *)e->ntiles.ptr, e->MB, phase, 0);
    for (int pass = 0; pass < 2; ++pass) {
        tn_reduce(e, phase, M_RAND);
        nn(e, phase, M_RAND);
    }
    tn_reduce(e, phase, M_GRAMV);
    launch("k_e_small", k_e_small, sb, 64, 0, e->stream, e->slots.ptr, e->max_slots, phase, 2, d);
    nn(e, phase, M_QR2);
}

void engine_init_slots(Engine *e) {
    const DensePtrs d = dense_ptrs(e);
    launch("k_e_rand", k_e_rand, tile_grid(e), 256, 0, e->stream, e->slots.ptr, (const Tile *)e->tiles.ptr,
           (const int32_t *)e->ntiles.ptr, e->MB, (int)PH_INIT, 1);
    block_qr(e, PH_INIT);
    launch("k_e_advance", k_e_advance, (e->max_slots + 63) / 64, 64, 0, e->stream, e->slots.ptr, e->max_slots, e->MB,
           (int)PH_INIT, d);
}

static void record_step(Engine *e) {
    const DensePtrs d = dense_ptrs(e);
    const Tile *tp = e->tiles.ptr;
    const int32_t *nt = e->ntiles.ptr;
    launch("k_e_prepx", k_e_prepx, tile_grid(e), 256, 0, e->stream, e->slots.ptr, tp, nt, e->MB, (int)PH_STEP);
    launch("k_e_spmm", k_e_spmm, sm_count() * e->spmm_mult, 256, 0, e->stream, e->slots.ptr, tp, nt, (int)PH_STEP);
    tn_reduce(e, PH_STEP, M_LOC);
    nn(e, PH_STEP, M_LOC);
    tn_reduce(e, PH_STEP, M_FULL);
    nn(e, PH_STEP, M_FULL);
    launch("k_e_tupdate", k_e_tupdate, e->max_slots, 256, 0, e->stream, e->slots.ptr, e->max_slots, e->MB, d);
    block_qr(e, PH_STEP);
    launch("k_e_advance", k_e_advance, (e->max_slots + 63) / 64, 64, 0, e->stream, e->slots.ptr, e->max_slots, e->MB,
           (int)PH_STEP, d);
    launch("k_e_ritz", k_e_ritz, e->max_slots, 256, ritz_smem(e->MB), e->stream, e->slots.ptr, e->max_slots, e->MB, d);
    launch("k_e_restart_rows", k_e_restart_rows, tile_grid(e), 256, restart_smem(e->MB), e->stream, e->slots.ptr, tp,
           nt, e->MB, d);
    launch("k_e_restart_slot", k_e_restart_slot, e->max_slots, 256, 0, e->stream, e->slots.ptr, e->max_slots, e->MB,
           d);
    launch("k_e_count", k_e_count, 1, 256, 0, e->stream, e->slots.ptr, e->max_slots, e->counters.ptr);
}

void engine_step(Engine *e) {
    if (!e->exec) {
        // capture one step; the launches read all control from device memory
        const bool tr = trace_on();
        if (tr) {  // events cannot be recorded inside a capture: run traced steps eagerly
            record_step(e);
            return;
        }
        CI_CUDA(cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal));
        try {
            record_step(e);
        } catch (...) {
            cudaGraph_t g;
            cudaStreamEndCapture(e->stream, &g);
            if (g) cudaGraphDestroy(g);
            throw;
        }
        CI_CUDA(cudaStreamEndCapture(e->stream, &e->graph));
        CI_CUDA(cudaGraphInstantiate(&e->exec, e->graph, 0));
    }
    if (trace_on()) {
        record_step(e);
        return;
    }
    CI_CUDA(cudaGraphLaunch(e->exec, e->stream));
}

static void drop_graph(Engine *e) {
    CI_CUDA(cudaStreamSynchronize(e->stream));
    if (e->exec) cudaGraphExecDestroy(e->exec);
    if (e->graph) cudaGraphDestroy(e->graph);
    e->exec = nullptr;
    e->graph = nullptr;
}

int engine_autotune(Engine *e) {
    // cache key: device, slots, total rows (to a power of two)
    int dev = 0;
    CI_CUDA(cudaGetDevice(&dev));
    int64_t rows = 0;
    for (const Tile &t : e->host_tiles) rows += t.nr;
    int lg = 0;
    while ((int64_t)1 << lg < rows) ++lg;
    const int64_t key = ((int64_t)dev << 48) | ((int64_t)e->max_slots << 8) | lg;
    static std::mutex mu;
    static std::map<int64_t, std::pair<int, int>> cache;
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end()) {
            if (e->tile_mult != it->second.first || e->spmm_mult != it->second.second) drop_graph(e);
            e->tile_mult = it->second.first;
            e->spmm_mult = it->second.second;
            e->tuned = true;
            return 0;
        }
    }
    cudaEvent_t a, b;
    CI_CUDA(cudaEventCreate(&a));
    CI_CUDA(cudaEventCreate(&b));
    int steps = 0;
    double best = 1e300;
    int best_t = e->tile_mult, best_s = e->spmm_mult;
    auto trial = [&](int tm, int smult) -> bool {
        drop_graph(e);
        e->tile_mult = tm;
        e->spmm_mult = smult;
        engine_step(e);   // capture and run
        CI_CUDA(cudaEventRecord(a, e->stream));
        engine_step(e);   // timed replay
        CI_CUDA(cudaEventRecord(b, e->stream));
        CI_CUDA(cudaEventSynchronize(b));
        steps += 2;
        float ms = 0.f;
        CI_CUDA(cudaEventElapsedTime(&ms, a, b));
        if (ms < best) { best = ms; best_t = tm; best_s = smult; }
        return engine_running(e) > 0;
    };
    bool live = true;
    for (int tm : {4, 2, 8, 16})
        if (live) live = trial(tm, 8);
    const int bt = best_t;
    for (int smult : {4, 16})
        if (live) live = trial(bt, smult);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e->tile_mult != best_t || e->spmm_mult != best_s) drop_graph(e);
    e->tile_mult = best_t;
    e->spmm_mult = best_s;
    e->tuned = true;
    e->tuned_step_ms = best;
    if (live) {   // a finished batch says little about the others
        std::lock_guard<std::mutex> lk(mu);
        cache[key] = {best_t, best_s};
    }
    return steps;
}

int engine_running(Engine *e) {
    CI_CUDA(cudaMemcpyAsync(e->pinned_counter, e->counters.ptr, sizeof(int32_t), cudaMemcpyDeviceToHost, e->stream));
    CI_CUDA(cudaStreamSynchronize(e->stream));
    return e->pinned_counter[0];
}

void engine_true_residuals(Engine *e) {
    const DensePtrs d = dense_ptrs(e);
    const Tile *tp = e->tiles.ptr;
    const int32_t *nt = e->ntiles.ptr;
    const int sb = (e->max_slots + 63) / 64;
    for (int c0 = 0; c0 < EKMAX; c0 += EB) {
        nn(e, PH_FINAL, M_RITZ, c0);  // W = Q S[:, c0:c0+8]
        launch("k_e_prepx", k_e_prepx, tile_grid(e), 256, 0, e->stream, e->slots.ptr, tp, nt, e->MB, (int)PH_FINAL);
        launch("k_e_spmm", k_e_spmm, tile_grid(e), 256, 0, e->stream, e->slots.ptr, tp, nt, (int)PH_FINAL);
        launch("k_e_resid", k_e_resid, tile_grid(e), 256, 0, e->stream, e->slots.ptr, tp, nt, d, e->MB, c0);
        tn_reduce(e, PH_FINAL, M_RESID);
        launch("k_e_store_resid", k_e_store_resid, sb, 64, 0, e->stream, e->slots.ptr, e->max_slots, d, c0);
    }
    launch("k_e_mark_final", k_e_mark_final, sb, 64, 0, e->stream, e->slots.ptr, e->max_slots, d, e->MB);
    CI_CUDA(cudaStreamSynchronize(e->stream));
}

void engine_results(Engine *e, int i, double *evals, double *res_est, double *res_true, int *iters, int *state) {
    SlotDev h;
    CI_CUDA(cudaMemcpyAsync(&h, e->slots.ptr + i, sizeof(SlotDev), cudaMemcpyDeviceToHost, e->stream));
    double ev[EKMAX], re[EKMAX], rt[EKMAX];
    CI_CUDA(cudaMemcpyAsync(ev, e->dn.evals.ptr + (int64_t)i * EKMAX, sizeof(ev), cudaMemcpyDeviceToHost, e->stream));
    CI_CUDA(cudaMemcpyAsync(re, e->dn.res.ptr + (int64_t)i * EKMAX, sizeof(re), cudaMemcpyDeviceToHost, e->stream));
    CI_CUDA(cudaMemcpyAsync(rt, e->dn.tres.ptr + (int64_t)i * EKMAX, sizeof(rt), cudaMemcpyDeviceToHost, e->stream));
    CI_CUDA(cudaStreamSynchronize(e->stream));
    for (int j = 0; j < h.k; ++j) {
        if (evals) evals[j] = ev[j];
        if (res_est) res_est[j] = re[j];
        if (res_true) res_true[j] = rt[j];
    }
    if (iters) *iters = h.it;
    if (state) *state = h.state;
}

}  // namespace ci
