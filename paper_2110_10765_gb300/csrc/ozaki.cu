// FP64 products of the Lanczos reorthogonalisation (Fig. 1, eigensolve) on
// the fifth-generation tensor cores.  Both operands are cut into eight
// balanced base-256 digit planes (Ozaki, Ogita, Oishi and Rump, 2012:
// error-free splitting; Ootomo, Ozaki and Yokota, 2024: the same on
// low-precision matrix units); a digit is an integer in [-128, 127], exact in
// FP16, a product of two digits is exact, and tcgen05.mma sums at most 2^10
// of them (|sum| <= 2^24) exactly in its FP32 accumulator.  Every digit-plane
// product is therefore exact; the planes are recombined with integer
// arithmetic and rounded to FP64 once per output.  Digits reach 2^-62
// relative to each operand's scale, below FP64's own rounding.
//
// The basis A (orthonormal columns, |A| <= 1) is read in a fixed-point
// shadow form kept beside it, Y = trunc(A 2^62) + 0x8080..80 as uint64
// (k_oz_fix): byte 7-k of Y is digit k + 128, so cutting A into planes costs
// byte permutes only.  The vectors (B, C) are cut from FP64 in the kernels,
// each with a power-of-two scale above its largest entry.
//
//   k_oz_tn:  part[blk] = A[rows of blk]^T B   (B: 8 vectors, scale per block)
//   k_oz_nn:  W = beta W + alpha A C            (C [na][8], scale per column)
//
// A digit of x with scale 2^s: X = trunc(x 2^(62-s)) as a two's-complement
// int64, Y = X + 0x8080..80; byte 7-k of Y is d_k + 128 and
// x = 2^s sum_k d_k 2^(-6-8k) up to 2^(s-62).  Eight balanced digits hold
// |X| <= 0x7F7F..7F, i.e. |x| < 1.99 * 2^s: the basis takes s = 0, a vector
// s = 1 + the exponent of its largest entry (|x| < 2^s).
#include <cuda.h>

#include <algorithm>

#include "problem.cuh"
#include "tc.cuh"

namespace ci {

namespace {

constexpr unsigned long long kBias = 0x8080808080808080ull;   // all digits zero

// Biased fixed-point form of x with scale 2^s (see above); bad is set when
// |x| is out of range or not finite.
__device__ __forceinline__ unsigned long long oz_fix(double x, int s, int &bad) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7FF);
    const int sh = e - 1013 - s;
    const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
    unsigned long long X = 0ull;
    if (e != 0) {   // zero and subnormals (far below the last digit) give 0
        if (sh > 10) bad = 1;
        X = sh >= 0 ? (m << (sh < 10 ? sh : 10)) : (sh > -64 ? (m >> (-sh)) : 0ull);
        if (X > 0x7F7F7F7F7F7F7F7Full) bad = 1;
    }
    if (b >> 63) X = 0ull - X;
    return X + kBias;
}

__device__ __forceinline__ __half2 h2_of(uint32_t u) { return *reinterpret_cast<const __half2 *>(&u); }
__device__ __forceinline__ uint32_t u_of(__half2 h) { return *reinterpret_cast<const uint32_t *>(&h); }

// Digits of two biased values a (low half) and b (high half) as FP16 pairs,
// out[k] = (d_k(a), d_k(b)), k = 0..7: the bytes go under the FP16 pattern
// 0x64xx (= 1024 + byte) and 1152 is subtracted, giving byte - 128.
__device__ __forceinline__ void oz_pack2(unsigned long long a, unsigned long long b, uint32_t out[8]) {
    const __half2 off = __half2half2(__ushort_as_half((unsigned short)0x6480));   // 1152
    const uint32_t ah = (uint32_t)(a >> 32), al = (uint32_t)a, bh = (uint32_t)(b >> 32), bl = (uint32_t)b;
    uint32_t t[4];
    t[0] = __byte_perm(ah, bh, 0x6273);   // a.d0 b.d0 a.d1 b.d1
    t[1] = __byte_perm(ah, bh, 0x4051);   // a.d2 b.d2 a.d3 b.d3
    t[2] = __byte_perm(al, bl, 0x6273);   // d4, d5
    t[3] = __byte_perm(al, bl, 0x4051);   // d6, d7
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        out[2 * q] = u_of(__hsub2(h2_of(__byte_perm(t[q], 0x64646464u, 0x4140)), off));
        out[2 * q + 1] = u_of(__hsub2(h2_of(__byte_perm(t[q], 0x64646464u, 0x4342)), off));
    }
}

// Eight K-consecutive biased values -> eight 16-byte rows of K-major tiles
// (digit plane k at dst + k * plane_stride).
__device__ __forceinline__ void oz_store8(const unsigned long long y[8], unsigned char *dst, uint32_t plane_stride) {
    uint32_t h[4][8];
#pragma unroll
    for (int p = 0; p < 4; ++p) oz_pack2(y[2 * p], y[2 * p + 1], h[p]);
#pragma unroll
    for (int k = 0; k < 8; ++k)
        *reinterpret_cast<uint4 *>(dst + k * plane_stride) = make_uint4(h[0][k], h[1][k], h[2][k], h[3][k]);
}

// Byte offset of element (row, k) in a K-major no-swizzle tile with KG
// core matrices along K.
__device__ __forceinline__ uint32_t tile_off(int row, int k, int KG) {
    return (uint32_t)(((row >> 3) * KG + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ int exponent_of(double x) { return (int)((__double_as_longlong(x) >> 52) & 0x7FF) - 1023; }

// (I 2^24 + R) 2^e as a double, truncated toward zero (|I| < 2^62,
// |R| < 2^47): integer arithmetic only.
__device__ __forceinline__ double oz_to_double(long long I, long long R, int e) {
    const __int128 v = ((__int128)I << 24) + (__int128)R;
    const bool neg = v < 0;
    unsigned __int128 u = neg ? (unsigned __int128)(-v) : (unsigned __int128)v;
    const unsigned long long hi = (unsigned long long)(u >> 64), lo = (unsigned long long)u;
    if ((hi | lo) == 0ull) return 0.0;
    const int lz = hi ? __clzll((long long)hi) : 64 + __clzll((long long)lo);
    u <<= lz;                                           // leading one at bit 127
    const unsigned long long top = (unsigned long long)(u >> 64);
    const int ex = 127 - lz + e + 1023;                 // biased exponent of the leading one
    if (ex <= 0) return 0.0;                            // below the normal range: negligible here
    const unsigned long long bits = ((unsigned long long)ex << 52) | ((top >> 11) & 0xFFFFFFFFFFFFFull) |
                                    (neg ? 0x8000000000000000ull : 0ull);
    return __longlong_as_double((long long)bits);
}

constexpr int kWaitPolls = 1 << 22;   // bounded mbarrier waits (error flag 2 when exhausted)

}  // namespace

// ---------------------------------------------------------------- the shadow

// Y[r][c] = biased fixed point of A[r][c] (scale 2^0) for c < nc; bit 0 of
// *flag when an entry has |a| >= 1.99 or is not finite; x32 (nullable,
// [dim][nc]) also receives the entries rounded to FP32.  One thread per
// element, consecutive threads along a row (32-bit indices: dim * nc < 2^31).
__global__ void k_oz_fix(int dim, int nc, const double *__restrict__ A, int lda, unsigned long long *__restrict__ Y,
                         int ldy, int *flag, float *__restrict__ x32) {
    pdl_wait();
    int bad = 0;
    const int total = dim * nc;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int r = t / nc, c = t - r * nc;
        const double x = __ldg(A + (int64_t)r * lda + c);
        Y[(int64_t)r * ldy + c] = oz_fix(x, 0, bad);
        if (x32) x32[t] = (float)x;
    }
    if (bad) atomicOr(flag, 1);
}

// dst[r][c] = src[r][c] and Y[r][c] = its biased fixed point, c < nc: a
// column copy into the basis that keeps the shadow current; x32 (nullable,
// [dim][nc]) also receives the columns rounded to FP32 (the input of the
// next FP32 SpMM).  When skip (nullable) is set the kernel returns at once
// (the columns, their shadow and their FP32 copy are already in place).
__global__ void k_oz_copy_fix(int dim, int nc, const double *__restrict__ src, int lds, double *__restrict__ dst,
                              int ldd, unsigned long long *__restrict__ Y, int ldy, float *__restrict__ x32, int *flag,
                              const int *skip) {
    pdl_wait();
    if (skip && *skip) return;
    int bad = 0;
    const int total = dim * nc;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int r = t / nc, c = t - r * nc;
        const double x = __ldg(src + (int64_t)r * lds + c);
        dst[(int64_t)r * ldd + c] = x;
        Y[(int64_t)r * ldy + c] = oz_fix(x, 0, bad);
        if (x32) x32[t] = (float)x;
    }
    if (bad) atomicOr(flag, 1);
}

// ---------------------------------------------------------------- staging of the shadow

// Both products read the basis shadow through a ring of raw tiles in shared
// memory, one tensor (TMA) copy per stage issued by a loader thread, from a
// 2-D tensor map over the shadow's rows that starts at the 16-byte aligned
// column at or below A's first one (m = 1 when A starts at an odd column)
// and ends at A's last column, so that the box reads nothing else and is
// zero-filled past it.  The ring holds as many stages as fit in its bytes
// (at most kMaxRaw), so that tens of kilobytes per SM are in flight whatever
// the basis width.
constexpr int kMaxRaw = 16;

__device__ __forceinline__ bool pipe_wait(uint64_t *mbar, uint32_t parity, volatile int *abort_, int *flag) {
    if (tc::mbar_wait(mbar, parity, kWaitPolls)) return true;
    *abort_ = 1;
    atomicOr(flag, 2);
    return false;
}

// pipe_wait by every lane of a warp, with one outcome for the whole warp
// (the warp then runs collective instructions: tcgen05.ld, __syncwarp).
__device__ __forceinline__ bool warp_wait(uint64_t *mbar, uint32_t parity, volatile int *abort_, int *flag) {
    const bool ok = !*abort_ && tc::mbar_wait(mbar, parity, kWaitPolls);
    if (__all_sync(0xffffffffu, ok)) return true;
    if ((threadIdx.x & 31) == 0) {
        *abort_ = 1;
        atomicOr(flag, 2);
    }
    return false;
}

__device__ __forceinline__ ulonglong2 lds_u64x2(const unsigned char *p) {
    return *reinterpret_cast<const ulonglong2 *>(p);
}

// ---------------------------------------------------------------- W = beta W + alpha A C

// One CTA per SM over 128-row tiles of A and W, as a pipeline of warp roles:
//   loader (1 warp) copies the rows of a stage (128 rows, <= 32 columns);
//   converters (8 warps) cut the stage into the eight FP16 digit planes a_i
//     (two plane stages);
//   one thread issues the MMAs of a stage: a_i times the planes
//     [c_0 .. c_{7-i}] of C side by side (N = 8 j + n, K = column of A),
//     accumulated into TMEM columns 8 (i + j) + n, so that column block t
//     collects S_t[n] = sum_{i+j=t} a_i c_j directly (|S_t| <= 8 * 64 * 2^14
//     = 2^23: exact in FP32); N is rounded up to a multiple of 16, the extra
//     products land in block t = 8, which is not read;
//   epilogue (16 warps; a thread takes two vectors of one row) reads S_0..S_7
//     of its row and vectors and forms (A C)[r][n] = 2^(s_n - 68)
//     sum_t S_t 256^(7-t) in integers, rounded once, then
//     W = beta W + alpha (A C).
// Two TMEM accumulators of 128 columns let the MMAs of a tile run while the
// epilogue drains the one before.  Every wait is bounded (flag bit 2).
constexpr int kNnConvWarps = 8;
constexpr int kNnEpiWarps = 16;   // four per TMEM lane group, two vectors each
constexpr int kNnVec = 32 / kNnEpiWarps;   // vectors per epilogue thread
constexpr int kNnThreads = 32 * (kNnConvWarps + kNnEpiWarps + 2);   // + MMA warp + loader warp
constexpr int kNnKc = 32;                                  // columns of A per stage
constexpr uint32_t kNnPlane = 128u * kNnKc * 2u;           // one 128 x 32 digit plane
constexpr uint32_t kNnStage = 8u * kNnPlane;               // the eight planes of a stage (two stages)
constexpr uint32_t kNnRawBytes = 2u * 128u * 272u;         // the raw ring
constexpr int kNnItems = 2;                                // 8-column pieces per converter thread

// Row stride (bytes) of the raw ring for a given width and start parity:
// the converters read 8 g + 2 m elements of a row (pairs), and an odd
// number of 16-byte units keeps rows of consecutive lanes on distinct banks.
static uint32_t nn_raw_stride(int na, int m) {
    const int groups = (std::min(na, kNnKc) + 7) / 8;
    const int units = (8 * groups + 2 * m) / 2;   // 16-byte units
    return 16u * (uint32_t)(units | 1);
}

// ymap: boxes of bc columns x 128 rows (bc = raw row stride / 8).
// skip: nullable; when *skip is set the kernel returns at once (W untouched).
__global__ void __launch_bounds__(kNnThreads, 1) k_oz_nn(const __grid_constant__ CUtensorMap ymap, int m, int bc,
                                                  int64_t dim, int na, const double *__restrict__ C,
                                                  double *__restrict__ W, int ldw, double alpha, double beta,
                                                  int *flag, const int *skip) {
    pdl_wait();
    if (skip && *skip) return;
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t rfull[kMaxRaw], rempty[kMaxRaw], full[2], empty[2], tfull[2], tempty[2], done;
    __shared__ uint32_t tmem_base;
    __shared__ int emax[8];
    __shared__ volatile int abort_;
    const uint32_t stride = 8u * (uint32_t)bc;
    const int R = min(kMaxRaw, (int)(kNnRawBytes / (128u * stride)));
    const int nck = (na + kNnKc - 1) / kNnKc;   // stages per tile
    const int KGB = nck * (kNnKc / 8);          // core matrices of C along K
    unsigned char *raw = sm + 2 * kNnStage;
    unsigned char *sB = raw + kNnRawBytes;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid < 8) emax[tid] = -100000;
    if (tid == 0) {
        abort_ = 0;
        for (int q = 0; q < R; ++q) { tc::mbar_init(&rfull[q], 1); tc::mbar_init(&rempty[q], 32 * kNnConvWarps); }
        for (int q = 0; q < 2; ++q) {
            tc::mbar_init(&full[q], 32 * kNnConvWarps);
            tc::mbar_init(&empty[q], 1);
            tc::mbar_init(&tfull[q], 1);
            tc::mbar_init(&tempty[q], kNnEpiWarps);
        }
        tc::mbar_init(&done, 1);
    }
    if (warp == 0) tc::tmem_alloc(&tmem_base, 256);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base;
    {   // column scales of C: thread t takes column t & 7 of rows t >> 3, + kNnThreads / 8, ..
        int em = -100000;
        for (int r = tid >> 3; r < na; r += kNnThreads / 8) {
            const double c = C[r * 8 + (tid & 7)];
            if (c != 0.0) em = max(em, exponent_of(c));
        }
#pragma unroll
        for (int o = 8; o < 32; o <<= 1) em = max(em, __shfl_xor_sync(0xffffffffu, em, o));
        if (lane < 8 && em > -100000) atomicMax(&emax[tid & 7], em);
    }
    __syncthreads();
    int sc[8];   // |C[k][n]| < 2^sc[n]
#pragma unroll
    for (int n = 0; n < 8; ++n) sc[n] = emax[n] < -10000 ? 0 : emax[n] + 1;
    // digit planes of C as the B operand: row 8 j + n, K = k (zero digits for k >= na)
    for (int e = tid; e < KGB * 4 * 8; e += blockDim.x) {
        const int n = e & 7, k = (e >> 3) * 2;
        const double c0 = k < na ? C[k * 8 + n] : 0.0, c1 = k + 1 < na ? C[(k + 1) * 8 + n] : 0.0;
        int bad = 0;
        uint32_t h[8];
        oz_pack2(oz_fix(c0, sc[n], bad), oz_fix(c1, sc[n], bad), h);
        if (bad) atomicOr(flag, 1);
#pragma unroll
        for (int j = 0; j < 8; ++j) *reinterpret_cast<uint32_t *>(sB + tile_off(8 * j + n, k, KGB)) = h[j];
    }
    tc::fence_async_smem();
    __syncthreads();
    const int64_t ntiles = (dim + 127) / 128;
    const int my_tiles = (int64_t)blockIdx.x < ntiles ? (int)((ntiles - 1 - blockIdx.x) / gridDim.x + 1) : 0;
    const int nstage = my_tiles * nck;
    // stage s: tile blockIdx.x + (s / nck) gridDim.x, columns 32 (s % nck) .. (ncols of them)
    if (warp < kNnConvWarps) {
        // ---- converters: pieces it = tid + 256 u: row it & 127, columns 8 (it >> 7) .. + 7 of the stage
        for (int s = 0; s < nstage; ++s) {
            const int slot = s % R, c = s % nck;
            const int ncols = min(kNnKc, na - kNnKc * c);
            const int groups = (ncols + 7) / 8, kst = (ncols + 15) / 16;
            if (abort_ || !pipe_wait(&rfull[slot], (s / R) & 1, &abort_, flag)) break;
            const int pst = s & 1;
            if (s >= 2 && !pipe_wait(&empty[pst], ((s >> 1) - 1) & 1, &abort_, flag)) break;
            const unsigned char *rs = raw + slot * (128u * stride);
            unsigned char *sa = sm + pst * kNnStage;
#pragma unroll
            for (int u = 0; u < kNnItems; ++u) {
                const int it = tid + 32 * kNnConvWarps * u, g = it >> 7;
                unsigned char *dst = sa + tile_off(it & 127, 8 * g, kNnKc / 8);
                if (g < groups) {
                    unsigned long long y[8];
                    const unsigned char *p = rs + (it & 127) * stride + 64 * g;   // element 8 g (even)
                    if (m == 0) {
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const ulonglong2 v = lds_u64x2(p + 16 * q);
                            y[2 * q] = v.x;
                            y[2 * q + 1] = v.y;
                        }
                    } else {   // elements 8 g + 1 .. 8 g + 8
                        ulonglong2 v = lds_u64x2(p);
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const ulonglong2 w = lds_u64x2(p + 16 * (q + 1));
                            y[2 * q] = v.y;
                            y[2 * q + 1] = w.x;
                            v = w;
                        }
                    }
                    oz_store8(y, dst, kNnPlane);
                } else if (g < 2 * kst) {   // inside the last K step, past the columns: zero digits
#pragma unroll
                    for (int k = 0; k < 8; ++k) *reinterpret_cast<uint4 *>(dst + k * kNnPlane) = make_uint4(0, 0, 0, 0);
                }
            }
            tc::mbar_arrive(&rempty[slot]);
            tc::fence_async_smem();
            tc::mbar_arrive(&full[pst]);
        }
    } else if (warp < kNnConvWarps + kNnEpiWarps) {
        // ---- epilogue: warp 8 + q reads TMEM lanes 32 (q & 3) .. + 31 (rows) and
        // takes the vectors n = kNnVec (q >> 2) .. + kNnVec - 1 of those rows
        const int q = warp - kNnConvWarps, lg = q & 3, n0 = kNnVec * (q >> 2);
        const bool flip = alpha == -1.0, unit = alpha == 1.0 || flip;
        const int bmode = beta == 0.0 ? 0 : (beta == 1.0 ? 1 : 2);
        const bool wvec = ((uintptr_t)W % 16) == 0 && (ldw % 2) == 0;
        // this thread's entries of W in tile lt, fetched one tile ahead
        auto wload = [&](int lt, double (&x)[kNnVec]) {
            const int64_t r = ((int64_t)blockIdx.x + (int64_t)lt * gridDim.x) * 128 + 32 * lg + lane;
            if (bmode == 0 || lt >= my_tiles || r >= dim) return;
            const double *w = W + r * ldw + n0;
            if (wvec) {
#pragma unroll
                for (int n = 0; n < kNnVec; n += 2) {
                    const double2 a2 = *reinterpret_cast<const double2 *>(w + n);
                    x[n] = a2.x;
                    x[n + 1] = a2.y;
                }
            } else {
#pragma unroll
                for (int n = 0; n < kNnVec; ++n) x[n] = w[n];
            }
        };
        // The FP64 update of a tile's outputs is issued at the start of the next
        // tile and stored after that tile's integer work, so that the latency of
        // the FP64 pipe overlaps it.
        auto update = [&](const double (&wo)[kNnVec], const double (&d)[kNnVec], double (&o)[kNnVec]) {
#pragma unroll
            for (int k = 0; k < kNnVec; ++k) {
                const double ad = unit ? d[k] : alpha * d[k];
                o[k] = bmode == 0 ? ad : (bmode == 1 ? (unit ? wo[k] + d[k] : fma(alpha, d[k], wo[k])) : fma(beta, wo[k], ad));
            }
        };
        auto wstore = [&](double *w, const double (&o)[kNnVec]) {
            if (wvec) {
#pragma unroll
                for (int k = 0; k < kNnVec; k += 2) *reinterpret_cast<double2 *>(w + k) = make_double2(o[k], o[k + 1]);
            } else {
#pragma unroll
                for (int k = 0; k < kNnVec; ++k) w[k] = o[k];
            }
        };
        double wnext[kNnVec] = {}, pw[kNnVec] = {}, pd[kNnVec] = {};   // next W; the pending tile's W and A C
        double *pwp = nullptr;
        wload(0, wnext);
        for (int lt = 0; lt < my_tiles; ++lt) {
            const int buf = lt & 1;
            const int64_t r = ((int64_t)blockIdx.x + (int64_t)lt * gridDim.x) * 128 + 32 * lg + lane;
            double wold[kNnVec];
#pragma unroll
            for (int n = 0; n < kNnVec; ++n) wold[n] = wnext[n];
            wload(lt + 1, wnext);
            double pout[kNnVec];
            if (pwp) update(pw, pd, pout);
            if (!warp_wait(&tfull[buf], (lt >> 1) & 1, &abort_, flag)) break;
            tc::fence_after_sync();
            float v[8 * kNnVec];   // v[kNnVec t + k] = S_t[n0 + k]
            tc::ld8xN<kNnVec>(tmem + ((uint32_t)(32 * lg) << 16) + 128u * buf + n0, v);
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&tempty[buf]);
            double d[kNnVec];
#pragma unroll
            for (int k = 0; k < kNnVec; ++k) {
                // sum_t S_t 256^(7-t) = I 2^24 + R exactly (|I| < 2^56, |R| < 2^40)
                long long I = __float2int_rn(v[k]);
#pragma unroll
                for (int t = 1; t <= 4; ++t) I = I * 256 + __float2int_rn(v[kNnVec * t + k]);
                long long Rr = __float2int_rn(v[5 * kNnVec + k]);
                Rr = Rr * 256 + __float2int_rn(v[6 * kNnVec + k]);
                Rr = Rr * 256 + __float2int_rn(v[7 * kNnVec + k]);
                if (flip) { I = -I; Rr = -Rr; }
                d[k] = oz_to_double(I, Rr, sc[n0 + k] - 68);
            }
            if (pwp) wstore(pwp, pout);
            pwp = r < dim ? W + r * ldw + n0 : nullptr;
#pragma unroll
            for (int k = 0; k < kNnVec; ++k) { pw[k] = wold[k]; pd[k] = d[k]; }
        }
        if (pwp) {
            double pout[kNnVec];
            update(pw, pd, pout);
            wstore(pwp, pout);
        }
    } else if (warp == kNnConvWarps + kNnEpiWarps) {
        // ---- MMA issue (one thread)
        if (lane == 0) {
            int s = 0;
            for (int lt = 0; lt < my_tiles && !abort_; ++lt) {
                const int buf = lt & 1;
                if (lt >= 2 && !pipe_wait(&tempty[buf], ((lt >> 1) - 1) & 1, &abort_, flag)) break;
                tc::fence_after_sync();
                const uint32_t dcol = tmem + 128u * buf;
                bool ok = true;
                for (int c = 0; c < nck; ++c, ++s) {
                    const int pst = s & 1;
                    const int kst = (min(kNnKc, na - kNnKc * c) + 15) / 16;
                    if (!pipe_wait(&full[pst], (s >> 1) & 1, &abort_, flag)) { ok = false; break; }
                    tc::fence_after_sync();
                    const unsigned char *sa = sm + pst * kNnStage;
                    for (int i = 0; i < 8; ++i) {
                        const int N = 16 * ((9 - i) / 2);   // 8 (8 - i) rounded up to 16
                        const uint32_t idesc = tc::idesc_f16_f32(128, N);
                        for (int ks = 0; ks < kst; ++ks) {
                            const uint64_t ad =
                                tc::desc_kmajor(tc::smem_addr(sa + i * kNnPlane + ks * 256), 128, (kNnKc / 8) * 128);
                            const uint64_t bd =
                                tc::desc_kmajor(tc::smem_addr(sB + (c * (kNnKc / 8) + 2 * ks) * 128), 128, KGB * 128);
                            tc::mma_f16(dcol + 8 * i, ad, bd, idesc, c > 0 || i > 0 || ks > 0);
                        }
                    }
                    tc::commit(&empty[pst]);
                }
                if (!ok) break;
                tc::commit(&tfull[buf]);
            }
            tc::commit(&done);   // every MMA issued above has completed when this phase does
            if (!tc::mbar_wait(&done, 0, kWaitPolls)) atomicOr(flag, 2);
        }
    } else {
        // ---- loader: one tensor copy per stage
        if (lane == 0) {
            for (int s = 0; s < nstage && !abort_; ++s) {
                const int slot = s % R;
                if (s >= R && !pipe_wait(&rempty[slot], ((s / R) - 1) & 1, &abort_, flag)) break;
                const int64_t r0 = ((int64_t)blockIdx.x + (int64_t)(s / nck) * gridDim.x) * 128;
                tc::mbar_expect_tx(&rfull[slot], 128u * stride);
                tc::tma_2d(raw + slot * (128u * stride), &ymap, kNnKc * (s % nck), (int)r0, &rfull[slot]);
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, 256);
    }
}

// ---------------------------------------------------------------- part = A^T B

// One CTA per SM sums its contiguous rows [q0, q1) of A^T B, in 64-row
// stages (the MMA's K) grouped into segments of at most 1024 rows.  The M
// dimension of an operand stacks PP = 128 / MC digit planes of A^T, MC =
// 16, 32 or 64 the columns of A rounded up (M-row MC h + m holds plane
// PP p + h of column m; operands p = 0 .. 8 / PP - 1), the B operand holds
// the digit planes of the eight vectors side by side (N = 8 n + j).
// Accumulator p of a segment (TMEM columns 64 p ..) collects D[PP p + h][m][n][j]
// over the segment's rows; at most 1024 rows keep |D| <= 2^24 exact.  Two
// segment accumulators (2 x 256 columns) alternate, so the epilogue of a
// segment runs while the next one is multiplied.  Roles as in k_oz_nn: the
// loader copies a stage's rows of the shadow, converters (8 warps) cut them
// and the stage's rows of B into the digit planes (two plane stages), one
// thread issues the MMAs, four epilogue warps (one TMEM lane each: plane
// offset h, column m) add up the plane pairs of equal weight i + j <= 7 of a
// segment in 32-bit integers and keep the weighted sum over segments in
// 128-bit integers; at the end the lanes of a column are added and the
// block's part is rounded once.
constexpr int kTnConvWarps = 8;
constexpr int kTnEpiWarps = 4;
constexpr int kTnThreads = 32 * (kTnConvWarps + kTnEpiWarps + 2);   // + MMA warp + loader warp
constexpr int kOzTnRows = 64;
constexpr int kOzTnMaxRows = 1024;   // rows of one segment: |D| <= 1024 * 128^2 = 2^24
constexpr uint32_t kTnAop = 128u * kOzTnRows * 2u;    // one 128 x 64 A operand
constexpr uint32_t kTnBop = 64u * kOzTnRows * 2u;     // the 64 x 64 B operand
constexpr uint32_t kTnStage = 4u * kTnAop + kTnBop;   // two plane stages
constexpr uint32_t kTnRawBytes = 83968u;   // the raw ring: A's rows and B's rows of each stage

// ymap: boxes of bc columns x 64 rows of the shadow; bmap: boxes of bw
// columns x 64 rows of B from its 16-byte aligned column at or below B's
// first (B's vector n at raw column n + mb).
template <int MC>
__global__ void __launch_bounds__(kTnThreads, 1) k_oz_tn(const __grid_constant__ CUtensorMap ymap,
                                                  const __grid_constant__ CUtensorMap bmap, int m, int bc, int mb,
                                                  int bw, int64_t dim, int na, const double *__restrict__ B, int ldb,
                                                  double *__restrict__ part, int64_t rows_per_blk, int *flag) {
    pdl_wait();
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t rfull[kMaxRaw], rempty[kMaxRaw], full[2], empty[2], tfull[2], tempty[2], done;
    __shared__ uint32_t tmem_base;
    __shared__ int emax[8];
    __shared__ volatile int abort_;
    unsigned char *raw = sm + 2 * kTnStage;
    __int128 *red = reinterpret_cast<__int128 *>(raw);   // [PP - 1][MC][8]: the h >= 1 sums, once the ring is idle
    constexpr int KG = kOzTnRows / 8;
    constexpr int PP = 128 / MC, NOP = 8 / PP;             // planes per operand, operands
    constexpr int ITEMS = 8 * MC;                          // (column, 8-row group) pieces of a stage
    constexpr int NIT = (ITEMS + 32 * kTnConvWarps - 1) / (32 * kTnConvWarps);
    const uint32_t stride = 8u * (uint32_t)bc;
    const uint32_t aslot = kOzTnRows * stride, slotb = aslot + kOzTnRows * 8u * (uint32_t)bw;
    const int R = min(kMaxRaw, (int)(kTnRawBytes / slotb));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t q0 = min(dim, (int64_t)blockIdx.x * rows_per_blk);
    const int64_t q1 = min(dim, q0 + rows_per_blk);
    const int64_t nrows = q1 - q0;
    const int nst = (int)((nrows + kOzTnRows - 1) / kOzTnRows);                 // stages
    const int nseg0 = (int)((nrows + kOzTnMaxRows - 1) / kOzTnMaxRows);
    const int seg_st = nseg0 ? (nst + nseg0 - 1) / nseg0 : 1;                   // stages per segment (<= 16)
    const int nseg = (nst + seg_st - 1) / seg_st;
    if (tid < 8) emax[tid] = -100000;
    if (tid == 0) {
        abort_ = 0;
        for (int q = 0; q < R; ++q) { tc::mbar_init(&rfull[q], 1); tc::mbar_init(&rempty[q], 32 * kTnConvWarps); }
        for (int q = 0; q < 2; ++q) {
            tc::mbar_init(&full[q], 32 * kTnConvWarps);
            tc::mbar_init(&empty[q], 1);
            tc::mbar_init(&tfull[q], 1);
            tc::mbar_init(&tempty[q], kTnEpiWarps);
        }
        tc::mbar_init(&done, 1);
    }
    if (warp == 0) tc::tmem_alloc(&tmem_base, 512);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base;
    {   // vector scales over this block's rows: thread t takes vector t & 7 of rows t >> 3, + kTnThreads / 8, ..
        constexpr int kStep = kTnThreads / 8;
        int em = -100000;
        const int n = tid & 7;
        int64_t r = tid >> 3;
        for (; r + 7 * kStep < nrows; r += 8 * kStep) {   // eight independent loads in flight
            double x[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) x[k] = B[(q0 + r + k * kStep) * ldb + n];
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (x[k] != 0.0) em = max(em, exponent_of(x[k]));
        }
        for (; r < nrows; r += kStep) {
            const double x = B[(q0 + r) * ldb + n];
            if (x != 0.0) em = max(em, exponent_of(x));
        }
#pragma unroll
        for (int o = 8; o < 32; o <<= 1) em = max(em, __shfl_xor_sync(0xffffffffu, em, o));
        if (lane < 8 && em > -100000) atomicMax(&emax[n], em);
    }
    __syncthreads();
    int sc[8];   // |B[r][n]| < 2^sc[n] over this block's rows
#pragma unroll
    for (int n = 0; n < 8; ++n) sc[n] = emax[n] < -10000 ? 0 : emax[n] + 1;

    if (warp < kTnConvWarps) {
        // ---- converters: A pieces it = tid + 256 u (column it % MC of stage rows 8 (it / MC) ..
        // + 7); B vector bn of rows brl, brl + 1
        const int bn = tid & 7, brl = 2 * (tid >> 3);
        for (int s = 0; s < nst; ++s) {
            const int slot = s % R, pst = s & 1;
            if (abort_ || !pipe_wait(&rfull[slot], (s / R) & 1, &abort_, flag)) break;
            const int64_t t0 = q0 + (int64_t)s * kOzTnRows;
            const unsigned char *rb = raw + slot * slotb + aslot + 8 * (bn + mb);   // B rows (zero past dim)
            const double wa = t0 + brl < q1 ? *reinterpret_cast<const double *>(rb + brl * (8 * bw)) : 0.0;
            const double wb = t0 + brl + 1 < q1 ? *reinterpret_cast<const double *>(rb + (brl + 1) * (8 * bw)) : 0.0;
            unsigned long long y[NIT][8];
#pragma unroll
            for (int u = 0; u < NIT; ++u) {
                const int it = tid + 32 * kTnConvWarps * u, mc = it % MC;
                if (it >= ITEMS || mc >= na) continue;
                const unsigned char *rs = raw + slot * slotb + (8 * (it / MC)) * stride + 8 * (mc + m);
#pragma unroll
                for (int k = 0; k < 8; ++k) y[u][k] = *reinterpret_cast<const unsigned long long *>(rs + k * stride);
            }
            tc::mbar_arrive(&rempty[slot]);
            if (s >= 2 && !pipe_wait(&empty[pst], ((s >> 1) - 1) & 1, &abort_, flag)) break;
            unsigned char *sa = sm + pst * kTnStage, *sb = sa + 4 * kTnAop;
            // the 8 rows of column mc are one 16-byte row of each plane; plane i of
            // column mc sits in operand i / PP at M-row MC (i % PP) + mc
#pragma unroll
            for (int u = 0; u < NIT; ++u) {
                const int it = tid + 32 * kTnConvWarps * u, mc = it % MC, rg = it / MC;
                if (it >= ITEMS || mc >= na) continue;
                uint32_t hp[4][8];
#pragma unroll
                for (int p = 0; p < 4; ++p) oz_pack2(y[u][2 * p], y[u][2 * p + 1], hp[p]);
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    *reinterpret_cast<uint4 *>(sa + (i / PP) * kTnAop + tile_off(MC * (i % PP) + mc, 8 * rg, KG)) =
                        make_uint4(hp[0][i], hp[1][i], hp[2][i], hp[3][i]);
            }
            int bad = 0;
            uint32_t h[8];
            oz_pack2(oz_fix(wa, sc[bn], bad), oz_fix(wb, sc[bn], bad), h);
            if (bad) atomicOr(flag, 1);
#pragma unroll
            for (int j = 0; j < 8; ++j) *reinterpret_cast<uint32_t *>(sb + tile_off(8 * bn + j, brl, KG)) = h[j];
            tc::fence_async_smem();
            tc::mbar_arrive(&full[pst]);
        }
    } else if (warp < kTnConvWarps + kTnEpiWarps) {
        // ---- epilogue: TMEM lane L = 32 q + lane is (h = L / MC, column m = L % MC); it holds
        // D[i][m][n][j] of the planes i = PP p + h at columns 256 buf + 64 p + 8 n + j
        const int q = warp - kTnConvWarps;
        const int L = 32 * q + lane, h = L / MC, mc = L % MC;
        __int128 acc[8];
#pragma unroll
        for (int n = 0; n < 8; ++n) acc[n] = 0;
        for (int sg = 0; sg < nseg; ++sg) {
            const int buf = sg & 1;
            if (!warp_wait(&tfull[buf], (sg >> 1) & 1, &abort_, flag)) break;
            tc::fence_after_sync();
#pragma unroll 1
            for (int n = 0; n < 8; ++n) {
                float v[32];   // v[8 p + j] = D[PP p + h][mc][n][j] (p < NOP)
                tc::ld4x8(tmem + ((uint32_t)(32 * q) << 16) + 256u * buf + 8u * n, v);
                // U_k = sum over the pairs with PP p + j = k, i.e. i + j = k + h, of the
                // segment's exact integer sums (|U_k| <= 4 * 2^24); the pairs with
                // i + j > 7 lie below the digits' resolution and are left out
                int U[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) U[k] = 0;
#pragma unroll
                for (int p = 0; p < NOP; ++p)
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int k = PP * p + j;
                        if (k <= 7 && k <= 7 - h) U[k] += __float2int_rn(v[8 * p + j]);
                    }
                // sum_k U_k 2^(56 - 8 k) = I 2^24 + R; in units of 2^(s_n - 68) the
                // pairs contribute that times 2^(-8 h) (exact: U_k = 0 for k > 7 - h)
                const long long I = ((long long)U[0] << 32) + ((long long)U[1] << 24) + ((long long)U[2] << 16) +
                                    ((long long)U[3] << 8) + (long long)U[4];
                const long long Rr = ((long long)U[5] << 16) + ((long long)U[6] << 8) + (long long)U[7];
                __int128 x = ((__int128)I << 24) + (__int128)Rr;
                x >>= 8 * h;
                acc[n] += x;
            }
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&tempty[buf]);
        }
        if (h > 0) {
#pragma unroll
            for (int n = 0; n < 8; ++n) red[((h - 1) * MC + mc) * 8 + n] = acc[n];
        }
        tc::named_sync(1, 32 * kTnEpiWarps);
        if (h == 0 && mc < na) {
#pragma unroll
            for (int n = 0; n < 8; ++n) {
                __int128 t = acc[n];
                for (int g = 1; g < PP; ++g) t += red[((g - 1) * MC + mc) * 8 + n];
                const long long hi = (long long)(t >> 64);
                const unsigned long long lo = (unsigned long long)t;
                const int e = sc[n] - 68;
                part[((int64_t)blockIdx.x * na + mc) * 8 + n] = fma((double)hi, ldexp(1.0, e + 64), ldexp((double)lo, e));
            }
        }
    } else if (warp == kTnConvWarps + kTnEpiWarps) {
        // ---- MMA issue (one thread)
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_f16_f32(128, 64);
            for (int s = 0; s < nst && !abort_; ++s) {
                const int sg = s / seg_st, buf = sg & 1, pst = s & 1;
                const bool first = s == sg * seg_st, last = s == nst - 1 || s + 1 == (sg + 1) * seg_st;
                if (first && sg >= 2 && !pipe_wait(&tempty[buf], ((sg >> 1) - 1) & 1, &abort_, flag)) break;
                if (!pipe_wait(&full[pst], (s >> 1) & 1, &abort_, flag)) break;
                tc::fence_after_sync();
                const unsigned char *sa = sm + pst * kTnStage, *sb = sa + 4 * kTnAop;
                for (int p = 0; p < NOP; ++p)
#pragma unroll
                    for (int ks = 0; ks < kOzTnRows / 16; ++ks) {
                        const uint64_t ad = tc::desc_kmajor(tc::smem_addr(sa + p * kTnAop + ks * 256), 128, KG * 128);
                        const uint64_t bd = tc::desc_kmajor(tc::smem_addr(sb + ks * 256), 128, KG * 128);
                        tc::mma_f16(tmem + 256u * buf + 64u * p, ad, bd, idesc, !first || ks > 0);
                    }
                tc::commit(&empty[pst]);
                if (last) tc::commit(&tfull[buf]);
            }
            tc::commit(&done);
            if (!tc::mbar_wait(&done, 0, kWaitPolls)) atomicOr(flag, 2);
        }
    } else {
        // ---- loader: one tensor copy per stage
        if (lane == 0) {
            for (int s = 0; s < nst && !abort_; ++s) {
                const int slot = s % R;
                if (s >= R && !pipe_wait(&rempty[slot], ((s / R) - 1) & 1, &abort_, flag)) break;
                const int y = (int)(q0 + (int64_t)s * kOzTnRows);
                tc::mbar_expect_tx(&rfull[slot], slotb);
                tc::tma_2d(raw + slot * slotb, &ymap, 0, y, &rfull[slot]);
                tc::tma_2d(raw + slot * slotb + aslot, &bmap, 0, y, &rfull[slot]);
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, 512);
    }
}

// ---------------------------------------------------------------- launchers

static size_t oz_nn_smem(int na) {
    const int KGB = ((na + kNnKc - 1) / kNnKc) * (kNnKc / 8);
    return (size_t)2 * kNnStage + kNnRawBytes + (size_t)8 * KGB * 128;   // plane stages, raw ring, C planes
}
constexpr size_t kOzTnSmem = (size_t)2 * kTnStage + kTnRawBytes;
static_assert(kTnRawBytes >= 112 * 8 * sizeof(__int128), "the final sums reuse the raw ring");

bool oz_supported(int na) { return na >= 1 && na <= 64; }

using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiled encode_tiled() {
    static EncodeTiled fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        CI_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
        if (!p || q != cudaDriverEntryPointSuccess) fail(CI_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
        fn = reinterpret_cast<EncodeTiled>(p);
    }
    return fn;
}

// Tensor map over rows of 8-byte elements P[r * ld + c] (ld even), columns
// from the 16-byte aligned one at or below P (m = 1 when P is odd) to the
// ncols-th from P, all `rows` rows, boxes of bc x br elements.
static CUtensorMap rows_map(const void *P, int ld, int64_t rows, int ncols, int bc, int br, int &m) {
    if ((ld & 1) || ((uintptr_t)P & 7)) fail(CI_ERR_INTERNAL, "tensor-core product: odd row stride or misaligned rows");
    if (rows >= ((int64_t)1 << 31)) fail(CI_ERR_CAPACITY, "tensor-core product: %lld rows", (long long)rows);
    m = (int)(((uintptr_t)P >> 3) & 1);
    CUtensorMap map;
    const cuuint64_t gdim[2] = {(cuuint64_t)(ncols + m), (cuuint64_t)rows};
    const cuuint64_t gstride[1] = {(cuuint64_t)ld * 8};
    const cuuint32_t box[2] = {(cuuint32_t)bc, (cuuint32_t)br};
    const cuuint32_t es[2] = {1, 1};
    const CUresult r = encode_tiled()(&map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2,
                                      const_cast<void *>(static_cast<const void *>(static_cast<const char *>(P) - 8 * m)),
                                      gdim, gstride, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) fail(CI_ERR_CUDA, "tensor map of the product operands: error %d", (int)r);
    return map;
}

void oz_fix(int64_t dim, int nc, const double *A, int lda, unsigned long long *Y, int ldy, int *flag,
            cudaStream_t s, float *x32) {
    if (dim == 0 || nc == 0) return;
    if (dim * nc >= ((int64_t)1 << 31)) fail(CI_ERR_CAPACITY, "basis shadow: %lld entries", (long long)(dim * nc));
    launch_pdl("k_oz_fix", k_oz_fix, grid_for(dim * nc, 256, sm_count() * 16), 256, 0, s, (int)dim, nc, A, lda, Y, ldy,
               flag, x32);
}

void oz_copy_fix(int64_t dim, int nc, const double *src, int lds, double *dst, int ldd, unsigned long long *Y, int ldy,
                 float *x32, int *flag, cudaStream_t s, const int *skip) {
    if (dim == 0 || nc == 0) return;
    if (dim * nc >= ((int64_t)1 << 31)) fail(CI_ERR_CAPACITY, "basis shadow: %lld entries", (long long)(dim * nc));
    launch_pdl("k_copy_cols", k_oz_copy_fix, grid_for(dim * nc, 256, sm_count() * 16), 256, 0, s, (int)dim, nc, src, lds,
               dst, ldd, Y, ldy, x32, flag, skip);
}

void oz_nn(int64_t dim, const unsigned long long *Y, int ldy, int na, const double *C, double *W, int ldw,
           double alpha, double beta, int *flag, cudaStream_t s, const int *skip) {
    static bool attr = false;
    if (!attr) {
        CI_CUDA(cudaFuncSetAttribute(k_oz_nn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)oz_nn_smem(64)));
        attr = true;
    }
    if (dim == 0) return;
    const int bc = (int)nn_raw_stride(na, ((uintptr_t)Y >> 3) & 1) / 8;
    int m = 0;
    const CUtensorMap map = rows_map(Y, ldy, dim, na, bc, 128, m);
    const int64_t ntiles = (dim + 127) / 128;
    const int grid = (int)std::min<int64_t>(ntiles, sm_count());
    launch_pdl("k_oz_nn", k_oz_nn, grid, kNnThreads, oz_nn_smem(na), s, map, m, bc, dim, na, C, W, ldw, alpha, beta,
               flag, skip);
}

// Row blocks of oz_tn: one per SM (a block takes any number of rows in
// segments of at most 1024), fewer for a short A.
int oz_tn_blocks(int64_t dim) {
    return (int)std::max<int64_t>(1, std::min<int64_t>(sm_count(), (dim + kOzTnRows - 1) / kOzTnRows));
}

void oz_tn(int64_t dim, const unsigned long long *Y, int ldy, int na, const double *B, int ldb, double *part,
           int nblk, int *flag, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        CI_CUDA(cudaFuncSetAttribute(k_oz_tn<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kOzTnSmem));
        CI_CUDA(cudaFuncSetAttribute(k_oz_tn<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kOzTnSmem));
        CI_CUDA(cudaFuncSetAttribute(k_oz_tn<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kOzTnSmem));
        attr = true;
    }
    const int bc = (int)((na + (((uintptr_t)Y >> 3) & 1) + 1) & ~1);   // A's columns from the aligned one
    const int bw = 8 + 2 * (int)(((uintptr_t)B >> 3) & 1);             // B's eight, from the aligned one
    int m = 0, mb = 0;
    const CUtensorMap ymap = rows_map(Y, ldy, std::max<int64_t>(dim, 1), na, bc, kOzTnRows, m);
    const CUtensorMap bmap = rows_map(B, ldb, std::max<int64_t>(dim, 1), 8, bw, kOzTnRows, mb);
    const int64_t rpb = (dim + nblk - 1) / nblk;
    auto kern = na <= 16 ? k_oz_tn<16> : (na <= 32 ? k_oz_tn<32> : k_oz_tn<64>);
    launch_pdl("k_oz_tn", kern, nblk, kTnThreads, kOzTnSmem, s, ymap, bmap, m, bc, mb, bw, dim, na, B, ldb, part, rpb, flag);
}

}  // namespace ci
