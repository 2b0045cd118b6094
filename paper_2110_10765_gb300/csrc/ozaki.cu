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

// Integer-valued floats to integers without a conversion instruction:
// f + 1.5 * 2^23 holds an integer |f| <= 2^22 in its low mantissa bits,
// its bit pattern is 0x4B400000 + f.
constexpr float kMagic = 12582912.0f;
constexpr uint32_t kMagicBits = 0x4B400000u;
// Any integer-valued |f| <= 2^24, from its fields.
__device__ __forceinline__ int f2i_exact(float f) {
    const uint32_t b = __float_as_uint(f);
    const int e = (int)((b >> 23) & 0xFF);
    if (e < 127) return 0;
    const uint32_t m = (b & 0x7FFFFFu) | 0x800000u;
    const int sh = 150 - e;
    const uint32_t mag = sh >= 0 ? (m >> sh) : (m << 1);
    return (b >> 31) ? -(int)mag : (int)mag;
}

// Columns c, c+1 of a shadow row (kBias for a column >= na): one 16-byte
// load when both exist and the row is 16-byte aligned there, else 8-byte
// loads (a thick restart may leave a block at an odd column).
__device__ __forceinline__ ulonglong2 load_pair(const unsigned long long *p, bool ok0, bool ok1, bool vec16) {
    if (ok0 && ok1 && vec16) return __ldg(reinterpret_cast<const ulonglong2 *>(p));
    ulonglong2 v = make_ulonglong2(kBias, kBias);
    if (ok0) v.x = __ldg(p);
    if (ok1) v.y = __ldg(p + 1);
    return v;
}

}  // namespace

// ---------------------------------------------------------------- the shadow

// Y[r][c] = biased fixed point of A[r][c] (scale 2^0) for c < nc; bit 0 of
// *flag when an entry has |a| >= 1.99 or is not finite.  One thread per
// element, consecutive threads along a row (32-bit indices: dim * nc < 2^31).
__global__ void k_oz_fix(int dim, int nc, const double *__restrict__ A, int lda, unsigned long long *__restrict__ Y,
                         int ldy, int *flag) {
    int bad = 0;
    const int total = dim * nc;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int r = t / nc, c = t - r * nc;
        Y[(int64_t)r * ldy + c] = oz_fix(__ldg(A + (int64_t)r * lda + c), 0, bad);
    }
    if (bad) atomicOr(flag, 1);
}

// dst[r][c] = src[r][c] and Y[r][c] = its biased fixed point, c < nc: a
// column copy into the basis that keeps the shadow current.
__global__ void k_oz_copy_fix(int dim, int nc, const double *__restrict__ src, int lds, double *__restrict__ dst,
                              int ldd, unsigned long long *__restrict__ Y, int ldy, int *flag) {
    int bad = 0;
    const int total = dim * nc;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int r = t / nc, c = t - r * nc;
        const double x = __ldg(src + (int64_t)r * lds + c);
        dst[(int64_t)r * ldd + c] = x;
        Y[(int64_t)r * ldy + c] = oz_fix(x, 0, bad);
    }
    if (bad) atomicOr(flag, 1);
}

// ---------------------------------------------------------------- W = beta W + alpha A C

// One CTA per SM; 128-row tiles of A and W.  The eight digit planes a_i of
// the tile are the A operands (128 x Kp, K-major), the digit planes c_j of C
// side by side the B operand (N = 8 j + n, K = column of A); accumulator D_i
// holds a_i [c_0 .. c_{7-i}] (N = 8 (8 - i)), 288 TMEM columns in all.  A row
// then needs S_t[n] = sum_{i+j=t} D_i[8 j + n] (t <= 7, exact in FP32) and
// (A C)[r][n] = 2^(s_n - 68) sum_t S_t 256^(7-t).  Each thread loads four
// 8-column pieces of the next tile while the tensor core works on this one.
constexpr int kNnThreads = 512;
constexpr int kNnItems = 2;   // 8-column pieces per thread and tile (128 rows x 64 columns / 512)

__global__ void __launch_bounds__(kNnThreads, 1) k_oz_nn(int64_t dim, const unsigned long long *__restrict__ Y, int ldy,
                                                  int na, const double *__restrict__ C, double *__restrict__ W,
                                                  int ldw, double alpha, double beta, int *flag) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    __shared__ int emax[8];
    const int Kp = (na + 15) & ~15, KG = Kp / 8;
    const uint32_t plane = 16u * KG * 128u;   // bytes of one 128 x Kp digit plane
    unsigned char *sA = sm;
    unsigned char *sB = sm + 8 * plane;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid < 8) emax[tid] = -100000;
    if (tid == 0) tc::mbar_init(&mbar, 1);
    if (warp == 0) tc::tmem_alloc(&tmem_base, 512);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base;
    // column scales of C
    for (int e = tid; e < na * 8; e += blockDim.x) {
        const double c = C[e];
        if (c != 0.0) atomicMax(&emax[e & 7], exponent_of(c));
    }
    __syncthreads();
    int sc[8];   // |C[m][n]| < 2^sc[n]
#pragma unroll
    for (int n = 0; n < 8; ++n) sc[n] = emax[n] < -10000 ? 0 : emax[n] + 1;
    // digit planes of C (pairs of K-adjacent elements, one column n)
    for (int e = tid; e < (Kp / 2) * 8; e += blockDim.x) {
        const int n = e & 7, m = (e >> 3) * 2;
        const double c0 = m < na ? C[m * 8 + n] : 0.0, c1 = m + 1 < na ? C[(m + 1) * 8 + n] : 0.0;
        int bad = 0;
        uint32_t h[8];
        oz_pack2(oz_fix(c0, sc[n], bad), oz_fix(c1, sc[n], bad), h);
        if (bad) atomicOr(flag, 1);
#pragma unroll
        for (int j = 0; j < 8; ++j) *reinterpret_cast<uint32_t *>(sB + tile_off(8 * j + n, m, KG)) = h[j];
    }
    const bool flip = alpha == -1.0, unit = alpha == 1.0 || flip;
    const int bmode = beta == 0.0 ? 0 : (beta == 1.0 ? 1 : 2);
    const bool vec16 = ((uintptr_t)Y % 16) == 0 && (ldy % 2) == 0;
    const int64_t ntiles = (dim + 127) / 128;
    const int items = 128 * KG;   // 8-column pieces of a tile
    // this thread's pieces of a tile: row rl = it / KG, columns 8 (it % KG) ..
    auto load = [&](int64_t r0, ulonglong2 v[kNnItems][4]) {
#pragma unroll
        for (int u = 0; u < kNnItems; ++u) {
            const int it = tid + kNnThreads * u;
            const int rl = it / KG, m0 = 8 * (it - rl * KG);
            const int64_t r = r0 + rl;
            const bool rok = it < items && r < dim;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                v[u][q] = load_pair(Y + r * ldy + m0 + 2 * q, rok && m0 + 2 * q < na, rok && m0 + 2 * q + 1 < na, vec16);
        }
    };
    ulonglong2 pre[kNnItems][4];
    if (blockIdx.x < ntiles) load((int64_t)blockIdx.x * 128, pre);
    uint32_t phase = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t r0 = tile * 128;
#pragma unroll
        for (int u = 0; u < kNnItems; ++u) {
            const int it = tid + kNnThreads * u;
            if (it >= items) continue;
            const int rl = it / KG, m0 = 8 * (it - rl * KG);
            const unsigned long long y[8] = {pre[u][0].x, pre[u][0].y, pre[u][1].x, pre[u][1].y,
                                             pre[u][2].x, pre[u][2].y, pre[u][3].x, pre[u][3].y};
            oz_store8(y, sA + tile_off(rl, m0, KG), plane);
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            uint32_t col = 0;
            for (int i = 0; i < 8; ++i) {
                const int N = 8 * (8 - i);
                const uint32_t idesc = tc::idesc_f16_f32(128, N);
                for (int ks = 0; ks < Kp / 16; ++ks) {
                    const uint64_t ad = tc::desc_kmajor(tc::smem_addr(sA + i * plane + ks * 256), 128, KG * 128);
                    const uint64_t bd = tc::desc_kmajor(tc::smem_addr(sB + ks * 256), 128, KG * 128);
                    tc::mma_f16(tmem + col, ad, bd, idesc, ks > 0);
                }
                col += N;
            }
            tc::commit(&mbar);
        }
        if (tile + gridDim.x < ntiles) load((tile + gridDim.x) * 128, pre);   // overlaps the tensor core
        // this thread's two entries of W, also fetched while the tensor core works
        const int wg = warp >> 2, wrl = (warp & 3) * 32 + lane;
        double wold[2] = {0.0, 0.0};
        if (bmode != 0 && r0 + wrl < dim) {
            const double *w = W + (r0 + wrl) * ldw + 2 * wg;
            wold[0] = w[0];
            wold[1] = w[1];
        }
        const bool ok = __syncthreads_and(tc::mbar_wait(&mbar, phase, kWaitPolls));
        if (!ok) {   // the tensor core did not finish: report, give it one more bounded wait, stop
            if (tid == 0) atomicOr(flag, 2);
            tc::mbar_wait(&mbar, phase, kWaitPolls);
            break;
        }
        phase ^= 1u;
        tc::fence_after_sync();
        {   // warps w, w + 4, w + 8, w + 12 read the same 32 lanes (rows); warp group g takes vectors 2g, 2g+1
            const int g = warp >> 2, rl = (warp & 3) * 32 + lane;
            const int64_t r = r0 + rl;
            // S_t = sum_{i+j=t} D_i[8 j + n] (t + 1 terms, |D| <= 2^20) as
            // sums of the bit patterns of D + kMagic
            uint32_t S[8][2];
#pragma unroll
            for (int t = 0; t < 8; ++t)
#pragma unroll
                for (int n = 0; n < 2; ++n) S[t][n] = 0u - (uint32_t)(t + 1) * kMagicBits;
            uint32_t col = 0;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                float v[16];   // v[2 j + n] = D_i[8 j + 2 g + n]
                tc::ld8x2(tmem + ((uint32_t)((warp & 3) * 32) << 16) + col + 2 * g, v);
#pragma unroll
                for (int j = 0; j < 8 - i; ++j)
#pragma unroll
                    for (int n = 0; n < 2; ++n) S[i + j][n] += __float_as_uint(v[2 * j + n] + kMagic);
                col += 8 * (8 - i);
            }
            if (r < dim) {
                double *w = W + r * ldw + 2 * g;
#pragma unroll
                for (int n = 0; n < 2; ++n) {
                    // sum_t S_t 256^(7-t) = I 2^24 + R exactly (|I| < 2^56, |R| < 2^40)
                    long long I = (int)S[0][n];
#pragma unroll
                    for (int t = 1; t <= 4; ++t) I = I * 256 + (int)S[t][n];
                    long long R = (int)S[5][n];
                    R = R * 256 + (int)S[6][n];
                    R = R * 256 + (int)S[7][n];
                    if (flip) { I = -I; R = -R; }
                    double d = oz_to_double(I, R, sc[2 * g + n] - 68);
                    if (!unit) d *= alpha;
                    w[n] = bmode == 0 ? d : (bmode == 1 ? wold[n] + d : fma(beta, wold[n], d));
                }
            }
        }
        tc::fence_before_sync();
        __syncthreads();
    }
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, 512);
    }
}

// ---------------------------------------------------------------- part = A^T B

// Block blk sums rows [blk rows_per_blk, ...) in tiles of 64 rows (the MMA's
// K).  The M dimension stacks two digit planes of A^T (rows 64 h + m hold
// plane 2 p + h of column m); the B operand holds the digit planes of the
// eight vectors side by side (N = 8 j + n).  Accumulator p (TMEM columns
// 64 p ...) collects D[2p + h][m][j][n]; a block has at most 1024 rows, so
// the sums (|D| <= 2^24) stay exact in TMEM and are read once at the end;
// only the pairs i + j <= 7 are used (the others lie below the digits'
// resolution).
// Each thread cuts 8 rows of one column pair of A (loaded for the next
// tile while the tensor core works) and a row pair of one vector.
constexpr int kOzTnRows = 64;
constexpr int kOzTnMaxRows = 1024;   // rows of one block: |D| <= 1024 * 128^2 = 2^24

__global__ void __launch_bounds__(256, 2) k_oz_tn(int64_t dim, const unsigned long long *__restrict__ Y, int ldy, int na,
                                               const double *__restrict__ B, int ldb, double *__restrict__ part,
                                               int64_t rows_per_blk, int *flag) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    __shared__ int emax[8];
    constexpr int KG = kOzTnRows / 8;
    constexpr uint32_t aplane = 16u * KG * 128u;   // one 128 x 64 A operand
    unsigned char *sA = sm;                        // 4 operands
    unsigned char *sB = sm + 4 * aplane;           // 64 x 64
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t r0 = blockIdx.x * rows_per_blk;
    const int64_t r1 = min(dim, r0 + rows_per_blk);
    if (tid < 8) emax[tid] = -100000;
    if (tid == 0) tc::mbar_init(&mbar, 1);
    if (warp == 0) tc::tmem_alloc(&tmem_base, 256);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base;
    // vector scales over this block's rows
    for (int64_t e = tid; e < (r1 - r0) * 8; e += blockDim.x) {
        const double x = B[(r0 + (e >> 3)) * ldb + (e & 7)];
        if (x != 0.0) atomicMax(&emax[e & 7], exponent_of(x));
    }
    __syncthreads();
    int sc[8];   // |B[r][n]| < 2^sc[n] over this block's rows
#pragma unroll
    for (int n = 0; n < 8; ++n) sc[n] = emax[n] < -10000 ? 0 : emax[n] + 1;
    const int cp = tid & 31, rg = tid >> 5;           // A: columns 2cp, 2cp+1 of rows 8rg .. 8rg+7
    const int bn = tid & 7, brl = 2 * (tid >> 3);     // B: vector bn, rows brl, brl+1
    const bool colok = 2 * cp < na, col1ok = 2 * cp + 1 < na;
    const bool vec16 = ((uintptr_t)Y % 16) == 0 && (ldy % 2) == 0;
    auto load = [&](int64_t t0, ulonglong2 a[8], double &wa, double &wb) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int64_t r = t0 + 8 * rg + q;
            a[q] = load_pair(Y + r * ldy + 2 * cp, colok && r < r1, col1ok && r < r1, vec16);
        }
        wa = t0 + brl < r1 ? B[(t0 + brl) * ldb + bn] : 0.0;
        wb = t0 + brl + 1 < r1 ? B[(t0 + brl + 1) * ldb + bn] : 0.0;
    };
    uint32_t phase = 0;
    bool failed = false;
    ulonglong2 pa[8];
    double pwa = 0.0, pwb = 0.0;
    if (r0 < r1) load(r0, pa, pwa, pwb);
    for (int64_t t0 = r0; t0 < r1; t0 += kOzTnRows) {
        {   // A digit planes: the 8 rows of column 2cp (then 2cp + 1) are one 16-byte row of each plane;
            // plane i of column m sits in operand i >> 1 at M-row 64 (i & 1) + m
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                unsigned long long y[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) y[q] = c ? pa[q].y : pa[q].x;
                uint32_t h[4][8];
#pragma unroll
                for (int p = 0; p < 4; ++p) oz_pack2(y[2 * p], y[2 * p + 1], h[p]);
                const int m = 2 * cp + c;
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    *reinterpret_cast<uint4 *>(sA + (i >> 1) * aplane + tile_off(64 * (i & 1) + m, 8 * rg, KG)) =
                        make_uint4(h[0][i], h[1][i], h[2][i], h[3][i]);
            }
        }
        {   // B digit planes
            int bad = 0;
            uint32_t h[8];
            oz_pack2(oz_fix(pwa, sc[bn], bad), oz_fix(pwb, sc[bn], bad), h);
            if (bad) atomicOr(flag, 1);
#pragma unroll
            for (int j = 0; j < 8; ++j) *reinterpret_cast<uint32_t *>(sB + tile_off(8 * j + bn, brl, KG)) = h[j];
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t idesc = tc::idesc_f16_f32(128, 64);
            for (int p = 0; p < 4; ++p)
                for (int ks = 0; ks < kOzTnRows / 16; ++ks) {
                    const uint64_t ad = tc::desc_kmajor(tc::smem_addr(sA + p * aplane + ks * 256), 128, KG * 128);
                    const uint64_t bd = tc::desc_kmajor(tc::smem_addr(sB + ks * 256), 128, KG * 128);
                    tc::mma_f16(tmem + 64 * p, ad, bd, idesc, t0 > r0 || ks > 0);
                }
            tc::commit(&mbar);
        }
        if (t0 + kOzTnRows < r1) load(t0 + kOzTnRows, pa, pwa, pwb);   // overlaps the tensor core
        const bool ok = __syncthreads_and(tc::mbar_wait(&mbar, phase, kWaitPolls));
        if (!ok) {
            if (tid == 0) atomicOr(flag, 2);
            tc::mbar_wait(&mbar, phase, kWaitPolls);
            failed = true;
            break;
        }
        phase ^= 1u;
        tc::fence_before_sync();
        __syncthreads();
    }
    // planes of A combined exactly in 128-bit integers: with the block's
    // sums D_j (j = 0..7) of plane i, column m, vector n,
    // sum_j D_j 256^(7-j) = I 2^24 + R, and the plane contributes
    // (I 2^24 + R) 2^(40 - 8 i) in units of 2^(s_n - 108) (bits below that
    // unit are dropped for i = 6, 7)
    __int128 *red = reinterpret_cast<__int128 *>(sm);   // [8 planes][64][8]: 64 KB of the free operand area
    tc::fence_after_sync();
    {
        const int R = (warp & 3) * 32 + lane, h = R >> 6, m = R & 63, g = warp >> 2;
#pragma unroll
        for (int pp = 0; pp < 2; ++pp) {
            const int p = 2 * g + pp, i = 2 * p + h;
            float v[64];
            if (r0 < r1 && !failed) {
                tc::ld64(tmem + ((uint32_t)((warp & 3) * 32) << 16) + 64 * p, v);
            } else {
#pragma unroll
                for (int q = 0; q < 64; ++q) v[q] = 0.f;
            }
#pragma unroll
            for (int n = 0; n < 8; ++n) {
                int d[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) d[j] = j <= 7 - i ? f2i_exact(v[8 * j + n]) : 0;
                long long I = d[0];
#pragma unroll
                for (int j = 1; j <= 4; ++j) I = I * 256 + d[j];
                long long Rr = d[5];
                Rr = Rr * 256 + d[6];
                Rr = Rr * 256 + d[7];
                __int128 x = (__int128)I << (64 - 8 * i);
                const int sr = 40 - 8 * i;
                x += sr >= 0 ? ((__int128)Rr << sr) : (__int128)(Rr >> (-sr));
                red[(i * 64 + m) * 8 + n] = x;
            }
        }
    }
    __syncthreads();
    for (int o = tid; o < na * 8; o += blockDim.x) {
        __int128 t = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) t += red[i * 512 + o];
        const long long hi = (long long)(t >> 64);
        const unsigned long long lo = (unsigned long long)t;
        const int e = sc[o & 7] - 108;
        part[(int64_t)blockIdx.x * na * 8 + o] = fma((double)hi, ldexp(1.0, e + 64), ldexp((double)lo, e));
    }
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, 256);
    }
}

// ---------------------------------------------------------------- launchers

static size_t oz_nn_smem(int na) {
    const int KG = ((na + 15) & ~15) / 8;
    return (size_t)(8 * 16 + 8) * KG * 128;   // eight 128-row A planes + the C planes (64 rows)
}
constexpr size_t kOzTnSmem = (size_t)(4 * 16 + 8) * (kOzTnRows / 8) * 128;

bool oz_supported(int na) { return na >= 1 && na <= 64; }

void oz_fix(int64_t dim, int nc, const double *A, int lda, unsigned long long *Y, int ldy, int *flag,
            cudaStream_t s) {
    if (dim == 0 || nc == 0) return;
    if (dim * nc >= ((int64_t)1 << 31)) fail(CI_ERR_CAPACITY, "basis shadow: %lld entries", (long long)(dim * nc));
    launch("k_oz_fix", k_oz_fix, grid_for(dim * nc, 256, sm_count() * 16), 256, 0, s, (int)dim, nc, A, lda, Y, ldy,
           flag);
}

void oz_copy_fix(int64_t dim, int nc, const double *src, int lds, double *dst, int ldd, unsigned long long *Y, int ldy,
                 int *flag, cudaStream_t s) {
    if (dim == 0 || nc == 0) return;
    if (dim * nc >= ((int64_t)1 << 31)) fail(CI_ERR_CAPACITY, "basis shadow: %lld entries", (long long)(dim * nc));
    launch("k_copy_cols", k_oz_copy_fix, grid_for(dim * nc, 256, sm_count() * 16), 256, 0, s, (int)dim, nc, src, lds,
           dst, ldd, Y, ldy, flag);
}

void oz_nn(int64_t dim, const unsigned long long *Y, int ldy, int na, const double *C, double *W, int ldw,
           double alpha, double beta, int *flag, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        CI_CUDA(cudaFuncSetAttribute(k_oz_nn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)oz_nn_smem(64)));
        attr = true;
    }
    if (dim == 0) return;
    const int64_t ntiles = (dim + 127) / 128;
    const int grid = (int)std::min<int64_t>(ntiles, sm_count());
    launch("k_oz_nn", k_oz_nn, grid, kNnThreads, oz_nn_smem(na), s, dim, Y, ldy, na, C, W, ldw, alpha, beta, flag);
}

// Row blocks of oz_tn: two per SM, more when a block would exceed 1024
// rows (its TMEM sums stay exact up to that).
int oz_tn_blocks(int64_t dim) {
    int64_t nb = std::max<int64_t>(2 * sm_count(), (dim + kOzTnMaxRows - 1) / kOzTnMaxRows);
    nb = std::min<int64_t>(nb, std::max<int64_t>((dim + 63) / 64, 1));
    return (int)nb;
}

void oz_tn(int64_t dim, const unsigned long long *Y, int ldy, int na, const double *B, int ldb, double *part,
           int nblk, int *flag, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        CI_CUDA(cudaFuncSetAttribute(k_oz_tn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kOzTnSmem));
        attr = true;
    }
    const int64_t rpb = (dim + nblk - 1) / nblk;
    if (rpb > kOzTnMaxRows) fail(CI_ERR_INTERNAL, "tensor-core product: %lld rows per block", (long long)rpb);
    launch("k_oz_tn", k_oz_tn, nblk, 256, kOzTnSmem, s, dim, Y, ldy, na, B, ldb, part, rpb, flag);
}

}  // namespace ci
