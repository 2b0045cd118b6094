// Nonzero-count benchmark (Sec. 2.1, Listings 1-2, Figs. 3-4): for n
// independent N-particle states in MBS form (ascending s.p. indices), the
// number of states that differ from each in at most max_diff s.p. states.
//
// Three forms of the pair test, which give identical counts:
//   HYBRID  popcount of the XOR of the bits of the lowest 64 s.p. states
//           first; only pairs that pass compare their MBS lists (Listing 2);
//           before it, a cheaper bound (the XOR folded to 32 bits) rejects
//           most pairs with one population count;
//   MBS     the MBS comparison for every pair (no prefilter);
//   BITS    the complete bit representation (S <= 128): popcount only.
// The MBS comparison counts the common states of the two lists; two
// N-particle states then differ in 2 (N - common) states, the count that
// Listing 1 reaches by walking both sorted lists.
//
// Layout: a block owns 256 * R rows (R per thread, strided by 256 so that
// loads coalesce) and one chunk of columns; the chunk is staged through
// shared memory in tiles, each column read as a broadcast by all lanes.
// Row counts are added atomically per (row, chunk); the total per warp.
#include "problem.cuh"

namespace ci {

namespace {

constexpr int kCntThreads = 256;
constexpr int kCntTile = 1024;   // columns per shared-memory tile
constexpr int kCntMaxN = 32;

struct CountArgs {
    int64_t n;
    int N, max_diff;
    const uint16_t *mbs;     // [n][N]
    const uint64_t *bits;    // [n][2]: states 0..63, 64..127
    int64_t chunk;           // columns per chunk
    unsigned long long *rows_out;   // [n] or null
    unsigned long long *total;
};

__global__ void k_cnt_bits(const uint16_t *mbs, int64_t n, int N, uint64_t *bits) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t lo = 0, hi = 0;
        for (int k = 0; k < N; ++k) {
            const unsigned a = mbs[i * N + k];
            if (a < 64) lo |= 1ull << a;
            else if (a < 128) hi |= 1ull << (a - 64);
        }
        bits[2 * i] = lo;
        bits[2 * i + 1] = hi;
    }
}

// Common states of two ascending lists of na and nb entries: used on the
// rare pairs that pass the 64-state prefilter.
__device__ __noinline__ int common_states(const uint16_t *a, const uint16_t *b, int na, int nb) {
    int i = 0, j = 0, c = 0;
    while (i < na && j < nb) {
        const int x = a[i], y = b[j];
        c += x == y;
        i += x <= y;
        j += y <= x;
    }
    return c;
}

__device__ __forceinline__ void flush_counts(const CountArgs &a, int64_t row, unsigned long long c) {
    if (row < a.n && c && a.rows_out) atomicAdd(a.rows_out + row, c);
    unsigned long long s = row < a.n ? c : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(a.total, s);
}

// HYBRID (VAR 0) and BITS (VAR 2): R rows per thread, kept as 32-bit
// halves.  The population count is first taken of the XOR folded to 32 bits
// with OR (a lower bound of the true count, one POPC); a column goes to the
// exact test only when the smallest folded count over the thread's R rows is
// within max_diff (the common case is two LOP3, a POPC and a min per pair):
// the 64-bit popcount (and, for HYBRID, the MBS comparison; for BITS, the
// upper 64 states too).
template <int VAR, int R>
__global__ void __launch_bounds__(kCntThreads, VAR == 2 ? 2 : 3) k_count_bits(CountArgs a) {
    __shared__ uint2 slo[kCntTile];
    __shared__ uint2 shi[VAR == 2 ? kCntTile : 1];
    const int64_t r0 = (int64_t)blockIdx.x * kCntThreads * R + threadIdx.x;
    const int64_t c0 = (int64_t)blockIdx.y * a.chunk;
    const int64_t c1 = min(a.n, c0 + a.chunk);
    uint32_t l0[R], l1[R], h0[R], h1[R];
    unsigned cnt[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int64_t r = r0 + (int64_t)k * kCntThreads;
        const uint64_t lo = r < a.n ? a.bits[2 * r] : 0ull;
        const uint64_t hi = r < a.n ? a.bits[2 * r + 1] : 0ull;
        l0[k] = (uint32_t)lo;
        l1[k] = (uint32_t)(lo >> 32);
        h0[k] = (uint32_t)hi;
        h1[k] = (uint32_t)(hi >> 32);
        cnt[k] = 0;
    }
    const int md = a.max_diff;
    for (int64_t t0 = c0; t0 < c1; t0 += kCntTile) {
        const int nt = (int)min((int64_t)kCntTile, c1 - t0);
        __syncthreads();
        for (int e = threadIdx.x; e < nt; e += kCntThreads) {
            const uint64_t lo = a.bits[2 * (t0 + e)];
            slo[e] = make_uint2((uint32_t)lo, (uint32_t)(lo >> 32));
            if (VAR == 2) {
                const uint64_t hi = a.bits[2 * (t0 + e) + 1];
                shi[e] = make_uint2((uint32_t)hi, (uint32_t)(hi >> 32));
            }
        }
        __syncthreads();
        for (int j = 0; j < nt; ++j) {
            const uint2 b = slo[j];
            const uint2 bh = VAR == 2 ? shi[j] : make_uint2(0u, 0u);
            int m = 64;
#pragma unroll
            for (int k = 0; k < R; ++k) {
                uint32_t f = (l0[k] ^ b.x) | (l1[k] ^ b.y);
                if (VAR == 2) f |= (h0[k] ^ bh.x) | (h1[k] ^ bh.y);
                m = min(m, __popc(f));
            }
            if (m > md) continue;
            // rare: at least one row is near this column
#pragma unroll
            for (int k = 0; k < R; ++k) {
                uint32_t f = (l0[k] ^ b.x) | (l1[k] ^ b.y);
                if (VAR == 2) f |= (h0[k] ^ bh.x) | (h1[k] ^ bh.y);
                if (__popc(f) > md) continue;
                const int d64 = __popc(l0[k] ^ b.x) + __popc(l1[k] ^ b.y);
                if (VAR == 2) {
                    cnt[k] += (d64 + __popc(h0[k] ^ bh.x) + __popc(h1[k] ^ bh.y)) <= md;
                } else if (d64 <= md) {
                    // the lowest 64 states differ little; compare the MBS
                    // lists.  Their first popc(lo) entries are those states
                    // (ascending order), whose common count the bits give:
                    // only the entries from state 64 on are walked.
                    const int64_t r = r0 + (int64_t)k * kCntThreads;
                    if (r < a.n) {
                        const int na = __popc(l0[k]) + __popc(l1[k]), nb = __popc(b.x) + __popc(b.y);
                        const int c = (na + nb - d64) / 2 +
                                      common_states(a.mbs + r * a.N + na, a.mbs + (t0 + j) * a.N + nb, a.N - na,
                                                    a.N - nb);
                        cnt[k] += 2 * (a.N - c) <= md;
                    }
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < R; ++k) flush_counts(a, r0 + (int64_t)k * kCntThreads, cnt[k]);
}

// MBS (no prefilter), N known at compile time: R rows per thread, the row
// lists in registers, each column list a broadcast from shared memory.
template <int N, int R>
__global__ void __launch_bounds__(kCntThreads) k_count_mbs(CountArgs a) {
    __shared__ uint16_t smbs[kCntTile * N];
    const int64_t r0 = (int64_t)blockIdx.x * kCntThreads * R + threadIdx.x;
    const int64_t c0 = (int64_t)blockIdx.y * a.chunk;
    const int64_t c1 = min(a.n, c0 + a.chunk);
    int x[R][N];
    unsigned long long cnt[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int64_t r = r0 + (int64_t)k * kCntThreads;
#pragma unroll
        for (int i = 0; i < N; ++i) x[k][i] = r < a.n ? (int)a.mbs[r * N + i] : -1 - i;
        cnt[k] = 0;
    }
    const int need = N - a.max_diff / 2;   // common states needed
    for (int64_t t0 = c0; t0 < c1; t0 += kCntTile) {
        const int nt = (int)min((int64_t)kCntTile, c1 - t0);
        __syncthreads();
        for (int e = threadIdx.x; e < nt * N; e += kCntThreads) smbs[e] = a.mbs[t0 * N + e];
        __syncthreads();
        for (int j = 0; j < nt; ++j) {
            const uint16_t *b = smbs + j * N;
            int c[R];
#pragma unroll
            for (int k = 0; k < R; ++k) c[k] = 0;
#pragma unroll
            for (int q = 0; q < N; ++q) {
                const int y = b[q];
#pragma unroll
                for (int k = 0; k < R; ++k)
#pragma unroll
                    for (int i = 0; i < N; ++i) c[k] += x[k][i] == y;
            }
#pragma unroll
            for (int k = 0; k < R; ++k) cnt[k] += c[k] >= need;
        }
    }
#pragma unroll
    for (int k = 0; k < R; ++k) flush_counts(a, r0 + (int64_t)k * kCntThreads, cnt[k]);
}

// MBS with N known only at run time (N not in the unrolled set).
__global__ void __launch_bounds__(kCntThreads) k_count_mbs_any(CountArgs a) {
    extern __shared__ uint16_t smbs_any[];
    const int64_t r = (int64_t)blockIdx.x * kCntThreads + threadIdx.x;
    const int64_t c0 = (int64_t)blockIdx.y * a.chunk;
    const int64_t c1 = min(a.n, c0 + a.chunk);
    uint16_t x[kCntMaxN];
    for (int i = 0; i < a.N; ++i) x[i] = r < a.n ? a.mbs[r * a.N + i] : 0;
    unsigned long long cnt = 0;
    for (int64_t t0 = c0; t0 < c1; t0 += kCntTile) {
        const int nt = (int)min((int64_t)kCntTile, c1 - t0);
        __syncthreads();
        for (int e = threadIdx.x; e < nt * a.N; e += kCntThreads) smbs_any[e] = a.mbs[t0 * a.N + e];
        __syncthreads();
        if (r < a.n)
            for (int j = 0; j < nt; ++j)
                cnt += 2 * (a.N - common_states(x, smbs_any + j * a.N, a.N, a.N)) <= a.max_diff;
    }
    flush_counts(a, r, cnt);
}

template <int R>
static dim3 count_grid(int64_t n, int64_t &chunk) {
    const int64_t rb = (n + (int64_t)kCntThreads * R - 1) / ((int64_t)kCntThreads * R);
    // enough blocks for every SM several times over: split the columns
    const int64_t want = (int64_t)sm_count() * 8;
    int64_t nc = (want + rb - 1) / rb;
    if (nc < 1) nc = 1;
    chunk = (n + nc - 1) / nc;
    chunk = (chunk + kCntTile - 1) / kCntTile * kCntTile;
    nc = (n + chunk - 1) / chunk;
    if (rb > INT32_MAX || nc > 65535) fail(CI_ERR_CAPACITY, "count grid too large (n = %lld)", (long long)n);
    return dim3((unsigned)rb, (unsigned)nc);
}

template <int N>
static void launch_mbs(CountArgs a, cudaStream_t s) {
    constexpr int R = N <= 8 ? 2 : 1;
    dim3 g = count_grid<R>(a.n, a.chunk);
    launch("k_count_mbs", k_count_mbs<N, R>, g, kCntThreads, 0, s, a);
}

}  // namespace

void count_pairs(const uint16_t *mbs, int64_t n, int N, int S, int variant, int max_diff, int64_t *total,
                 int64_t *row_counts, cudaStream_t s) {
    if (n < 0) fail(CI_ERR_INVALID_ARG, "n < 0");
    if (N < 1 || N > kCntMaxN) fail(CI_ERR_INVALID_ARG, "N must be 1..%d (got %d)", kCntMaxN, N);
    if (S < N || S > 65535) fail(CI_ERR_INVALID_ARG, "S must be N..65535 (got %d)", S);
    if (max_diff < 0) fail(CI_ERR_INVALID_ARG, "max_diff < 0");
    if (variant != CI_COUNT_HYBRID && variant != CI_COUNT_MBS && variant != CI_COUNT_BITS)
        fail(CI_ERR_INVALID_ARG, "unknown count variant %d", variant);
    if (variant == CI_COUNT_BITS && S > 128) fail(CI_ERR_INVALID_ARG, "the bit form needs S <= 128 (got %d)", S);
    if (!total) fail(CI_ERR_INVALID_ARG, "total is NULL");
    if (n > 0 && !mbs) fail(CI_ERR_INVALID_ARG, "mbs is NULL");
    if (n > 0 && !is_device_pointer(mbs)) fail(CI_ERR_INVALID_ARG, "mbs must be a device pointer");
    if (row_counts && n > 0 && !is_device_pointer(row_counts))
        fail(CI_ERR_INVALID_ARG, "row_counts must be a device pointer");
    *total = 0;
    if (row_counts && n > 0) CI_CUDA(cudaMemsetAsync(row_counts, 0, sizeof(int64_t) * n, s));
    if (n == 0) return;
    DevBuf<unsigned long long> dtot(1);
    CI_CUDA(cudaMemsetAsync(dtot.ptr, 0, sizeof(unsigned long long), s));
    DevBuf<uint64_t> bits;
    CountArgs a{};
    a.n = n; a.N = N; a.max_diff = max_diff; a.mbs = mbs;
    a.rows_out = reinterpret_cast<unsigned long long *>(row_counts);
    a.total = dtot.ptr;
    if (variant != CI_COUNT_MBS) {
        bits.alloc((size_t)n * 2);
        launch("k_cnt_bits", k_cnt_bits, grid_for(n, 256), 256, 0, s, mbs, n, N, bits.ptr);
        a.bits = bits.ptr;
    }
    if (variant == CI_COUNT_HYBRID) {
        dim3 g = count_grid<8>(n, a.chunk);
        launch("k_count_hybrid", k_count_bits<0, 8>, g, kCntThreads, 0, s, a);
    } else if (variant == CI_COUNT_BITS) {
        dim3 g = count_grid<8>(n, a.chunk);
        launch("k_count_bits", k_count_bits<2, 8>, g, kCntThreads, 0, s, a);
    } else {
        switch (N) {
            case 4: launch_mbs<4>(a, s); break;
            case 8: launch_mbs<8>(a, s); break;
            case 12: launch_mbs<12>(a, s); break;
            case 16: launch_mbs<16>(a, s); break;
            case 20: launch_mbs<20>(a, s); break;
            default: {
                dim3 g = count_grid<1>(n, a.chunk);
                const int smem = (int)(sizeof(uint16_t) * kCntTile * N);
                CI_CUDA(cudaFuncSetAttribute(k_count_mbs_any, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
                launch("k_count_mbs", k_count_mbs_any, g, kCntThreads, smem, s, a);
            }
        }
    }
    unsigned long long h = 0;
    CI_CUDA(cudaMemcpyAsync(&h, dtot.ptr, sizeof(h), cudaMemcpyDeviceToHost, s));
    CI_CUDA(cudaStreamSynchronize(s));
    *total = (int64_t)h;
}

}  // namespace ci

extern "C" ci_status ci_count_pairs(const uint16_t *mbs, int64_t n, int32_t N, int32_t S, int32_t variant,
                                    int32_t max_diff, int64_t *total, int64_t *row_counts, void *stream) {
    return ci::guard([&] {
        cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
        ci::StreamScope scope(s);
        ci::count_pairs(mbs, n, N, S, variant, max_diff, total, row_counts, s);
    });
}
