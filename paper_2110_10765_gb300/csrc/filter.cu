// Species-level connectivity (Fig. 1, tile filter, Sec. 2.1, Listing 2):
// XOR + popcount over every pair of determinants of one species, count ->
// scan -> fill with warp ballots, and the like-particle part of every
// Slater-Condon element evaluated once per species pair.
#include "problem.cuh"

namespace ci {

// One sweep of a species list against itself.  It serves every list of
// that species (mode bits 1 << CONN_*): the XOR + popcount of a pair is
// taken once and each list applies its own keep rule.  Both species share
// the sweep when they are the same list (Z = N over one s.p. table).
template <class T>
struct FilterArgs {
    int64_t n;
    int A, S, W;
    int modes;                 // lists filled by this sweep
    const uint64_t *bits;      // [n][W]
    const int32_t *twoM;       // [n]
    const int32_t *local;      // [n]
    const uint8_t *occ;        // [n][A]
    const int32_t *q;          // [n] excess quanta
    const int64_t *blk_start;  // [nblk+1] 2M blocks of the sorted list
    int m2min, nblk, K;        // lowest 2M, blocks, largest |2m| of a state
    const T *eps;
    const T *U[2], *D[2], *C[2];   // like-particle tables: [0] protons, [1] neutrons
    const int32_t *pair_row, *pair_col;
    const int32_t *tr_base;    // proton list: row offset of a proton move in the pn table
    const int32_t *tr_idx;     // neutron lists: column index of a neutron move
    const int64_t *p_row_base; // proton list: first basis row of every determinant
    int32_t *count[kModes];    // pass 0, per list
    const int64_t *ptr[kModes];   // pass 1, per list
    ConnEntry<T> *ent;         // pass 1 (shared entry array)
    int32_t *tgt;              // pass 1: partner index of every entry
};

__device__ __forceinline__ int lowest_state(const uint64_t *x, int W) {
    for (int w = 0; w < W; ++w)
        if (x[w]) return w * 64 + __ffsll((long long)x[w]) - 1;
    return -1;
}

__device__ __forceinline__ int count_below(const uint64_t *K, int W, int o) {
    int c = 0;
    for (int w = 0; w < W; ++w) c += __popcll(K[w] & below_mask_word(o, w));
    return c;
}

__device__ __forceinline__ void flip(uint64_t *K, int o) { K[o >> 6] ^= 1ull << (o & 63); }

// Entry for row determinant s (bra) and partner t (ket) of one list: the
// like-particle Slater-Condon part with the species' tables (sp 0 protons,
// 1 neutrons) and what the row kernels need about the move.
template <class T>
__device__ __forceinline__ ConnEntry<T> make_entry(const FilterArgs<T> &a, int mode, int64_t s, int64_t t,
                                                   const uint64_t *bs, const uint64_t *bt, int d) {
    const bool proton = mode == CONN_OUTER || mode == CONN_O4;
    const int sp = proton ? 0 : 1;
    ConnEntry<T> e;
    e.tgt = (int32_t)t;
    e.local = a.local[t];
    const int S = a.S, W = a.W;
    if (d == 0) {
        // like-particle diagonal: one-body energies + every occupied pair
        const uint8_t *o = a.occ + s * a.A;
        const T *D = a.D[sp];
        T v = 0;
        for (int i = 0; i < a.A; ++i) v += a.eps[o[i]];
        for (int i = 0; i < a.A; ++i)
            for (int j = i + 1; j < a.A; ++j) v += D[o[i] * S + o[j]];
        e.info = make_info(0, 0, 0, 0);
        e.val = v;
    } else {
        uint64_t xa[kMaxWords], xc[kMaxWords], K[kMaxWords];
        for (int w = 0; w < kMaxWords; ++w) {
            uint64_t x = w < W ? (bs[w] ^ bt[w]) : 0ull;
            xa[w] = w < W ? (x & bt[w]) : 0ull;   // in the ket only: annihilated
            xc[w] = w < W ? (x & bs[w]) : 0ull;   // in the bra only: created
            K[w] = w < W ? bt[w] : 0ull;
        }
        if (d == 2) {
            int ao = lowest_state(xa, W), co = lowest_state(xc, W);
            int par = count_below(K, W, ao);       // a_a on the ket
            flip(K, ao);
            par += count_below(K, W, co);          // then a+_c
            // spectators: the ket's other particles
            const uint8_t *o = a.occ + t * a.A;
            T h = 0;
            const T *u = a.U[sp] + ((int64_t)co * S + ao) * S;
            for (int i = 0; i < a.A; ++i)
                if (o[i] != ao) h += u[o[i]];
            e.info = make_info(1, par & 1, ao, co);
            if (proton) e.local = a.tr_base[co * S + ao];
            else e.info = info_with_tcol(e.info, a.tr_idx[co * S + ao]);
            e.val = h;
        } else {
            // d == 4: (a<b) -> (c<d), operator a+_c a+_d a_b a_a on the ket
            int a1 = lowest_state(xa, W);
            flip(xa, a1);
            int b1 = lowest_state(xa, W);
            int c1 = lowest_state(xc, W);
            flip(xc, c1);
            int d1 = lowest_state(xc, W);
            int par = count_below(K, W, a1);
            flip(K, a1);
            par += count_below(K, W, b1);
            flip(K, b1);
            par += count_below(K, W, d1);
            flip(K, d1);
            par += count_below(K, W, c1);
            T v = a.C[sp][a.pair_row[c1 * S + d1] + a.pair_col[a1 * S + b1]];
            e.info = make_info(2, 0, a1, c1);
            e.val = (par & 1) ? -v : v;
        }
    }
    if (proton) {
        // the proton lists carry what the row kernels need about t (first
        // basis row, q, change of 2M) instead of t itself
        e.tgt = (int32_t)a.p_row_base[t];
        const int dslot = (a.twoM[t] - a.twoM[s]) / 2;
        e.info = info_with_partner(e.info, a.q[t], dslot);
    }
    return e;
}

// Each warp owns RW row determinants; the block's warps sweep the partner
// window in tiles of kTile determinants staged in shared memory (bits and
// 2M), so the window is read once per block.  Pass 0 counts the partners
// of every row and list; pass 1 writes their indices (the entries are
// evaluated afterwards by k_entries, one warp per row and list).  The window holds every
// determinant whose 2M is within 2K of a row's 2M (a single move changes
// 2M by at most 2K; a double move is kept only at equal 2M), and only the
// row's own 2M block when the sweep fills same-2M lists only.  Lanes take
// one partner each and a warp ballot per row and list keeps the partners
// in ascending order.
constexpr int kTile = 512;

template <class T, int W, int RW, int PASS>
__global__ void __launch_bounds__(256) k_filter(const FilterArgs<T> *jobs, const int64_t *job_blk, int njobs) {
    constexpr bool pass = PASS != 0;
    __shared__ uint64_t sbits[kTile * W];
    __shared__ int32_t sm2[kTile];
    int lo = 0, hi = njobs - 1;  // the job (one species list of one problem) of this block
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (job_blk[mid] <= (int64_t)blockIdx.x) lo = mid; else hi = mid - 1;
    }
    const FilterArgs<T> a = jobs[lo];  // by value: stores to ent cannot alias it
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t blk_row0 = ((int64_t)blockIdx.x - job_blk[lo]) * 8 * RW;
    const int64_t row0 = blk_row0 + (int64_t)wid * RW;
    const bool mO = a.modes & (1 << CONN_OUTER), m2 = a.modes & (1 << CONN_L2), m4 = a.modes & (1 << CONN_L4),
               mO4 = a.modes & (1 << CONN_O4);
    uint64_t bs[RW][kMaxWords];
    int ms[RW];
    int64_t out[RW][kModes];
    int cnt[RW][kModes];
#pragma unroll
    for (int i = 0; i < RW; ++i) {
        const int64_t s = row0 + i;
        const bool ok = s < a.n;
#pragma unroll
        for (int w = 0; w < kMaxWords; ++w) bs[i][w] = (ok && w < W) ? a.bits[s * W + w] : 0ull;
        ms[i] = ok ? a.twoM[s] : 0;
#pragma unroll
        for (int m = 0; m < kModes; ++m) {
            out[i][m] = (ok && pass && (a.modes >> m & 1)) ? a.ptr[m][s] : 0;
            cnt[i][m] = 0;
        }
    }
    // partner window of the block's rows (rows are sorted by 2M)
    const int64_t last = min(a.n - 1, blk_row0 + 8 * RW - 1);
    const int b0 = (a.twoM[blk_row0] - a.m2min) / 2, b1 = (a.twoM[last] - a.m2min) / 2;
    const int reach = (mO || m2) ? a.K : 0;
    (void)mO4;
    const int64_t t_lo = a.blk_start[max(b0 - reach, 0)];
    const int64_t t_hi = a.blk_start[min(b1 + reach + 1, a.nblk)];
    for (int64_t t0 = t_lo; t0 < t_hi; t0 += kTile) {
        const int nt = (int)min((int64_t)kTile, t_hi - t0);
        __syncthreads();
        for (int e = threadIdx.x; e < nt * W; e += blockDim.x) sbits[e] = a.bits[t0 * W + e];
        for (int e = threadIdx.x; e < nt; e += blockDim.x) sm2[e] = a.twoM[t0 + e];
        __syncthreads();
        for (int c0 = 0; c0 < nt; c0 += 32) {
            const int tl = c0 + lane;
            const bool tv = tl < nt;
            uint64_t bt[kMaxWords] = {};
#pragma unroll
            for (int w = 0; w < W; ++w) bt[w] = tv ? sbits[tl * W + w] : 0ull;
            const int mt = tv ? sm2[tl] : 0;
#pragma unroll
            for (int i = 0; i < RW; ++i) {
                int d = 0;
#pragma unroll
                for (int w = 0; w < W; ++w) d += __popcll(bs[i][w] ^ bt[w]);
                const bool sameM = mt == ms[i];
                const bool valid = tv && (row0 + i < a.n);
                const bool keep[kModes] = {mO && valid && d <= 2, m2 && valid && d <= 2,
                                           m4 && valid && d <= 4 && sameM, mO4 && valid && d == 4 && sameM};
#pragma unroll
                for (int m = 0; m < kModes; ++m) {
                    if (!(a.modes >> m & 1)) continue;   // uniform over the block
                    const unsigned bal = __ballot_sync(0xffffffffu, keep[m]);
                    if (pass && keep[m]) {
                        const int rank = __popc(bal & ((1u << lane) - 1u));
                        a.tgt[out[i][m] + rank] = (int32_t)(t0 + tl);
                    }
                    out[i][m] += __popc(bal);
                    cnt[i][m] += __popc(bal);
                }
            }
        }
    }
    if (!pass && lane == 0) {
#pragma unroll
        for (int i = 0; i < RW; ++i)
            if (row0 + i < a.n)
#pragma unroll
                for (int m = 0; m < kModes; ++m)
                    if (a.modes >> m & 1) a.count[m][row0 + i] = cnt[i][m];
    }
}

// Launch pass 0 (counts) or 1 (entries) for jobs sharing W, RW rows per warp.
template <class T, int W, int RW>
static void launch_filter(const std::vector<FilterArgs<T>> &jobs, int pass, cudaStream_t s) {
    if (jobs.empty()) return;
    std::vector<int64_t> blk(1, 0);
    for (auto &j : jobs) blk.push_back(blk.back() + (j.n + 8 * RW - 1) / (8 * RW));
    if (blk.back() == 0) return;
    if (blk.back() > INT32_MAX) fail(CI_ERR_CAPACITY, "species filter grid too large");
    DevBuf<FilterArgs<T>> dj(jobs.size());
    DevBuf<int64_t> db(blk.size());
    CI_CUDA(cudaMemcpyAsync(dj.ptr, jobs.data(), sizeof(FilterArgs<T>) * jobs.size(), cudaMemcpyHostToDevice, s));
    CI_CUDA(cudaMemcpyAsync(db.ptr, blk.data(), sizeof(int64_t) * blk.size(), cudaMemcpyHostToDevice, s));
    if (pass) launch("k_filter", k_filter<T, W, RW, 1>, (unsigned)blk.back(), 256, 0, s,
                     (const FilterArgs<T> *)dj.ptr, (const int64_t *)db.ptr, (int)jobs.size());
    else launch("k_filter_count", k_filter<T, W, RW, 0>, (unsigned)blk.back(), 256, 0, s,
                (const FilterArgs<T> *)dj.ptr, (const int64_t *)db.ptr, (int)jobs.size());
}

// Slater-Condon entries of every stored pair (s, tgt[e]) of the lists:
// one warp per row of a list, lanes over its entries.
template <class T, int W>
__global__ void __launch_bounds__(256) k_entries(const FilterArgs<T> *jobs, const int64_t *job_row, int njobs) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t rows = job_row[njobs];
    for (int64_t gr = warp; gr < rows; gr += nwarps) {
        int lo = 0, hi = njobs - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (job_row[mid] <= gr) lo = mid; else hi = mid - 1;
        }
        const FilterArgs<T> &a = jobs[lo];
        const int mode = __ffs(a.modes) - 1;
        const int64_t s = gr - job_row[lo];
        uint64_t bs[kMaxWords] = {};
#pragma unroll
        for (int w = 0; w < W; ++w) bs[w] = a.bits[s * W + w];
        const int64_t e1 = a.ptr[mode][s + 1];
        for (int64_t e = a.ptr[mode][s] + lane; e < e1; e += 32) {
            const int64_t t = a.tgt[e];
            uint64_t bt[kMaxWords] = {};
            int d = 0;
#pragma unroll
            for (int w = 0; w < W; ++w) {
                bt[w] = a.bits[t * W + w];
                d += __popcll(bs[w] ^ bt[w]);
            }
            a.ent[e] = make_entry<T>(a, mode, s, t, bs, bt, d);
        }
    }
}

template <class T, int W>
static void launch_entries(const std::vector<FilterArgs<T>> &jobs, cudaStream_t s) {
    if (jobs.empty()) return;
    std::vector<int64_t> off(1, 0);
    for (auto &j : jobs) off.push_back(off.back() + j.n);
    if (off.back() == 0) return;
    DevBuf<FilterArgs<T>> dj(jobs.size());
    DevBuf<int64_t> doff(off.size());
    CI_CUDA(cudaMemcpyAsync(dj.ptr, jobs.data(), sizeof(FilterArgs<T>) * jobs.size(), cudaMemcpyHostToDevice, s));
    CI_CUDA(cudaMemcpyAsync(doff.ptr, off.data(), sizeof(int64_t) * off.size(), cudaMemcpyHostToDevice, s));
    launch("k_entries", k_entries<T, W>, grid_for(off.back() * 32, 256, sm_count() * 8), 256, 0, s,
           (const FilterArgs<T> *)dj.ptr, (const int64_t *)doff.ptr, (int)jobs.size());
}

template <class T>
static void launch_entries_all(const std::vector<FilterArgs<T>> (&ejw)[kMaxWords], cudaStream_t s) {
    launch_entries<T, 1>(ejw[0], s);
    launch_entries<T, 2>(ejw[1], s);
    launch_entries<T, 3>(ejw[2], s);
    launch_entries<T, 4>(ejw[3], s);
}

template <class T>
static void filter_pass(const std::vector<FilterArgs<T>> &jobs, int pass, cudaStream_t s) {
    // rows per warp: 2 only when that still leaves every SM 16 blocks of
    // 8 warps (the sweep is latency bound, so more warps beat more reuse)
    std::vector<FilterArgs<T>> jw[kMaxWords];
    int64_t rows = 0;
    for (auto &j : jobs) {
        if (j.n == 0) continue;
        jw[j.W - 1].push_back(j);
        rows += j.n;
    }
    const bool wide = rows >= (int64_t)sm_count() * 16 * 16;
    if (wide) {
        launch_filter<T, 1, 2>(jw[0], pass, s); launch_filter<T, 2, 2>(jw[1], pass, s);
        launch_filter<T, 3, 2>(jw[2], pass, s); launch_filter<T, 4, 2>(jw[3], pass, s);
    } else {
        launch_filter<T, 1, 1>(jw[0], pass, s); launch_filter<T, 2, 1>(jw[1], pass, s);
        launch_filter<T, 3, 1>(jw[2], pass, s); launch_filter<T, 4, 1>(jw[3], pass, s);
    }
}

// Segment tables of one problem's lists (c: a cap on q, ds: a 2M slot,
// 2M(partner) = 2M(row) + 2(ds - K); entries are sorted by (2M, q, bits)).
//   seg2[n][ds][c]: end (relative to ptr[n]) of the L2 entries whose key
//   (2M, q) is <= (2M_n + 2(ds-K), c); with no Nmax cut the q part is ignored.
//   seg4[n][c]: end (relative) of the L4 entries with q <= c (all same 2M).
//   qmin2[n][ds]: q of the first L2 entry of slot ds (its smallest q), nq if
//   the slot is empty.
//   oseg2[p][ds][c], oseg4[p][c]: the same ends for the proton lists O2 and
//   O4, read from the packed (q, slot) of each entry.
// A row (p, n) then takes, per 2M slot of the proton partners, the q-prefix
// that can still meet a neutron partner under the Nmax cut.
template <class T>
struct SegJob {
    int64_t n, np;
    int nds, nq, K, cut;
    const int64_t *p2, *p4, *po, *po4;
    const ConnEntry<T> *e2, *e4, *eo, *eo4;
    const int32_t *twoM, *q;
    int32_t *seg2, *seg4, *qmin2, *oseg2, *oseg4;
};

// first entry of [lo, hi) whose key exceeds (slot, c); key(e) = (slot, q)
template <class T, class KeyF>
__device__ __forceinline__ int64_t upper_key(const ConnEntry<T> *e, int64_t lo, int64_t hi, int slot, int c, bool cut,
                                             KeyF key) {
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        int ks, kq;
        key(e[mid], ks, kq);
        const bool le = ks < slot || (ks == slot && (!cut || kq <= c));
        if (le) lo = mid + 1; else hi = mid;
    }
    return lo;
}

template <class T>
__global__ void k_seg(const SegJob<T> *jobs, const int64_t *job_off, int njobs) {
    const int64_t total = job_off[njobs];
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int jl = 0, jh = njobs - 1;
        while (jl < jh) {
            int mid = (jl + jh + 1) >> 1;
            if (job_off[mid] <= e) jl = mid; else jh = mid - 1;
        }
        const SegJob<T> &j = jobs[jl];
        int64_t r = e - job_off[jl];
        const int64_t sz2 = j.n * j.nds * j.nq, sz4 = j.n * j.nq, szm = j.n * j.nds;
        const int64_t szo2 = j.np * j.nds * j.nq;
        const bool cut = j.cut != 0;
        if (r < sz2) {   // seg2
            const int c = (int)(r % j.nq);
            const int ds = (int)((r / j.nq) % j.nds);
            const int64_t s = r / ((int64_t)j.nq * j.nds);
            const int mt = j.twoM[s] + 2 * (ds - j.K);
            const int64_t end = upper_key(j.e2, j.p2[s], j.p2[s + 1], mt, c, cut,
                                          [&](const ConnEntry<T> &x, int &ks, int &kq) {
                                              ks = j.twoM[x.tgt]; kq = j.q[x.tgt]; });
            j.seg2[r] = (int32_t)(end - j.p2[s]);
            continue;
        }
        r -= sz2;
        if (r < sz4) {   // seg4
            const int c = (int)(r % j.nq);
            const int64_t s = r / j.nq;
            int64_t lo = j.p4[s], hi = j.p4[s + 1];
            if (cut) {
                while (lo < hi) {
                    const int64_t mid = (lo + hi) >> 1;
                    if (j.q[j.e4[mid].tgt] <= c) lo = mid + 1; else hi = mid;
                }
            } else {
                lo = hi;
            }
            j.seg4[r] = (int32_t)(lo - j.p4[s]);
            continue;
        }
        r -= sz4;
        if (r < szm) {   // qmin2: first L2 entry of the slot
            const int ds = (int)(r % j.nds);
            const int64_t s = r / j.nds;
            const int mt = j.twoM[s] + 2 * (ds - j.K);
            const int64_t b = upper_key(j.e2, j.p2[s], j.p2[s + 1], mt - 2, 0, false,
                                        [&](const ConnEntry<T> &x, int &ks, int &kq) {
                                            ks = j.twoM[x.tgt]; kq = 0; });
            int qm = j.nq;
            if (b < j.p2[s + 1] && j.twoM[j.e2[b].tgt] == mt) qm = cut ? j.q[j.e2[b].tgt] : 0;
            j.qmin2[r] = qm;
            continue;
        }
        r -= szm;
        if (r < szo2) {  // oseg2: keys from the packed proton entries
            const int c = (int)(r % j.nq);
            const int ds = (int)((r / j.nq) % j.nds) - j.K;
            const int64_t s = r / ((int64_t)j.nq * j.nds);
            const int64_t end = upper_key(j.eo, j.po[s], j.po[s + 1], ds, c, cut,
                                          [&](const ConnEntry<T> &x, int &ks, int &kq) {
                                              ks = info_dslot(x.info); kq = info_q(x.info); });
            j.oseg2[r] = (int32_t)(end - j.po[s]);
            continue;
        }
        r -= szo2;
        {                // oseg4: all same 2M, q-prefix
            const int c = (int)(r % j.nq);
            const int64_t s = r / j.nq;
            const int64_t end = upper_key(j.eo4, j.po4[s], j.po4[s + 1], 0, c, cut,
                                          [&](const ConnEntry<T> &x, int &ks, int &kq) {
                                              ks = 0; kq = info_q(x.info); });
            j.oseg4[r] = (int32_t)(end - j.po4[s]);
        }
    }
}

// Cross ranks of the same-2M proton partners (one warp per proton row):
// for an O2 entry of 2M slot 0, the number of the row's O4 entries with a
// smaller partner index; for an O4 entry, the number of the row's slot-0 O2
// entries with a smaller partner index.  The fill merges the two lists by
// column with them.
struct XrankJob {
    int64_t np;
    int K, nq;
    const int64_t *po, *po4;
    const int32_t *oseg2;
    const int32_t *tgt;   // partner index per entry
    int32_t *xr;
};

__device__ __forceinline__ int64_t lower_tgt(const int32_t *tgt, int64_t lo, int64_t hi, int32_t key) {
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (tgt[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__global__ void k_xrank(const XrankJob *jobs, const int64_t *job_row, int njobs) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t gr = warp; gr < job_row[njobs]; gr += nwarps) {
        int lo = 0, hi = njobs - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (job_row[mid] <= gr) lo = mid; else hi = mid - 1;
        }
        const XrankJob &j = jobs[lo];
        const int64_t p = gr - job_row[lo];
        const int32_t *os = j.oseg2 + p * (2 * j.K + 1) * j.nq;
        const int64_t a0 = j.po[p] + (j.K == 0 ? 0 : os[(j.K - 1) * j.nq + j.nq - 1]);
        const int64_t a1 = j.po[p] + os[j.K * j.nq + j.nq - 1];
        const int64_t b0 = j.po4[p], b1 = j.po4[p + 1];
        for (int64_t e = a0 + lane; e < a1; e += 32) j.xr[e] = (int32_t)(lower_tgt(j.tgt, b0, b1, j.tgt[e]) - b0);
        for (int64_t e = b0 + lane; e < b1; e += 32) j.xr[e] = (int32_t)(lower_tgt(j.tgt, a0, a1, j.tgt[e]) - a0);
    }
}

template <class T>
static FilterArgs<T> filter_job(Problem *p, int species, int modes, const Tables<T> *tab = nullptr) {
    SpeciesList &sp = p->sp[species];
    const Tables<T> &t = tab ? *tab : p->tables<T>();
    FilterArgs<T> a{};
    a.n = sp.n; a.A = sp.A; a.S = p->S; a.W = sp.W; a.modes = modes;
    a.bits = sp.d_bits.ptr; a.twoM = sp.d_twoM.ptr; a.local = sp.d_local.ptr; a.occ = sp.d_occ.ptr;
    a.q = sp.d_q.ptr;
    a.blk_start = sp.d_blk_start.ptr; a.m2min = sp.m2min; a.nblk = sp.nblk; a.K = p->K;
    a.p_row_base = p->d_p_row_base.ptr;
    a.eps = t.eps.ptr;
    a.U[0] = t.Upp.ptr; a.D[0] = t.Dpp.ptr; a.C[0] = t.Cpp.ptr;
    a.U[1] = t.Unn.ptr; a.D[1] = t.Dnn.ptr; a.C[1] = t.Cnn.ptr;
    a.pair_row = p->like_row.ptr; a.pair_col = p->like_col.ptr;
    a.tr_base = p->tr_base.ptr; a.tr_idx = p->tr_idx.ptr;
    return a;
}

// Species connectivity of every problem of ps (Fig. 1, tile filter): count
// pass, one scan over all lists, one allocation, fill pass, segment tables.
template <class T>
void species_filter_group(const std::vector<Problem *> &ps_in, cudaStream_t s) {
    std::vector<Problem *> ps;
    for (Problem *p : ps_in)
        if (!p->conn<T>().ready) ps.push_back(p);
    if (ps.empty()) return;
    for (Problem *p : ps) enumerate_basis(p, s);
    stage_tables_group<T>(ps, s);
    // four lists per problem, their counts side by side in one array; one
    // sweep per species list (one per problem when the species coincide)
    std::vector<FilterArgs<T>> jobs;
    std::vector<ConnList<T> *> lists;
    std::vector<int> list_job, list_mode;
    std::vector<int64_t> cnt_off(1, 0);
    for (Problem *p : ps) {
        Connectivity<T> &c = p->conn<T>();
        const bool same = p->Z == p->N;
        const int first = (int)jobs.size();
        const int pmodes = (1 << CONN_OUTER) | (1 << CONN_O4), nmodes = (1 << CONN_L2) | (1 << CONN_L4);
        jobs.push_back(filter_job<T>(p, 0, same ? pmodes | nmodes : pmodes));
        if (!same) jobs.push_back(filter_job<T>(p, 1, nmodes));
        ConnList<T> *ls[kModes] = {&c.outer, &c.l2, &c.l4, &c.outer4};
        for (int m = 0; m < kModes; ++m) {
            const bool prot = m == CONN_OUTER || m == CONN_O4;
            lists.push_back(ls[m]);
            list_job.push_back(prot || same ? first : first + 1);
            list_mode.push_back(m);
            cnt_off.push_back(cnt_off.back() + (prot ? p->sp[0].n : p->sp[1].n));
        }
    }
    const int64_t ncnt = cnt_off.back();
    DevBuf<int32_t> cnt((size_t)ncnt);
    auto offs = std::make_shared<DevBuf<int64_t>>((size_t)ncnt + 1);
    for (size_t i = 0; i < lists.size(); ++i) jobs[list_job[i]].count[list_mode[i]] = cnt.ptr + cnt_off[i];
    filter_pass<T>(jobs, 0, s);
    exclusive_scan_i32(cnt.ptr, ncnt, offs->ptr, ps[0]->scan_scratch, s);
    // list boundaries: hb[i] = offs[cnt_off[i]]
    std::vector<int64_t> hb = gather_i64(offs->ptr, cnt_off, s);
    auto ents = std::make_shared<DevBuf<ConnEntry<T>>>((size_t)hb.back());
    auto tgts = std::make_shared<DevBuf<int32_t>>((size_t)hb.back());
    auto xrs = std::make_shared<DevBuf<int32_t>>((size_t)hb.back());
    for (size_t i = 0; i < lists.size(); ++i) {
        ConnList<T> &L = *lists[i];
        L.ptr_buf = offs;
        L.ent_buf = ents;
        L.tgt_buf = tgts;
        L.tgt = tgts->ptr;
        L.xr_buf = xrs;
        L.xr = xrs->ptr;
        L.ptr = offs->ptr + cnt_off[i];
        L.ent = ents->ptr;
        L.n = cnt_off[i + 1] - cnt_off[i];
        L.first = hb[i];
        L.total = hb[i + 1] - hb[i];
        FilterArgs<T> &j = jobs[list_job[i]];
        j.ptr[list_mode[i]] = L.ptr;
        j.ent = L.ent;
        j.tgt = tgts->ptr;
    }
    filter_pass<T>(jobs, 1, s);
    std::vector<FilterArgs<T>> ejw[kMaxWords];
    for (size_t i = 0; i < lists.size(); ++i) {
        FilterArgs<T> j = jobs[list_job[i]];
        j.modes = 1 << list_mode[i];
        j.n = lists[i]->n;
        ejw[j.W - 1].push_back(j);
    }
    launch_entries_all<T>(ejw, s);
    // segment tables
    std::vector<SegJob<T>> sj;
    std::vector<int64_t> soff(1, 0);
    for (Problem *p : ps) {
        Connectivity<T> &c = p->conn<T>();
        SpeciesList &P = p->sp[0], &Nn = p->sp[1];
        if (P.nq != Nn.nq) fail(CI_ERR_INTERNAL, "species q ranges differ");
        const int nq = Nn.nq, nds = p->nds;
        c.seg2.alloc((size_t)Nn.n * nds * nq);
        c.seg4.alloc((size_t)Nn.n * nq);
        c.qmin2.alloc((size_t)Nn.n * nds);
        c.oseg2.alloc((size_t)P.n * nds * nq);
        c.oseg4.alloc((size_t)P.n * nq);
        SegJob<T> j{};
        j.n = Nn.n; j.np = P.n; j.nds = nds; j.nq = nq; j.K = p->K; j.cut = p->nmax >= 0;
        j.p2 = c.l2.ptr; j.p4 = c.l4.ptr; j.po = c.outer.ptr; j.po4 = c.outer4.ptr;
        j.e2 = c.l2.ent; j.e4 = c.l4.ent; j.eo = c.outer.ent; j.eo4 = c.outer4.ent;
        j.twoM = Nn.d_twoM.ptr; j.q = Nn.d_q.ptr;
        j.seg2 = c.seg2.ptr; j.seg4 = c.seg4.ptr; j.qmin2 = c.qmin2.ptr; j.oseg2 = c.oseg2.ptr; j.oseg4 = c.oseg4.ptr;
        const int64_t w = Nn.n * nds * nq + Nn.n * nq + Nn.n * nds + P.n * nds * nq + P.n * nq;
        if (w == 0) continue;
        sj.push_back(j);
        soff.push_back(soff.back() + w);
    }
    if (!sj.empty()) {
        DevBuf<SegJob<T>> dsj(sj.size());
        DevBuf<int64_t> dso(soff.size());
        CI_CUDA(cudaMemcpyAsync(dsj.ptr, sj.data(), sizeof(SegJob<T>) * sj.size(), cudaMemcpyHostToDevice, s));
        CI_CUDA(cudaMemcpyAsync(dso.ptr, soff.data(), sizeof(int64_t) * soff.size(), cudaMemcpyHostToDevice, s));
        launch("k_seg", k_seg<T>, grid_for(soff.back(), 256, sm_count() * 16), 256, 0, s, (const SegJob<T> *)dsj.ptr,
               (const int64_t *)dso.ptr, (int)sj.size());
    }
    {
        std::vector<XrankJob> xj;
        std::vector<int64_t> xoff(1, 0);
        for (Problem *p : ps) {
            Connectivity<T> &c = p->conn<T>();
            if (p->sp[0].n == 0) continue;
            XrankJob j{};
            j.np = p->sp[0].n; j.K = p->K; j.nq = p->sp[0].nq;
            j.po = c.outer.ptr; j.po4 = c.outer4.ptr; j.oseg2 = c.oseg2.ptr;
            j.tgt = tgts->ptr; j.xr = xrs->ptr;
            xj.push_back(j);
            xoff.push_back(xoff.back() + j.np);
        }
        if (!xj.empty()) {
            DevBuf<XrankJob> dxj(xj.size());
            DevBuf<int64_t> dxo(xoff.size());
            CI_CUDA(cudaMemcpyAsync(dxj.ptr, xj.data(), sizeof(XrankJob) * xj.size(), cudaMemcpyHostToDevice, s));
            CI_CUDA(cudaMemcpyAsync(dxo.ptr, xoff.data(), sizeof(int64_t) * xoff.size(), cudaMemcpyHostToDevice, s));
            launch("k_xrank", k_xrank, grid_for(xoff.back() * 32, 256, sm_count() * 8), 256, 0, s,
                   (const XrankJob *)dxj.ptr, (const int64_t *)dxo.ptr, (int)xj.size());
        }
    }
    for (Problem *p : ps) p->conn<T>().ready = true;
}

template <class T>
void operator_entries(Problem *p, const Tables<T> &t, ConnEntry<T> *ents, cudaStream_t s) {
    Connectivity<T> &c = p->conn<T>();
    if (!c.ready) fail(CI_ERR_STATE, "species connectivity not built");
    std::vector<FilterArgs<T>> ejw[kMaxWords];
    const ConnList<T> *ls[kModes] = {&c.outer, &c.l2, &c.l4, &c.outer4};
    for (int m = 0; m < kModes; ++m) {
        const bool prot = m == CONN_OUTER || m == CONN_O4;
        FilterArgs<T> j = filter_job<T>(p, prot ? 0 : 1, 1 << m, &t);
        j.n = ls[m]->n;
        j.ptr[m] = ls[m]->ptr;
        j.ent = ents;
        j.tgt = const_cast<int32_t *>(ls[m]->tgt);
        ejw[j.W - 1].push_back(j);
    }
    launch_entries_all<T>(ejw, s);
}

template void operator_entries<float>(Problem *, const Tables<float> &, ConnEntry<float> *, cudaStream_t);
template void operator_entries<double>(Problem *, const Tables<double> &, ConnEntry<double> *, cudaStream_t);
template void species_filter_group<float>(const std::vector<Problem *> &, cudaStream_t);
template void species_filter_group<double>(const std::vector<Problem *> &, cudaStream_t);


}  // namespace ci
